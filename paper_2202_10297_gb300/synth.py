"""Seeded synthetic inputs shaped like the workloads of arXiv 2202.10297's operators.

This module only draws random numbers (numpy PCG64); it holds none of the
adjoint arithmetic.  Tests feed the same arrays to the CUDA library and to
the FP64 oracle, and the benchmark times the library on them.  The default
seed of workload ``i`` is ``SEED_BASE + i``.

Recipes (sizes are arguments; the benchmark uses the sizes in its config):
  prod_reduce  a ~ U[0.5, 1.5) FP64 with exactly ``nzeros`` entries set to 0
               at seeded distinct positions; ybar = 1.
  linrec       a ~ U[0.9, 1.0], b ~ N(0,1), cotangents ybar_A, ybar_B ~ N(0,1).
  normal       x ~ N(0,1) (the + and max scans, hist values, k-means).
  hist         vals ~ N(0,1) FP32, bins uniform on [0, m) or bounded
               Zipf(s=1.1) over ranks 1..m (bin = rank - 1) by inverse CDF;
               a fraction (1 %) of the indices is moved out of range, half
               below 0 and half at or above m; hsbar ~ N(0,1).
  scatter      is = the first m values of a seeded permutation of [0, n)
               (a keyed Feistel bijection, so no duplicates), optionally sorted.
  batch        segment lengths round(2^U[8, 20]), FP32/FP64 by a seeded coin,
               each with a product-reduce input (0, 1 or 2 zeros) and a
               linear-recurrence input.
"""
import numpy as np

SEED_BASE = 20220221


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _fill(gen, n, dtype, kind, lo=0.0, hi=1.0, chunk=1 << 24):
    """Draw n samples in chunks (bounded temporaries for 2^28-element arrays)."""
    out = np.empty(n, dtype=dtype)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        if kind == "normal":
            out[s:e] = gen.standard_normal(e - s, dtype=np.float64)
        else:
            out[s:e] = gen.uniform(lo, hi, e - s)
    return out


def normal(n, dtype=np.float32, seed=SEED_BASE + 1):
    return _fill(rng(seed), n, dtype, "normal")


def uniform(n, lo, hi, dtype=np.float32, seed=SEED_BASE + 1):
    return _fill(rng(seed), n, dtype, "uniform", lo, hi)


def prod_reduce(n, nzeros, dtype=np.float64, seed=SEED_BASE + 0):
    """a ~ U[0.5, 1.5) with exactly ``nzeros`` zeros at seeded positions."""
    g = rng(seed)
    a = _fill(g, n, dtype, "uniform", 0.5, 1.5)
    zpos = np.sort(g.choice(n, size=nzeros, replace=False)) if nzeros else np.zeros(0, np.int64)
    a[zpos] = 0
    return a, zpos


def linrec(n, dtype=np.float32, seed=SEED_BASE + 1):
    """(a, b, ybar_a, ybar_b) for the linear-recurrence scan."""
    g = rng(seed)
    a = _fill(g, n, dtype, "uniform", 0.9, 1.0)
    b = _fill(g, n, dtype, "normal")
    ya = _fill(g, n, dtype, "normal")
    yb = _fill(g, n, dtype, "normal")
    return a, b, ya, yb


def zipf_bins(gen, n, m, s=1.1, chunk=1 << 24):
    """Bins 0..m-1 drawn from a bounded Zipf(s) over ranks 1..m, by inverse CDF."""
    w = np.arange(1, m + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    out = np.empty(n, dtype=np.int64)
    for st in range(0, n, chunk):
        e = min(n, st + chunk)
        u = gen.random(e - st)
        out[st:e] = np.minimum(np.searchsorted(cdf, u, side="right"), m - 1)
    return out


def hist(n, m, dist="uniform", oor=0.01, itype=np.int32, seed=SEED_BASE + 2):
    """(vals FP32, inds, hsbar FP32) for reduce_by_index."""
    g = rng(seed)
    vals = _fill(g, n, np.float32, "normal")
    if dist == "uniform":
        inds = g.integers(0, m, size=n, dtype=np.int64)
    elif dist == "zipf":
        inds = zipf_bins(g, n, m)
    else:
        raise ValueError(dist)
    if oor > 0:
        sel = np.flatnonzero(g.random(n) < oor)
        half = sel.size // 2
        inds[sel[:half]] = -1 - g.integers(0, 1 << 20, size=half)
        inds[sel[half:]] = m + g.integers(0, 1 << 20, size=sel.size - half)
    hsbar = _fill(g, m, np.float32, "normal")
    return vals, inds.astype(itype), hsbar


def _mix(x, key):
    x = (x ^ key) * np.uint64(0x9E3779B97F4A7C15)
    x ^= x >> np.uint64(31)
    x = x * np.uint64(0xBF58476D1CE4E5B9)
    x ^= x >> np.uint64(29)
    return x


def permutation_prefix(n, m, seed, chunk=1 << 24):
    """The first m values of a seeded permutation of [0, n) (n <= 2^62).

    A 4-round balanced Feistel network on 2*h bits with keyed mixing is a
    bijection of [0, 2^(2h)); cycle-walking restricts it to [0, n).
    """
    g = rng(seed)
    bits = max(2, int(np.ceil(np.log2(max(n, 2)))))
    h = (bits + 1) // 2
    mask = np.uint64((1 << h) - 1)
    keys = g.integers(0, 1 << 62, size=4, dtype=np.int64).astype(np.uint64)

    def perm(x):
        L = x >> np.uint64(h)
        R = x & mask
        for k in keys:
            L, R = R, L ^ (_mix(R, k) & mask)
        return (L << np.uint64(h)) | R

    out = np.empty(m, dtype=np.int64)
    with np.errstate(over="ignore"):
        for s in range(0, m, chunk):
            e = min(m, s + chunk)
            y = perm(np.arange(s, e, dtype=np.uint64))
            bad = y >= np.uint64(n)
            while bad.any():
                y[bad] = perm(y[bad])
                bad = y >= np.uint64(n)
            out[s:e] = y.astype(np.int64)
    return out


def scatter(n, m, sort=False, itype=np.int32, seed=SEED_BASE + 2):
    """(is, ysbar FP32[n], xs_saved FP32[m]) for the scatter adjoint."""
    is_ = permutation_prefix(n, m, seed)
    if sort:
        is_ = np.sort(is_)
    g = rng(seed + 1000)
    ysbar = _fill(g, n, np.float32, "normal")
    xs_saved = _fill(g, m, np.float32, "normal")
    return is_.astype(itype), ysbar, xs_saved


def map_acc(nj, na, width=1, itype=np.int32, seed=SEED_BASE + 4):
    """(as FP32[na*width], is[nj], ws FP32[nj*width], xsbar FP32[nj])."""
    g = rng(seed)
    as_ = _fill(g, na * width, np.float32, "normal")
    is_ = g.integers(0, na, size=nj, dtype=np.int64).astype(itype)
    ws = _fill(g, nj * width, np.float32, "normal")
    xsbar = _fill(g, nj, np.float32, "normal")
    return as_, is_, ws, xsbar


def kmeans(N, d, k, seed=SEED_BASE + 4):
    """(X FP32[N, d], C FP32[k, d]) with N(0,1) entries."""
    g = rng(seed)
    X = _fill(g, N * d, np.float32, "normal").reshape(N, d)
    Cm = _fill(g, k * d, np.float32, "normal").reshape(k, d)
    return X, Cm


def batch_plan(nseg, lo=8, hi=20, seed=SEED_BASE + 3):
    """Per segment: length, dtype code (0 = FP32, 1 = FP64), zero count."""
    g = rng(seed)
    lens = np.rint(2.0 ** g.uniform(lo, hi, nseg)).astype(np.int64)
    dts = (g.random(nseg) < 0.5).astype(np.int32)
    zs = g.integers(0, 3, size=nseg).astype(np.int32)
    return lens, dts, zs
