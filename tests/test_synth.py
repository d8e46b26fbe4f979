"""The seeded synthetic inputs have the shapes, ranges and structure the
workloads state (no GPU): reproducible per seed, duplicate-free scatter
indices, 1% out-of-range reduce_by_index indices split between negative and
>= m, Zipf(1.1) bin frequencies, and the stated value ranges."""
import numpy as np

from paper_2202_10297_gb300 import synth


def test_same_seed_same_inputs():
    a1 = synth.linrec(1000, seed=5)
    a2 = synth.linrec(1000, seed=5)
    for x, y in zip(a1, a2):
        np.testing.assert_array_equal(x, y)
    assert not np.array_equal(synth.linrec(1000, seed=6)[0], a1[0])


def test_value_ranges():
    a, b, ya, yb = synth.linrec(1 << 16, np.float64)
    assert a.min() >= 0.9 and a.max() <= 1.0
    assert abs(b.mean()) < 0.05 and abs(b.std() - 1) < 0.05
    x, zpos = synth.prod_reduce(4096, 2)
    assert (x == 0).sum() == 2 and np.all(x[zpos] == 0)
    nz = x[x != 0]
    assert nz.min() >= 0.5 and nz.max() <= 1.5


def test_scatter_indices_are_a_permutation_prefix():
    n, m = 1 << 20, 1 << 16
    is_, ysbar, xs = synth.scatter(n, m)
    assert is_.shape == (m,) and ysbar.shape == (n,) and xs.shape == (m,)
    assert is_.min() >= 0 and is_.max() < n
    assert np.unique(is_).size == m  # duplicate-free
    srt, _, _ = synth.scatter(n, m, sort=True)
    np.testing.assert_array_equal(srt, np.sort(is_))


def test_hist_out_of_range_and_zipf():
    n, m = 1 << 20, 256
    vals, inds, hsbar = synth.hist(n, m, "zipf")
    oor = (inds < 0) | (inds >= m)
    assert abs(oor.mean() - 0.01) < 0.002
    assert abs((inds < 0).sum() - (inds >= m).sum()) <= 1  # half below, half above
    f = np.bincount(inds[~oor], minlength=m).astype(np.float64)
    # bounded Zipf(1.1): frequency of rank r proportional to r^-1.1
    assert abs(f[0] / f[1] - 2 ** 1.1) < 0.05 * 2 ** 1.1
    assert abs(f[0] / f[9] - 10 ** 1.1) < 0.15 * 10 ** 1.1
    _, u, _ = synth.hist(n, m, "uniform")
    fu = np.bincount(u[(u >= 0) & (u < m)], minlength=m)
    assert fu.min() > 0.8 * fu.mean() and fu.max() < 1.2 * fu.mean()


def test_batch_plan_lengths_and_kmeans_shapes():
    lens, dts, zs = synth.batch_plan(4096)
    assert lens.min() >= 2 ** 8 and lens.max() <= 2 ** 20
    assert set(np.unique(dts)) <= {0, 1} and set(np.unique(zs)) <= {0, 1, 2}
    X, C = synth.kmeans(1000, 32, 256)
    assert X.shape == (1000, 32) and C.shape == (256, 32) and X.dtype == np.float32
