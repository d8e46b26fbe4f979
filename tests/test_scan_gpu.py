"""GPU parity of the scan VJP (Sec. 5.2) against the FP64 oracle, through the C ABI.

Tolerances (relative L2 against the FP64 oracle on the same inputs):
FP32 1e-4 (1e-3 for scans longer than 2^24 elements), FP64 1e-12.
Record positions of max/min scans (where the adjoint is nonzero) must
match exactly.
"""
import numpy as np
import pytest
import torch

from paper_2202_10297_gb300 import synth

pytestmark = pytest.mark.gpu

TILE_F32 = 4 * 256 * 4  # elements per tile of the width-1 FP32 scan
SIZES = [1, 2, 3, 5, 17, 1000, TILE_F32 - 1, TILE_F32, TILE_F32 + 1, 3 * TILE_F32 + 5, 65536 + 7,
         200003]


def rel_l2(x, ref):
    x = np.asarray(x, np.float64)
    ref = np.asarray(ref, np.float64)
    d = np.linalg.norm(ref)
    return float(np.linalg.norm(x - ref) / (d if d > 0 else 1.0))


def tol(dt, n):
    if dt == np.float64:
        return 1e-12
    return 1e-3 if n > (1 << 24) else 1e-4


@pytest.fixture(scope="module")
def A():
    from paper_2202_10297_gb300 import adpar
    adpar.lib()
    return adpar


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def inputs(op, n, dt, seed):
    g = synth.rng(seed)
    if op == "mul":
        a = g.uniform(0.5, 1.5, n).astype(dt)
        if n > 10:
            a[g.choice(n, size=2, replace=False)] = 0  # zeros are safe: no division
    elif op in ("min", "max"):
        a = (np.round(g.standard_normal(n) * 8) / 8).astype(dt)  # forced ties
    else:
        a = g.standard_normal(n).astype(dt)
    y = g.standard_normal(n).astype(dt)
    return a, y


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["add", "mul", "min", "max"])
@pytest.mark.parametrize("n", SIZES)
def test_scan_vjp_width1(A, oracle, op, dt, n):
    a, y = inputs(op, n, dt, seed=n * 7 + len(op))
    ys = torch.empty(n, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
    ab, _, work = A.adpar_vjp_scan(op, dev(a), dev(y), ys_a=ys)
    torch.cuda.synchronize()
    assert A.adpar_workspace_status(work) == A.OK
    ref, _, rys, _ = oracle.scan_vjp(op, a, y)
    got = ab.cpu().numpy()
    assert rel_l2(got, ref) < tol(dt, n), (op, n, rel_l2(got, ref))
    assert rel_l2(ys.cpu().numpy(), rys) < tol(dt, n)
    if op in ("min", "max"):
        np.testing.assert_array_equal(got != 0, ref != 0)  # record positions, bit-exact


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 2, 7, 2047, 2048, 2049, 8192 + 3, 100001])
def test_scan_vjp_linrec(A, oracle, dt, n):
    a, b, ya, yb = synth.linrec(n, dt, seed=n)
    ysa = torch.empty(n, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
    ysb = torch.empty_like(ysa)
    ab, bb, _ = A.adpar_vjp_scan("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb), ys_a=ysa, ys_b=ysb)
    rab, rbb, rya, ryb = oracle.scan_vjp("linrec", a, ya, b, yb)
    assert rel_l2(ab.cpu().numpy(), rab) < tol(dt, n)
    assert rel_l2(bb.cpu().numpy(), rbb) < tol(dt, n)
    assert rel_l2(ysa.cpu().numpy(), rya) < tol(dt, n)
    assert rel_l2(ysb.cpu().numpy(), ryb) < tol(dt, n)


@pytest.mark.parametrize("op", ["add", "max", "linrec"])
def test_scan_vjp_accumulate(A, oracle, op):
    n = 50000
    dt = np.float64
    a, y = inputs(op, n, dt, seed=3)
    base = synth.normal(n, dt, seed=4)
    if op == "linrec":
        a, b, ya, yb = synth.linrec(n, dt, seed=5)
        ab0, bb0 = dev(base), dev(base[::-1].copy())
        A.adpar_vjp_scan(op, dev(a), dev(ya), b=dev(b), ybar_b=dev(yb), abar=ab0, bbar=bb0, accumulate=True)
        rab, rbb, _, _ = oracle.scan_vjp(op, a, ya, b, yb, abar=base, bbar=base[::-1].copy())
        assert rel_l2(ab0.cpu().numpy(), rab) < 1e-12
        assert rel_l2(bb0.cpu().numpy(), rbb) < 1e-12
    else:
        ab0 = dev(base)
        A.adpar_vjp_scan(op, dev(a), dev(y), abar=ab0, accumulate=True)
        ref, _, _, _ = oracle.scan_vjp(op, a, y, abar=base)
        assert rel_l2(ab0.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("op", ["add", "mul", "max", "linrec"])
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_primal_scan(A, oracle, op, dt):
    n = 123457
    if op == "linrec":
        a, b, _, _ = synth.linrec(n, dt, seed=6)
        ya, yb, _ = A.adpar_scan(op, dev(a), b=dev(b))
        _, _, rya, ryb = oracle.scan_vjp(op, a, np.zeros(n), b, np.zeros(n))
        assert rel_l2(ya.cpu().numpy(), rya) < tol(dt, n)
        assert rel_l2(yb.cpu().numpy(), ryb) < tol(dt, n)
    else:
        a, _ = inputs(op, n, dt, seed=8)
        ya, _, _ = A.adpar_scan(op, dev(a))
        _, _, rya, _ = oracle.scan_vjp(op, a, np.zeros(n))
        assert rel_l2(ya.cpu().numpy(), rya) < tol(dt, n)


@pytest.mark.parametrize("op", ["mul", "linrec"])
@pytest.mark.parametrize("n", [1, 2047, 2049, 3 * 2048 + 5, 4 * 4096 + 3, 100001])
def test_fp64_factored_and_minimal_workspace_paths(A, oracle, op, n):
    """With the recomputed ys requested, FP64 MUL reads the factored forward
    result when the workspace has room for it and both operators re-form the
    primal prefixes in the return sweep when it has only the minimal size:
    every path matches the oracle, with the recomputed ys and with
    accumulation into existing adjoints."""
    dt = np.float64
    code = A.OPS[op]
    if op == "linrec":
        a, b, ya, yb = synth.linrec(n, dt, seed=n + 11)
    else:
        a, ya = inputs("mul", n, dt, seed=n + 11)
        b = yb = None
    base = synth.normal(n, dt, seed=12)
    base_b = base[::-1].copy() if op == "linrec" else None
    rab, rbb, rya, ryb = oracle.scan_vjp(op, a, ya, b, yb, abar=base, bbar=base_b)
    full = A.adpar_workspace_size(A.RULE_SCAN, code, A.F64, n)
    minimal = A.adpar_workspace_size(A.RULE_SCAN | A.WS_MINIMAL, code, A.F64, n)
    assert full >= minimal + (8 * n if op == "mul" else 0)
    for nbytes in (full, minimal):
        work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        ab0 = dev(base)
        bb0 = dev(base_b) if op == "linrec" else None
        ysa = torch.empty(n, dtype=torch.float64, device="cuda")
        ysb = torch.empty_like(ysa) if op == "linrec" else None
        A.adpar_vjp_scan(op, dev(a), dev(ya), b=None if b is None else dev(b), ybar_b=None if yb is None else dev(yb),
                         abar=ab0, bbar=bb0, ys_a=ysa, ys_b=ysb, accumulate=True, work=work)
        torch.cuda.synchronize()
        assert A.adpar_workspace_status(work) == A.OK
        assert rel_l2(ab0.cpu().numpy(), rab) < 1e-12, (nbytes, rel_l2(ab0.cpu().numpy(), rab))
        assert rel_l2(ysa.cpu().numpy(), rya) < 1e-12
        if op == "linrec":
            assert rel_l2(bb0.cpu().numpy(), rbb) < 1e-12
            assert rel_l2(ysb.cpu().numpy(), ryb) < 1e-12


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("op", ["min", "max"])
@pytest.mark.parametrize("pattern", ["increasing", "decreasing", "sawtooth", "tile_edges", "plateaus"])
def test_minmax_scan_record_patterns(A, oracle, op, dt, pattern):
    """Record structure of the min/max rule: the adjoint is nonzero only at
    records (strictly beyond everything before; ties stay with the earlier
    element) and element 0.  Every element a record, none after the first,
    records in some tiles only, records on tile boundaries and long ties;
    the nonzero pattern is compared exactly."""
    n = 5 * 8192 + 77
    g = synth.rng(17)
    i = np.arange(n, dtype=np.float64)
    if pattern == "increasing":
        a = i
    elif pattern == "decreasing":
        a = -i
    elif pattern == "sawtooth":
        a = (i % 3000) + np.floor(i / 20000) * 4000  # a new high every 20000 elements
    elif pattern == "tile_edges":
        a = np.full(n, -1e6)
        for t, e in enumerate(range(0, n, 4096)):
            a[e] = t  # a record on every 4096-element boundary
    else:
        a = np.floor(i / 5000)  # plateaus: only each plateau's first element is a record
    if op == "min":
        a = -a
    a = a.astype(dt)
    y = g.standard_normal(n).astype(dt)
    ys = torch.empty(n, dtype=torch.float32 if dt == np.float32 else torch.float64, device="cuda")
    ab, _, work = A.adpar_vjp_scan(op, dev(a), dev(y), ys_a=ys)
    torch.cuda.synchronize()
    assert A.adpar_workspace_status(work) == A.OK
    ref, _, rys, _ = oracle.scan_vjp(op, a, y)
    got = ab.cpu().numpy()
    np.testing.assert_array_equal(got != 0, ref != 0)
    assert rel_l2(got, ref) < tol(dt, n)
    np.testing.assert_array_equal(ys.cpu().numpy(), rys.astype(dt))


def test_scan_zero_length_and_errors(A):
    e = torch.empty(0, device="cuda")
    ab, _, _ = A.adpar_vjp_scan("add", e, e)
    assert ab.numel() == 0
    x = torch.zeros(9, device="cuda")
    with pytest.raises(A.AdparError):
        A.adpar_vjp_scan("add", x[1:], x[1:])  # 4-byte offset: not 16-byte aligned


@pytest.mark.slow
@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_linrec_full_size(A, oracle, dt):
    """n = 2^26 pairs (the benchmark size), full comparison with the oracle."""
    n = 1 << 26
    a, b, ya, yb = synth.linrec(n, dt, seed=synth.SEED_BASE + 1)
    ab, bb, work = A.adpar_vjp_scan("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb))
    assert A.adpar_workspace_status(work) == A.OK
    rab, rbb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb)
    assert rel_l2(ab.cpu().numpy(), rab) < tol(dt, n)
    assert rel_l2(bb.cpu().numpy(), rbb) < tol(dt, n)


@pytest.mark.slow
@pytest.mark.parametrize("op", ["add", "max"])
def test_add_max_scan_full_size(A, oracle, op):
    """n = 2^28 FP32 (the benchmark size): full comparison with the oracle."""
    n = 1 << 28
    x = synth.normal(n, np.float32, seed=synth.SEED_BASE + 1)
    y = synth.normal(n, np.float32, seed=synth.SEED_BASE + 11)
    ab, _, work = A.adpar_vjp_scan(op, dev(x), dev(y))
    assert A.adpar_workspace_status(work) == A.OK
    got = ab.cpu().numpy()
    del ab
    ref, _, _, _ = oracle.scan_vjp(op, x, y)
    assert rel_l2(got, ref) < 1e-3
    if op == "max":
        np.testing.assert_array_equal(np.flatnonzero(got), np.flatnonzero(ref))


# tiles of 128 runs: 2048 FP64 / 4096 FP32 elements
RUN_SIZES = {np.float64: [1, 15, 16, 17, 2047, 2048, 2049, 3 * 2048 + 5, 100001, (1 << 20) + 3],
             np.float32: [1, 31, 32, 33, 4095, 4096, 4097, 3 * 4096 + 5, 100001, (1 << 20) + 3]}


@pytest.mark.parametrize("dt,n", [(dt, n) for dt in (np.float64, np.float32) for n in RUN_SIZES[dt]])
@pytest.mark.parametrize("accumulate", [False, True])
def test_linrec_runs_path(A, oracle, dt, n, accumulate):
    """The linear recurrence with the full workspace runs on per-thread runs
    of one 128-byte row (16 FP64 / 32 FP32 elements) and tiles of 128 runs
    (whole tiles through TMA, the last one element by element): ragged sizes
    around run and tile edges, overwrite and accumulation, against the
    oracle."""
    f64 = dt == np.float64
    a, b, ya, yb = synth.linrec(n, dt, seed=n + 21)
    base = synth.normal(n, dt, seed=22) if accumulate else np.zeros(n, dt)
    base_b = base[::-1].copy()
    rab, rbb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb, abar=base, bbar=base_b)
    ab0, bb0 = dev(base), dev(base_b)
    work = A.workspace(A.adpar_workspace_size(A.RULE_SCAN, A.OP_LINREC, A.F64 if f64 else A.F32, n))
    A.adpar_vjp_scan("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb), abar=ab0, bbar=bb0,
                     accumulate=accumulate, work=work)
    assert A.adpar_workspace_status(work) == A.OK
    tol = 1e-12 if f64 else 1e-4
    assert rel_l2(ab0.cpu().numpy(), rab) < tol
    assert rel_l2(bb0.cpu().numpy(), rbb) < tol


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("n", [1, 3, 4, 5, 8191, 8192, 8193, 16383, 16384, 16385, 3 * 16384 + 7, 1000003,
                               1000 * 16384 + 5])
@pytest.mark.parametrize("accumulate", [False, True])
def test_add_scan_runs_path(A, oracle, dt, n, accumulate):
    """The + scan VJP without the recomputed ys runs on 128-byte rows in
    tiles of 512 rows (16384 FP32 / 8192 FP64 elements) moved by TMA through
    a ring of tiles per block, with the carries formed from the tile sums of
    lower tickets (the last tile element by element): sizes around row and
    tile edges, a size with several tiles per block (the ring wraps),
    overwrite and accumulation, against the oracle."""
    y = synth.normal(n, dt, seed=n + 31)
    base = synth.normal(n, dt, seed=32) if accumulate else np.zeros(n, dt)
    ref, _, _, _ = oracle.scan_vjp("add", np.zeros(n), y, abar=base)
    ab0 = dev(base)
    work = A.workspace(A.adpar_workspace_size(A.RULE_SCAN, A.OP_ADD, A.F64 if dt == np.float64 else A.F32, n))
    A.adpar_vjp_scan("add", None, dev(y), abar=ab0, accumulate=accumulate, work=work)
    assert A.adpar_workspace_status(work) == A.OK
    assert rel_l2(ab0.cpu().numpy(), ref) < tol(dt, n)


@pytest.mark.parametrize("path,dt,n", [("runs", np.float64, 2048 * 8193 + 5), ("runs", np.float32, 4096 * 4097 + 7),
                                       ("minimal", np.float32, 4096 * 4097 + 9)])
def test_tile_carry_segments(A, oracle, path, dt, n):
    """More than 4096 tiles: the tile carries are scanned in segments of 4096
    tiles (one block each) and the earlier segments' fold is applied after
    (two and three segments, ragged last tile), on the runs path and on the
    minimal-workspace path, against the oracle."""
    f64 = dt == np.float64
    a, b, ya, yb = synth.linrec(n, dt, seed=n % 1000 + 41)
    rab, rbb, _, _ = oracle.scan_vjp("linrec", a, ya, b, yb)
    flags = A.RULE_SCAN | (A.WS_MINIMAL if path == "minimal" else 0)
    work = A.workspace(A.adpar_workspace_size(flags, A.OP_LINREC, A.F64 if f64 else A.F32, n))
    ab, bb, _ = A.adpar_vjp_scan("linrec", dev(a), dev(ya), b=dev(b), ybar_b=dev(yb), work=work)
    assert A.adpar_workspace_status(work) == A.OK
    t = tol(dt, n)
    assert rel_l2(ab.cpu().numpy(), rab) < t
    assert rel_l2(bb.cpu().numpy(), rbb) < t
