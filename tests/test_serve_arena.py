"""Host logic of the serving loop, without a GPU: the arena allocator that
admission draws on, the request layouts it sizes blocks from, and the
per-request index maps of scatter requests."""
import numpy as np
import pytest


def test_arena_first_fit_merge_and_failure():
    from paper_2202_10297_gb300.serve import Arena
    ar = Arena(10 * 256)
    a = ar.alloc(300)          # 2 blocks of 256
    b = ar.alloc(256)
    c = ar.alloc(1000)         # 4 blocks
    assert (a, b, c) == (0, 512, 768)
    assert ar.used == 7 * 256 and ar.peak == 7 * 256
    assert ar.alloc(4 * 256) is None          # 3 blocks left: real allocation failure
    ar.release(b, 256)
    d = ar.alloc(200)
    assert d == 512                            # first fit reuses the hole
    ar.release(a, 300)
    ar.release(d, 200)
    assert ar.largest_free() == 3 * 256        # 0..768 merged
    ar.release(c, 1000)
    assert ar.used == 0 and ar.largest_free() == ar.size and len(ar.starts) == 1
    assert ar.peak == 7 * 256


def test_arena_fragmentation_refuses_what_total_free_would_hold():
    from paper_2202_10297_gb300.serve import Arena
    ar = Arena(8 * 256)
    offs = [ar.alloc(256) for _ in range(8)]
    for o in offs[::2]:
        ar.release(o, 256)
    assert ar.free_bytes() == 4 * 256 and ar.largest_free() == 256
    assert ar.alloc(2 * 256) is None
    with pytest.raises(ValueError):
        ar.release(offs[0], 256)               # already free


def test_arena_random_sequence_against_byte_map():
    from paper_2202_10297_gb300.serve import Arena, ALIGN
    g = np.random.default_rng(0)
    size = 1 << 16
    ar = Arena(size)
    owner = np.zeros(size, dtype=np.int64)     # 0 = free
    live = {}
    for step in range(4000):
        if live and (g.random() < 0.45 or len(live) > 40):
            k = list(live)[int(g.integers(0, len(live)))]
            off, nb = live.pop(k)
            ar.release(off, nb)
            owner[off:off + -(-nb // ALIGN) * ALIGN] = 0
        else:
            nb = int(g.integers(1, 6000))
            off = ar.alloc(nb)
            need = -(-nb // ALIGN) * ALIGN
            if off is None:
                # no run of free bytes as long as the request at any aligned start
                free = owner == 0
                runs = [free[s:s + need].all() for s in range(0, size - need + 1, ALIGN)]
                assert not any(runs)
                continue
            assert off % ALIGN == 0 and off + need <= size
            assert (owner[off:off + need] == 0).all()
            owner[off:off + need] = step + 1
            live[step] = (off, nb)
        assert ar.used == int((owner != 0).sum())
    for off, nb in live.values():
        ar.release(off, nb)
    assert ar.used == 0 and ar.largest_free() == ar.size


def test_request_layouts_and_scatter_maps():
    from paper_2202_10297_gb300 import serve
    reqs = serve.make_requests(200, rate=1000.0, lo=8, hi=14, seed=11)
    assert all(a.arrival <= b.arrival for a, b in zip(reqs, reqs[1:]))
    assert {r.dtype for r in reqs} == set(serve.DTYPES) and {r.op for r in reqs} == set(serve.OPS)
    for r in reqs:
        assert r.off % 4 == 0
        arrays, ws = r.layout()
        esz = 8 if r.dtype == "f64" else 4
        out_elems = sum(k for name, k, _ in arrays if name != "is")
        assert r.bytes() >= out_elems * esz + ws
        if r.op == "scatter":
            is_ = serve.scatter_indices(r.n, r.n // 4, r.sc_s, r.sc_o)
            assert is_.min() >= 0 and is_.max() < r.n
            assert np.unique(is_).size == is_.size
    again = serve.make_requests(200, rate=1000.0, lo=8, hi=14, seed=11)
    assert [(r.op, r.dtype, r.n, r.off) for r in reqs] == [(r.op, r.dtype, r.n, r.off) for r in again]
