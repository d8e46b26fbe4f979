"""numpy front end of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It loads ``liboracle.so`` (plain C,
see ``adpar_oracle.c``) and converts every input to FP64 / int64 first, so
FP32 inputs are compared against the exact FP64 gradient of the same
numbers.  Each function names the part of arXiv 2202.10297 it states.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

ADD, MUL, MIN, MAX, LINREC = 0, 1, 2, 3, 4
OPS = {"add": ADD, "mul": MUL, "min": MIN, "max": MAX, "linrec": LINREC, "matrec2": 5}
WIDE = {"linrec": 2, "matrec2": 6}  # element width of the wide-element scan
GATHER, SCALE, SQDIST_ROW = 0, 1, 2
GFUNS = {"gather": GATHER, "scale": SCALE, "sqdist_row": SQDIST_ROW}

_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I8 = C.POINTER(C.c_int8)


def lib():
    global _lib
    if _lib is None:
        # ADPAR_ORACLE_LIB lets the mutation tests load a deliberately broken
        # build of this same source from a temporary directory.
        path = os.environ.get("ADPAR_ORACLE_LIB") or _build.build_oracle()
        L = C.CDLL(path)
        i64, dbl = C.c_int64, C.c_double
        L.oracle_reduce_vjp.argtypes = [C.c_int, i64, _D, dbl, _D, _D, _I64]
        L.oracle_prod_reduce_vjp.argtypes = [i64, _D, dbl, _D, _D, _I8, _I64, _D]
        L.oracle_scan_vjp.argtypes = [C.c_int, i64, _D, _D, _D, _D, _D, _D, _D, _D]
        L.oracle_hist_vjp.argtypes = [C.c_int, i64, i64, _D, _I64, _D, _D, _D, _I64]
        L.oracle_hist_prod_vjp.argtypes = [i64, i64, _D, _I64, _D, _D, _D, _I8,
                                           _I64, _I64, _D, _D]
        L.oracle_scatter_vjp.argtypes = [i64, i64, _I64, _D, _D, _D, _D]
        L.oracle_map_acc_vjp.argtypes = [C.c_int, i64, i64, C.c_int, _D, _I64, _D,
                                         _D, _D, _D]
        L.oracle_kmeans.argtypes = [i64, C.c_int, C.c_int, _D, _D, dbl, _D, _I64,
                                    _D, _D]
        L.oracle_reduce_general_vjp.argtypes = [C.c_int, i64, _D, _D, dbl, dbl, _D, _D, _D]
        L.oracle_scan_jvp.argtypes = [C.c_int, i64, _D, _D, _D, _D, _D, _D, _D, _D]
        L.oracle_hist_general_vjp.argtypes = [C.c_int, i64, i64, _D, _D, _I64, _D, _D, _D, _D,
                                              _D, _D]
        L.oracle_scan_wide_vjp.argtypes = [C.c_int, i64, C.c_int, _D, _D, _D, _D]
        L.oracle_kmeans_hessdiag.argtypes = [i64, C.c_int, C.c_int, _D, _D, dbl, _D]
        L.oracle_reduce_jvp.argtypes = [C.c_int, i64, _D, _D, _D, _D]
        L.oracle_prod_reduce_jvp.argtypes = [i64, _D, _D, _D, _D, _I8]
        L.oracle_hist_jvp.argtypes = [C.c_int, i64, i64, _D, _D, _I64, _D, _D]
        L.oracle_hist_prod_jvp.argtypes = [i64, i64, _D, _D, _I64, _D, _D, _I8]
        L.oracle_scatter_jvp.argtypes = [i64, i64, _I64, _D, _D]
        L.oracle_map_acc_jvp.argtypes = [C.c_int, i64, i64, C.c_int, _D, _I64, _D, _D, _D, _D]
        L.oracle_kmeans_fwd_rev.argtypes = [i64, C.c_int, C.c_int, _D, _D, _D, dbl, _D, _D]
        for f in ("oracle_reduce_vjp", "oracle_prod_reduce_vjp", "oracle_scan_vjp",
                  "oracle_hist_vjp", "oracle_hist_prod_vjp", "oracle_scatter_vjp",
                  "oracle_map_acc_vjp", "oracle_kmeans", "oracle_reduce_general_vjp", "oracle_scan_jvp",
                  "oracle_hist_general_vjp", "oracle_scan_wide_vjp", "oracle_kmeans_hessdiag",
                  "oracle_reduce_jvp", "oracle_prod_reduce_jvp", "oracle_hist_jvp", "oracle_hist_prod_jvp",
                  "oracle_scatter_jvp", "oracle_map_acc_jvp", "oracle_kmeans_fwd_rev"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _f64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _i64(x):
    return np.ascontiguousarray(np.asarray(x, dtype=np.int64))


def _p(x, t=_D):
    return None if x is None else x.ctypes.data_as(t)


def _check(rc, name):
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (name, rc))


def reduce_vjp(op, a, ybar=1.0, abar=None):
    """Reduce with + / min / max (Sec. 5.1).  Returns (y, abar, argidx)."""
    a = _f64(a)
    n = a.size
    out = np.zeros(n) if abar is None else _f64(abar).copy()
    y = C.c_double(0.0)
    arg = C.c_int64(-1)
    _check(lib().oracle_reduce_vjp(OPS[op], n, _p(a), float(ybar), C.byref(y),
                                   _p(out), C.byref(arg)), "reduce_vjp")
    return y.value, out, arg.value


def scan_jvp(op, a, adot, b=None, bdot=None):
    """Forward mode of the inclusive scan (dual numbers).  Returns
    (ys_a, ys_b, ysdot_a, ysdot_b); the b parts only for linrec."""
    a = _f64(a)
    ad = _f64(adot)
    n = a.size
    w2 = op == "linrec"
    ya, yd = np.empty(n), np.empty(n)
    yb = ydb = None
    if w2:
        b, bd = _f64(b), _f64(bdot)
        yb, ydb = np.empty(n), np.empty(n)
    _check(lib().oracle_scan_jvp(OPS[op], n, _p(a), _p(b) if w2 else None, _p(ad), _p(bd) if w2 else None,
                                 _p(ya), _p(yb), _p(yd), _p(ydb)), "scan_jvp")
    return ya, yb, yd, ydb


def reduce_general_vjp(op, a, ybar, b=None, ybar_b=0.0, abar=None, bbar=None):
    """Reduce with any supported operator by the plain tape sweep (Sec. 5.1.1,
    general rule).  Returns (y tuple, abar, bbar); ``bbar`` only for linrec."""
    a = _f64(a)
    n = a.size
    w2 = op == "linrec"
    ab = np.zeros(n) if abar is None else _f64(abar).copy()
    bb = None
    if w2:
        b = _f64(b)
        bb = np.zeros(n) if bbar is None else _f64(bbar).copy()
    y = np.zeros(2)
    _check(lib().oracle_reduce_general_vjp(OPS[op], n, _p(a), _p(b) if w2 else None, float(ybar),
                                           float(ybar_b), _p(ab), _p(bb) if w2 else None, _p(y)),
           "reduce_general_vjp")
    return (tuple(y) if w2 else (y[0],)), ab, bb


def prod_reduce_vjp(a, ybar=1.0, abar=None):
    """Reduce with * (Sec. 5.1.1), extended exponent.

    Returns a dict: abar (FP64 values, accumulated onto ``abar``), log
    (ln|contribution|), sign, nzero, first_zero, lognz, signnz, y.
    """
    a = _f64(a)
    n = a.size
    val = np.zeros(n) if abar is None else _f64(abar).copy()
    lg = np.empty(n)
    sg = np.empty(n, dtype=np.int8)
    auxi = np.zeros(2, dtype=np.int64)
    auxd = np.zeros(3)
    _check(lib().oracle_prod_reduce_vjp(n, _p(a), float(ybar), _p(val), _p(lg),
                                        _p(sg, _I8), _p(auxi, _I64), _p(auxd)),
           "prod_reduce_vjp")
    return dict(abar=val, log=lg, sign=sg, nzero=int(auxi[0]),
                first_zero=int(auxi[1]), lognz=float(auxd[0]),
                signnz=int(auxd[1]), y=float(auxd[2]))


def scan_vjp(op, a, ybar, b=None, ybbar=None, abar=None, bbar=None):
    """Inclusive scan (Sec. 5.2).  Returns (abar, bbar, ys_a, ys_b).

    For ``linrec`` the element is the pair (a, b); otherwise b is unused.
    """
    a = _f64(a)
    yb = _f64(ybar)
    n = a.size
    w2 = op == "linrec"
    ab = np.zeros(n) if abar is None else _f64(abar).copy()
    ys0 = np.empty(n)
    if w2:
        b = _f64(b)
        ybb = _f64(ybbar)
        bb = np.zeros(n) if bbar is None else _f64(bbar).copy()
        ys1 = np.empty(n)
    else:
        b = ybb = bb = ys1 = None
    _check(lib().oracle_scan_vjp(OPS[op], n, _p(a), _p(b), _p(yb), _p(ybb),
                                 _p(ab), _p(bb), _p(ys0), _p(ys1)), "scan_vjp")
    return ab, bb, ys0, ys1


def hist_vjp(op, vals, inds, m, hsbar, valsbar=None):
    """reduce_by_index with + / min / max (Sec. 5.1.2).

    Returns (valsbar, hs, argidx[m]).
    """
    v = _f64(vals)
    ix = _i64(inds)
    hb = _f64(hsbar)
    n = v.size
    vb = np.zeros(n) if valsbar is None else _f64(valsbar).copy()
    hs = np.empty(max(m, 1))
    arg = np.empty(max(m, 1), dtype=np.int64)
    _check(lib().oracle_hist_vjp(OPS[op], n, m, _p(v), _p(ix, _I64), _p(hb), _p(vb),
                                 _p(hs), _p(arg, _I64)), "hist_vjp")
    return vb, hs[:m], arg[:m]


def hist_prod_vjp(vals, inds, m, hsbar, valsbar=None):
    """reduce_by_index with * (Sec. 5.1.2 with the * rule of Sec. 5.1.1)."""
    v = _f64(vals)
    ix = _i64(inds)
    hb = _f64(hsbar)
    n = v.size
    vb = np.zeros(n) if valsbar is None else _f64(valsbar).copy()
    lg = np.empty(n)
    sg = np.empty(n, dtype=np.int8)
    nz = np.empty(max(m, 1), dtype=np.int64)
    fz = np.empty(max(m, 1), dtype=np.int64)
    lnz = np.empty(max(m, 1))
    snz = np.empty(max(m, 1))
    _check(lib().oracle_hist_prod_vjp(n, m, _p(v), _p(ix, _I64), _p(hb), _p(vb),
                                      _p(lg), _p(sg, _I8), _p(nz, _I64), _p(fz, _I64),
                                      _p(lnz), _p(snz)), "hist_prod_vjp")
    return dict(valsbar=vb, log=lg, sign=sg, nzero=nz[:m], first_zero=fz[:m],
                lognz=lnz[:m], signnz=snz[:m].astype(np.int64))


def scan_wide_vjp(op, a, ybar, abar=None):
    """Scan over elements of d scalars (rows of [n, d]) with full d x d
    Jacobians (Sec. 5.2, generalised lin_o).  Returns (abar [n, d], ys [n, d])."""
    d = WIDE[op]
    a = _f64(a).reshape(-1, d)
    yb = _f64(ybar).reshape(-1, d)
    n = a.shape[0]
    ab = np.zeros((n, d)) if abar is None else _f64(abar).reshape(n, d).copy()
    ys = np.empty((n, d))
    _check(lib().oracle_scan_wide_vjp(OPS[op], n, d, _p(a), _p(yb), _p(ab), _p(ys)), "scan_wide_vjp")
    return ab, ys


def hist_general_vjp(op, vals, inds, m, hsbar, b=None, hsbar_b=None, valsbar=None, bbar=None):
    """reduce_by_index with any operator by the plain tape sweep (Sec. 5.1.2,
    general rule), bins combined in index order.  Returns
    (valsbar, bbar, hs_a, hs_b); the b parts only for linrec."""
    v = _f64(vals)
    ix = _i64(inds)
    n = v.size
    w2 = op == "linrec"
    hb = _f64(hsbar)
    vb = np.zeros(n) if valsbar is None else _f64(valsbar).copy()
    hs_a = np.empty(max(m, 1))
    bv = hbb = bb = hs_b = None
    if w2:
        bv, hbb = _f64(b), _f64(hsbar_b)
        bb = np.zeros(n) if bbar is None else _f64(bbar).copy()
        hs_b = np.empty(max(m, 1))
    _check(lib().oracle_hist_general_vjp(OPS[op], n, m, _p(v), _p(bv), _p(ix, _I64), _p(hb), _p(hbb),
                                         _p(vb), _p(bb), _p(hs_a), _p(hs_b)), "hist_general_vjp")
    return vb, bb, hs_a[:m], (hs_b[:m] if w2 else None)


def scatter_vjp(n, is_, ysbar, vsbar=None, ys=None, xs_saved=None):
    """Scatter (Sec. 5.3).  Returns (xsbar, vsbar, ys_restored)."""
    ix = _i64(is_)
    m = ix.size
    yb = _f64(ysbar).copy()
    vb = np.zeros(m) if vsbar is None else _f64(vsbar).copy()
    yr = None if ys is None else _f64(ys).copy()
    xs = None if xs_saved is None else _f64(xs_saved)
    _check(lib().oracle_scatter_vjp(n, m, _p(ix, _I64), _p(yb), _p(vb), _p(yr),
                                    _p(xs)), "scatter_vjp")
    return yb, vb, yr


def map_acc_vjp(g, as_, is_, xsbar, ws=None, width=1, asbar=None, wsbar=None):
    """map with a free array turned into an accumulator (Sec. 5.4).

    Returns (asbar, wsbar).
    """
    a = _f64(as_)
    ix = _i64(is_)
    xb = _f64(xsbar)
    nj = ix.size
    na = a.size // width
    w = None if ws is None else _f64(ws)
    ab = np.zeros(a.size) if asbar is None else _f64(asbar).copy()
    wb = None
    if w is not None:
        wb = np.zeros(w.size) if wsbar is None else _f64(wsbar).copy()
    _check(lib().oracle_map_acc_vjp(GFUNS[g], nj, na, width, _p(a), _p(ix, _I64),
                                    _p(w), _p(xb), _p(ab), _p(wb)), "map_acc_vjp")
    return ab, wb


def kmeans_hessdiag(X, Cm, ybar=1.0):
    """Hessian diagonal of the k-means cost in C with the argmins held fixed
    (Sec. 7.4): 2 ybar times each centroid's count, [k, d]."""
    X = _f64(X)
    Cm = _f64(Cm)
    N, d = X.shape
    k = Cm.shape[0]
    H = np.empty((k, d))
    _check(lib().oracle_kmeans_hessdiag(N, d, k, _p(X), _p(Cm), float(ybar), _p(H)), "kmeans_hessdiag")
    return H


def kmeans(X, Cm, ybar=1.0):
    """k-means cost with squared distances and its gradient in C (Sec. 7.4).

    Returns (loss, argmin[N], mind[N], Cbar[k, d]).
    """
    X = _f64(X)
    Cm = _f64(Cm)
    N, d = X.shape
    k = Cm.shape[0]
    loss = C.c_double(0.0)
    arg = np.empty(N, dtype=np.int64)
    mind = np.empty(N)
    cb = np.zeros((k, d))
    _check(lib().oracle_kmeans(N, d, k, _p(X), _p(Cm), float(ybar), C.byref(loss),
                               _p(arg, _I64), _p(mind), _p(cb)), "kmeans")
    return loss.value, arg, mind, cb


# ------------------------------------------------------------ forward mode
def reduce_jvp(op, a, adot):
    """Forward mode of reduce with +, min, max (Sec. 3 dual numbers over the
    loop of Sec. 5.1).  Returns (y, ydot)."""
    a, ad = _f64(a), _f64(adot)
    y, yd = np.zeros(1), np.zeros(1)
    _check(lib().oracle_reduce_jvp(OPS[op], a.size, _p(a), _p(ad), _p(y), _p(yd)), "reduce_jvp")
    return float(y[0]), float(yd[0])


def prod_reduce_jvp(a, adot):
    """Forward mode of reduce with * (extended exponent).  Returns a dict:
    ydot (FP64 value), log (ln|ydot|), sign."""
    a, ad = _f64(a), _f64(adot)
    v, lg = np.zeros(1), np.zeros(1)
    sg = np.zeros(1, dtype=np.int8)
    _check(lib().oracle_prod_reduce_jvp(a.size, _p(a), _p(ad), _p(v), _p(lg), _p(sg, _I8)), "prod_reduce_jvp")
    return dict(ydot=float(v[0]), log=float(lg[0]), sign=int(sg[0]))


def hist_jvp(op, vals, vdot, inds, m):
    """Forward mode of reduce_by_index with +, min, max (Sec. 5.1.2's loop on
    dual numbers).  Returns (hs, hsdot), each [m]."""
    v, vd, ix = _f64(vals), _f64(vdot), _i64(inds)
    hs, hd = np.zeros(m), np.zeros(m)
    _check(lib().oracle_hist_jvp(OPS[op], v.size, m, _p(v), _p(vd), _p(ix, _I64), _p(hs), _p(hd)), "hist_jvp")
    return hs, hd


def hist_prod_jvp(vals, vdot, inds, m):
    """Forward mode of reduce_by_index with * (extended exponent).  Returns a
    dict of [m] arrays: hsdot (FP64 values), log, sign."""
    v, vd, ix = _f64(vals), _f64(vdot), _i64(inds)
    val, lg = np.zeros(m), np.zeros(m)
    sg = np.zeros(m, dtype=np.int8)
    _check(lib().oracle_hist_prod_jvp(v.size, m, _p(v), _p(vd), _p(ix, _I64), _p(val), _p(lg), _p(sg, _I8)),
           "hist_prod_jvp")
    return dict(hsdot=val, log=lg, sign=sg)


def scatter_jvp(n, is_, vsdot, xsdot):
    """Forward mode of scatter (Sec. 5.3): ysdot = xsdot with ysdot[is_j] = vsdot_j."""
    ix, vd = _i64(is_), _f64(vsdot)
    out = _f64(xsdot).copy()
    assert out.size == n
    _check(lib().oracle_scatter_jvp(n, ix.size, _p(ix, _I64), _p(vd), _p(out)), "scatter_jvp")
    return out


def map_acc_jvp(g, as_, is_, asdot, ws=None, wsdot=None, width=1):
    """Forward mode of map with a free array (Sec. 5.4).  Returns xsdot [nj]."""
    a, ix, ad = _f64(as_), _i64(is_), _f64(asdot)
    w = None if ws is None else _f64(ws)
    wd = None if wsdot is None else _f64(wsdot)
    na = a.size // width
    out = np.zeros(ix.size)
    _check(lib().oracle_map_acc_jvp(GFUNS[g], ix.size, na, width, _p(a), _p(ix, _I64), _p(w), _p(ad), _p(wd),
                                    _p(out)), "map_acc_jvp")
    return out


def kmeans_fwd_rev(X, Cm, Cdot, ybar=1.0):
    """Forward over reverse for the k-means cost (Sec. 7.4): the tangent, along
    Cdot, of the loss and of its gradient in C.  Returns (ydot, Cbardot [k, d])."""
    X, Cm, Cd = _f64(X), _f64(Cm), _f64(Cdot)
    N, d = X.shape
    k = Cm.shape[0]
    yd = np.zeros(1)
    out = np.zeros((k, d))
    _check(lib().oracle_kmeans_fwd_rev(N, d, k, _p(X), _p(Cm), _p(Cd), float(ybar), _p(yd), _p(out)),
           "kmeans_fwd_rev")
    return float(yd[0]), out
