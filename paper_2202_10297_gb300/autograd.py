"""torch.autograd.Function wrappers of the adpar rules.

Every forward runs the primal operator in the library's kernels and saves
only its INPUTS; every backward re-executes the primal inside the VJP
kernels (the redundant-execution policy of Sec. 4: no tape, no stored
intermediate) and returns the adjoints the paper's rule gives.

    scan(op, a, b=None)           inclusive scan; LINREC returns (A, B); reverse
                                  and forward mode (torch.autograd.forward_ad)
    reduce(op, a)                 0-dim result; reverse and forward mode
    reduce_by_index(op, vals, inds, m, b=None)
                                  LINREC (b given) by the general rule; the
                                  special rules also in forward mode
    scan_wide(op, a)              scan over [n, d] elements ("linrec", "matrec2")
    scatter(xs, is_, vs)          out of place: xs is not modified; both modes
    map_acc(g, as_, is_, ws=None, width=1)   both modes
    kmeans_loss(X, C)             gradient with respect to C only; forward
                                  mode in C
    kmeans_hvp(X, C, Cdot)        forward over reverse: Hessian-vector product
"""
import torch

from . import adpar as A


def _c(t):
    return None if t is None else t.contiguous()


class _Scan(torch.autograd.Function):
    @staticmethod
    def forward(ctx, op, a, b):
        ya, yb, _ = A.adpar_scan(op, a, b=b)
        ctx.op = op
        ctx.save_for_backward(a, b)
        ctx.save_for_forward(a, b)
        return (ya, yb) if op == "linrec" else ya

    @staticmethod
    def jvp(ctx, _, ta, tb):
        # forward mode: the dual-number scan (adpar_jvp_scan)
        a, b = ctx.saved_tensors
        ta = torch.zeros_like(a) if ta is None else ta.contiguous()
        if ctx.op == "linrec":
            tb = torch.zeros_like(a) if tb is None else tb.contiguous()
            yd_a, yd_b, _, _ = A.adpar_jvp_scan("linrec", a, ta, b=b, bdot=tb)
            return yd_a, yd_b
        yd_a, _, _, _ = A.adpar_jvp_scan(ctx.op, a, ta)
        return yd_a

    @staticmethod
    def backward(ctx, ga, gb=None):
        a, b = ctx.saved_tensors
        if ctx.op == "linrec":
            ga = torch.zeros_like(a) if ga is None else ga
            gb = torch.zeros_like(a) if gb is None else gb
            abar, bbar, _ = A.adpar_vjp_scan("linrec", a, _c(ga), b=b, ybar_b=_c(gb))
            return None, abar, bbar
        abar, _, _ = A.adpar_vjp_scan(ctx.op, a, _c(ga))
        return None, abar, None


def scan(op, a, b=None):
    """Inclusive scan with op in {add, mul, min, max, linrec} (Sec. 5.2)."""
    return _Scan.apply(op, _c(a), _c(b))


class _Reduce(torch.autograd.Function):
    @staticmethod
    def forward(ctx, op, a):
        y, _ = A.adpar_reduce(op, a)
        ctx.op = op
        ctx.save_for_backward(a)
        ctx.save_for_forward(a)
        return y.reshape(())

    @staticmethod
    def jvp(ctx, _, ta):
        # forward mode: the dual-number reduce (adpar_jvp_reduce)
        (a,) = ctx.saved_tensors
        ta = torch.zeros_like(a) if ta is None else ta.contiguous()
        return A.adpar_jvp_reduce(ctx.op, a, ta)["ydot"].reshape(())

    @staticmethod
    def backward(ctx, g):
        (a,) = ctx.saved_tensors
        out = A.adpar_vjp_reduce(ctx.op, a, g.reshape(1))
        return None, out["abar"]


def reduce(op, a):
    """reduce with op in {add, mul, min, max} (Sec. 5.1)."""
    return _Reduce.apply(op, _c(a))


class _Hist(torch.autograd.Function):
    @staticmethod
    def forward(ctx, op, vals, inds, m):
        hs, _ = A.adpar_hist(op, vals, inds, m)
        ctx.op, ctx.m = op, m
        ctx.save_for_backward(vals, inds)
        ctx.save_for_forward(vals, inds)
        return hs

    @staticmethod
    def jvp(ctx, _, tv, _ti, _tm):
        vals, inds = ctx.saved_tensors
        tv = torch.zeros_like(vals) if tv is None else tv.contiguous()
        return A.adpar_jvp_hist(ctx.op, vals, tv, inds, ctx.m)["hsdot"]

    @staticmethod
    def backward(ctx, g):
        vals, inds = ctx.saved_tensors
        out = A.adpar_vjp_hist(ctx.op, inds, ctx.m, _c(g), vals=vals)
        return None, out["valsbar"], None, None


class _HistGeneral(torch.autograd.Function):
    """reduce_by_index by the general rule (radix sort by bin, segmented
    scans); its forward is the same call with a zero cotangent, which
    recomputes the bins."""

    @staticmethod
    def forward(ctx, op, a, b, inds, m):
        z = torch.zeros(m, dtype=a.dtype, device=a.device)
        _, _, hs_a, hs_b = A.adpar_vjp_hist_general(op, a, inds, m, z, b=b, hsbar_b=z, want_hs=True)
        ctx.op, ctx.m = op, m
        ctx.save_for_backward(a, b, inds)
        return hs_a, hs_b

    @staticmethod
    def backward(ctx, ga, gb):
        a, b, inds = ctx.saved_tensors
        ga = torch.zeros(ctx.m, dtype=a.dtype, device=a.device) if ga is None else ga.contiguous()
        gb = torch.zeros(ctx.m, dtype=a.dtype, device=a.device) if gb is None else gb.contiguous()
        ab, bb, _, _ = A.adpar_vjp_hist_general(ctx.op, a, inds, ctx.m, ga, b=b, hsbar_b=gb)
        return None, ab, bb, None, None


def reduce_by_index(op, vals, inds, m, b=None):
    """reduce_by_index (Sec. 5.1.2): op in {add, mul, min, max} by the special
    rules; "linrec" (b given) by the general rule, returning the bins (A, B)."""
    if op == "linrec":
        return _HistGeneral.apply(op, _c(vals), _c(b), _c(inds), int(m))
    return _Hist.apply(op, _c(vals), _c(inds), int(m))


class _ScanWide(torch.autograd.Function):
    """Scan over [n, d] elements (the d x d lin_o rule); the forward is the
    same call with a zero cotangent, which recomputes the scan."""

    @staticmethod
    def forward(ctx, op, a):
        _, ys = A.adpar_vjp_scan_wide(op, a, torch.zeros_like(a), want_ys=True)
        ctx.op = op
        ctx.save_for_backward(a)
        return ys

    @staticmethod
    def backward(ctx, g):
        (a,) = ctx.saved_tensors
        ab, _ = A.adpar_vjp_scan_wide(ctx.op, a, g.contiguous())
        return None, ab


def scan_wide(op, a):
    """Inclusive scan over the rows of a [n, d] array: "linrec" (d = 2) or
    "matrec2" (d = 6, the 2x2 matrix linear recurrence)."""
    return _ScanWide.apply(op, _c(a))


class _Scatter(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xs, is_, vs):
        ys = xs.clone()  # the functional form consumes a copy of xs
        A.adpar_scatter(is_, vs, ys)
        ctx.save_for_backward(is_)
        ctx.save_for_forward(is_)
        ctx.shapes = (xs, vs)
        return ys

    @staticmethod
    def jvp(ctx, txs, _ti, tvs):
        (is_,) = ctx.saved_tensors
        xs, vs = ctx.shapes
        ysdot = torch.zeros_like(xs) if txs is None else txs.clone().contiguous()
        tvs = torch.zeros_like(vs) if tvs is None else tvs.contiguous()
        return A.adpar_jvp_scatter(is_, tvs, ysdot)

    @staticmethod
    def backward(ctx, g):
        (is_,) = ctx.saved_tensors
        xsbar = g.clone()  # becomes xs_bar in place
        xsbar, vsbar = A.adpar_vjp_scatter(is_, xsbar)
        return xsbar, None, vsbar


def scatter(xs, is_, vs):
    """ys = scatter xs is vs with duplicate-free is (Sec. 5.3)."""
    return _Scatter.apply(_c(xs), _c(is_), _c(vs))


class _MapAcc(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, as_, is_, ws, width):
        xs = A.adpar_map_acc(g, as_, is_, ws=ws, width=width)
        ctx.g, ctx.width = g, width
        ctx.save_for_backward(as_, is_, ws)
        ctx.save_for_forward(as_, is_, ws)
        return xs

    @staticmethod
    def jvp(ctx, _g, tas, _ti, tws, _w):
        as_, is_, ws = ctx.saved_tensors
        tas = torch.zeros_like(as_) if tas is None else tas.contiguous()
        tws = None if (tws is None or ws is None) else tws.contiguous()
        return A.adpar_jvp_map_acc(ctx.g, as_, is_, tas, ws=ws, wsdot=tws, width=ctx.width)

    @staticmethod
    def backward(ctx, gx):
        as_, is_, ws = ctx.saved_tensors
        asbar, wsbar = A.adpar_vjp_map_acc(ctx.g, as_, is_, _c(gx), ws=ws, width=ctx.width,
                                           want_wsbar=ws is not None)
        return None, asbar, None, wsbar, None


def map_acc(g, as_, is_, ws=None, width=1):
    """xs[j] = g(as[is_j], ws_j) with g in {gather, scale, sqdist_row} (Sec. 5.4)."""
    return _MapAcc.apply(g, _c(as_), _c(is_), _c(ws), int(width))


class _KMeans(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, C):
        out = A.adpar_kmeans_vjp(X, C, want_grad=False)
        ctx.save_for_backward(X, C)
        ctx.save_for_forward(X, C)
        return out["loss"].reshape(())

    @staticmethod
    def jvp(ctx, tX, tC):
        X, C = ctx.saved_tensors
        if tX is not None and bool((tX != 0).any()):
            raise NotImplementedError("kmeans_loss differentiates with respect to the centroids only")
        tC = torch.zeros_like(C) if tC is None else tC.contiguous()
        ydot, _ = A.adpar_kmeans_fwd_rev(X, C, tC)
        return ydot.reshape(())

    @staticmethod
    def backward(ctx, g):
        X, C = ctx.saved_tensors
        if ctx.needs_input_grad[0]:
            raise NotImplementedError("kmeans_loss differentiates with respect to the centroids only")
        out = A.adpar_kmeans_vjp(X, C, ybar=g.reshape(1).to(torch.float32))
        return None, out["Cbar"]


def kmeans_loss(X, C):
    """sum_i min_k ||x_i - c_k||^2 (Sec. 7.4, squared distances); gradient in
    C; forward mode in C as well."""
    return _KMeans.apply(_c(X), _c(C))


def kmeans_hvp(X, C, Cdot, ybar=1.0):
    """Hessian-vector product of the k-means cost in C by forward mode over
    the VJP (Sec. 7.4): the tangent of the gradient along Cdot."""
    return A.adpar_kmeans_fwd_rev(_c(X), _c(C), _c(Cdot), ybar=ybar)[1]
