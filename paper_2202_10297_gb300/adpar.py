"""Python binding of the libadpar C ABI (argument marshalling only).

Each ``adpar_*`` function here has the name of the C entry point it calls
(declared in include/adpar.h).  It takes torch CUDA tensors, checks dtypes
and shapes, passes raw device pointers, the current CUDA stream and a
workspace to the library, and raises :class:`AdparError` on a non-zero
status.  PyTorch only provides device memory and streams; every step of
every rule runs in the library's kernels.  There is no CPU fallback: if
libadpar.so is missing, loading fails loudly.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libadpar.so")

F32, F64 = 0, 1
I32, I64 = 0, 1
OP_ADD, OP_MUL, OP_MIN, OP_MAX, OP_LINREC, OP_MATREC2 = 0, 1, 2, 3, 4, 5
OPS = {"add": OP_ADD, "mul": OP_MUL, "min": OP_MIN, "max": OP_MAX, "linrec": OP_LINREC, "matrec2": OP_MATREC2}
WIDE = {OP_LINREC: 2, OP_MATREC2: 6}  # element width D of adpar_vjp_scan_wide
G_GATHER, G_SCALE, G_SQDIST_ROW = 0, 1, 2
GFUNS = {"gather": G_GATHER, "scale": G_SCALE, "sqdist_row": G_SQDIST_ROW}
RULE_REDUCE, RULE_SCAN, RULE_HIST, RULE_SCATTER, RULE_MAP_ACC, RULE_KMEANS, RULE_REDUCE_GENERAL, RULE_SCAN_VEC, \
    RULE_HIST_GENERAL, RULE_SCAN_WIDE, RULE_JVP_REDUCE, RULE_JVP_HIST, RULE_KMEANS_FWD_REV = range(13)
WS_MINIMAL = 0x100  # or'ed into a rule: the smallest accepted workspace
ACCUMULATE, PROD_LOGDOMAIN, SCATTER_RESTORE, FULL_LIN_O = 0x1, 0x4, 0x8, 0x10
OK, ERR_INVALID, ERR_TIMEOUT, ERR_TOO_LARGE = 0, 1, 6, 7


class AdparError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__("%s: %s (status %d)" % (fn, status_string(status), status))


class OpDesc(C.Structure):
    _fields_ = [("op", C.c_int32), ("dtype", C.c_int32), ("width", C.c_int32)]


class ProdAux(C.Structure):
    _fields_ = [("nzero", C.c_int64), ("first_zero", C.c_int64), ("exp2", C.c_int64),
                ("mant", C.c_double), ("log_abs_nz", C.c_double), ("sign", C.c_int32),
                ("reserved", C.c_int32)]


PROD_AUX_BYTES = C.sizeof(ProdAux)


class JvpAux(C.Structure):
    _fields_ = [("log_abs", C.c_double), ("sign", C.c_int32), ("reserved", C.c_int32)]


JVP_AUX_BYTES = C.sizeof(JvpAux)
JVP_AUX_DTYPE = [("log_abs", "<f8"), ("sign", "<i4"), ("reserved", "<i4")]

_lib = None
_VP = C.c_void_p


def lib():
    """The loaded libadpar (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libadpar.so not found at %s: run paper_2202_10297_gb300.build.build() "
                               "(or __graft_entry__.build()) first" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        L.adpar_status_string.restype = C.c_char_p
        L.adpar_status_string.argtypes = [C.c_int]
        L.adpar_version.restype = C.c_char_p
        L.adpar_workspace_size.restype = C.c_size_t
        L.adpar_workspace_size.argtypes = [C.c_int, OpDesc, C.c_int64, C.c_int64]
        L.adpar_workspace_status.restype = C.c_int
        L.adpar_workspace_status.argtypes = [_VP, _VP, C.POINTER(C.c_int)]
        L.adpar_vjp_scan.restype = C.c_int
        L.adpar_vjp_scan.argtypes = [OpDesc, C.c_int64] + [_VP] * 8 + [C.c_uint32, _VP, C.c_size_t, _VP]
        L.adpar_vjp_scan_noalloc.restype = C.c_int
        L.adpar_vjp_scan_noalloc.argtypes = [OpDesc, C.c_int64] + [_VP] * 8 + [C.c_uint32, _VP]
        L.adpar_noalloc_scratch_bytes.restype = C.c_size_t
        L.adpar_noalloc_scratch_bytes.argtypes = []
        L.adpar_noalloc_status.restype = C.c_int
        L.adpar_noalloc_status.argtypes = [_VP, C.POINTER(C.c_int)]
        L.adpar_noalloc_selftest_timeout.restype = C.c_int
        L.adpar_noalloc_selftest_timeout.argtypes = [_VP]
        L.adpar_scan.restype = C.c_int
        L.adpar_scan.argtypes = [OpDesc, C.c_int64] + [_VP] * 4 + [_VP, C.c_size_t, _VP]
        L.adpar_vjp_scan_vec.restype = C.c_int
        L.adpar_vjp_scan_vec.argtypes = [OpDesc, C.c_int64, C.c_int64] + [_VP] * 6 + [C.c_uint32, _VP, C.c_size_t, _VP]
        L.adpar_jvp_scan.restype = C.c_int
        L.adpar_jvp_scan.argtypes = [OpDesc, C.c_int64] + [_VP] * 8 + [_VP, C.c_size_t, _VP]
        L.adpar_kmeans_hessdiag.restype = C.c_int
        L.adpar_kmeans_hessdiag.argtypes = [C.c_int, _VP, _VP, C.c_size_t, _VP, C.c_uint32, _VP]
        L.adpar_vjp_scan_wide.restype = C.c_int
        L.adpar_vjp_scan_wide.argtypes = [OpDesc, C.c_int64] + [_VP] * 4 + [C.c_uint32, _VP, C.c_size_t, _VP]
        L.adpar_vjp_hist_general.restype = C.c_int
        L.adpar_vjp_hist_general.argtypes = [OpDesc, C.c_int64, C.c_int64, _VP, _VP, _VP, C.c_int] + [_VP] * 6 + \
            [C.c_uint32, _VP, C.c_size_t, _VP]
        L.adpar_vjp_reduce_general.restype = C.c_int
        L.adpar_vjp_reduce_general.argtypes = [OpDesc, C.c_int64] + [_VP] * 8 + [C.c_uint32, _VP, C.c_size_t, _VP]
        _bind_optional(L)
        _lib = L
    return _lib


def _bind_optional(L):
    """Signatures of the entry points other than the scan."""
    sigs = {
        "adpar_vjp_reduce": [OpDesc, C.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.c_uint32, _VP,
                             C.c_size_t, _VP],
        "adpar_vjp_hist": [OpDesc, C.c_int64, C.c_int64, _VP, _VP, C.c_int, _VP, _VP, _VP, _VP, _VP,
                           _VP, C.c_uint32, _VP, C.c_size_t, _VP],
        "adpar_vjp_scatter": [C.c_int, C.c_int64, C.c_int64, _VP, C.c_int, _VP, _VP, _VP, _VP,
                              C.c_uint32, _VP],
        "adpar_vjp_map_acc": [C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int, _VP, _VP, C.c_int, _VP,
                              _VP, _VP, _VP, C.c_uint32, _VP, C.c_size_t, _VP],
        "adpar_kmeans_vjp": [C.c_int64, C.c_int, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP, C.c_uint32, _VP,
                             C.c_size_t, _VP],
        "adpar_reduce": [OpDesc, C.c_int64, _VP, _VP, _VP, _VP, _VP, C.c_size_t, _VP],
        "adpar_selftest_timeout": [_VP, C.c_size_t, _VP],
        "adpar_jvp_reduce": [OpDesc, C.c_int64, _VP, _VP, _VP, _VP, _VP, _VP, C.c_size_t, _VP],
        "adpar_jvp_hist": [OpDesc, C.c_int64, C.c_int64, _VP, _VP, _VP, C.c_int, _VP, _VP, _VP, _VP, C.c_size_t,
                           _VP],
        "adpar_jvp_scatter": [C.c_int, C.c_int64, C.c_int64, _VP, C.c_int, _VP, _VP, _VP],
        "adpar_jvp_map_acc": [C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int, _VP, _VP, C.c_int, _VP, _VP, _VP,
                              _VP, _VP],
        "adpar_kmeans_fwd_rev": [C.c_int64, C.c_int, C.c_int, _VP, _VP, _VP, _VP, _VP, _VP, C.c_uint32, _VP,
                                 C.c_size_t, _VP],
        "adpar_hist": [OpDesc, C.c_int64, C.c_int64, _VP, _VP, C.c_int, _VP, _VP, _VP, _VP, C.c_size_t, _VP],
        "adpar_scatter": [C.c_int, C.c_int64, C.c_int64, _VP, C.c_int, _VP, _VP, _VP, _VP],
        "adpar_map_acc": [C.c_int, C.c_int, C.c_int64, C.c_int64, C.c_int, _VP, _VP, C.c_int, _VP, _VP, _VP],
    }
    for name, argt in sigs.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = C.c_int
            f.argtypes = argt


def status_string(status):
    return lib().adpar_status_string(int(status)).decode()


def version():
    return lib().adpar_version().decode()


def _dtype_code(t):
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError("values must be float32 or float64, got %s" % t.dtype)


def _itype_code(t):
    if t.dtype == torch.int32:
        return I32
    if t.dtype == torch.int64:
        return I64
    raise TypeError("indices must be int32 or int64, got %s" % t.dtype)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


def _check(fn, status):
    if status != OK:
        raise AdparError(fn, status)


def adpar_workspace_size(rule, op, dtype, n, m=0, width=None):
    """Bytes of workspace a call needs (C: adpar_workspace_size)."""
    if width is None:
        width = 2 if op == OP_LINREC else 1
    sz = lib().adpar_workspace_size(rule, OpDesc(op, dtype, width), n, m)
    if sz == C.c_size_t(-1).value:
        raise ValueError("invalid workspace request")
    return sz


def workspace(nbytes, device=None):
    """A workspace buffer (256-byte aligned by the CUDA caching allocator)."""
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or "cuda")


def adpar_workspace_status(work, stream=None):
    """Device status word left in ``work`` by the last call (synchronises)."""
    st = C.c_int(0)
    _check("adpar_workspace_status",
           lib().adpar_workspace_status(_ptr(work), _stream(stream), C.byref(st)))
    return st.value


def adpar_vjp_scan(op, a, ybar_a, b=None, ybar_b=None, abar=None, bbar=None, ys_a=None, ys_b=None,
                   accumulate=False, work=None, stream=None):
    """VJP of an inclusive scan (C: adpar_vjp_scan).  Returns (abar, bbar, work).

    ``op`` is a name ("add", "mul", "min", "max", "linrec") or code.
    Missing outputs are allocated; ``ys_a``/``ys_b`` are filled when given.
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    ref = ybar_a
    n = ref.numel()
    dt = _dtype_code(ref)
    w = 2 if opc == OP_LINREC else 1
    if abar is None:
        abar = torch.empty_like(ref) if not accumulate else torch.zeros_like(ref)
    if w == 2 and bbar is None:
        bbar = torch.empty_like(ref) if not accumulate else torch.zeros_like(ref)
    # a given workspace is used if it has at least the minimal size (the
    # FP64 MUL/LINREC return sweep then re-forms the primal prefixes)
    if work is None or work.numel() < adpar_workspace_size(RULE_SCAN | WS_MINIMAL, opc, dt, n):
        work = workspace(adpar_workspace_size(RULE_SCAN, opc, dt, n), ref.device)
    for t in (a, b, ybar_b, abar, bbar, ys_a, ys_b):
        if t is not None and (t.dtype != ref.dtype or t.numel() != n):
            raise ValueError("all scan arrays must share dtype and length")
    st = lib().adpar_vjp_scan(OpDesc(opc, dt, w), n, _ptr(a), _ptr(b), _ptr(ybar_a), _ptr(ybar_b),
                              _ptr(abar), _ptr(bbar), _ptr(ys_a), _ptr(ys_b),
                              ACCUMULATE if accumulate else 0, _ptr(work), work.numel(),
                              _stream(stream))
    _check("adpar_vjp_scan", st)
    return abar, bbar, work


def adpar_vjp_reduce_general(op, a, ybar_a, b=None, ybar_b=None, abar=None, bbar=None, accumulate=False,
                             work=None, stream=None):
    """Reduce VJP by the general rule (C: adpar_vjp_reduce_general).

    ``ybar_a``/``ybar_b`` are scalars or one-element device tensors.
    Returns (abar, bbar, y) with y a device tensor of the operator's width.
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = a.numel()
    dt = _dtype_code(a)
    w = 2 if opc == OP_LINREC else 1

    def scalar(v):
        if isinstance(v, torch.Tensor):
            return v.to(device=a.device, dtype=a.dtype).reshape(1).contiguous()
        return torch.full((1,), float(v), dtype=a.dtype, device=a.device)
    ya = scalar(ybar_a)
    yb = scalar(ybar_b if ybar_b is not None else 0.0) if w == 2 else None
    if abar is None:
        abar = torch.zeros_like(a) if accumulate else torch.empty_like(a)
    if w == 2 and bbar is None:
        bbar = torch.zeros_like(a) if accumulate else torch.empty_like(a)
    for t in (b, abar, bbar):
        if t is not None and (t.dtype != a.dtype or t.numel() != n):
            raise ValueError("all reduce arrays must share dtype and length")
    y = torch.empty(2 if w == 2 else 1, dtype=a.dtype, device=a.device)
    need = adpar_workspace_size(RULE_REDUCE_GENERAL, opc, dt, n)
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    st = lib().adpar_vjp_reduce_general(OpDesc(opc, dt, w), n, _ptr(a), _ptr(b), _ptr(ya), _ptr(yb), _ptr(abar),
                                        _ptr(bbar), _ptr(y[0:1]), _ptr(y[1:2]) if w == 2 else None,
                                        ACCUMULATE if accumulate else 0, _ptr(work), work.numel(),
                                        _stream(stream))
    _check("adpar_vjp_reduce_general", st)
    return abar, bbar, y


def adpar_vjp_scan_wide(op, a, ybar, abar=None, want_ys=False, accumulate=False, full_lin_o=False, work=None,
                        stream=None):
    """VJP of a scan over [n, D] rows by the d x d lin_o (C: adpar_vjp_scan_wide).

    ``op`` is "linrec" (D = 2) or "matrec2" (D = 6); ``full_lin_o`` forces
    the full d x d lin_o where a blockwise one applies.  Returns (abar, ys),
    ys only with ``want_ys``.
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    D = WIDE[opc]
    if a.dim() != 2 or a.shape[1] != D or ybar.shape != a.shape:
        raise ValueError("a and ybar must be [n, %d]" % D)
    n = a.shape[0]
    dt = _dtype_code(a)
    if abar is None:
        abar = torch.zeros_like(a) if accumulate else torch.empty_like(a)
    ys = torch.empty_like(a) if want_ys else None
    need = adpar_workspace_size(RULE_SCAN_WIDE, opc, dt, n, 0, width=D)
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    flags = (ACCUMULATE if accumulate else 0) | (FULL_LIN_O if full_lin_o else 0)
    st = lib().adpar_vjp_scan_wide(OpDesc(opc, dt, D), n, _ptr(a), _ptr(ybar), _ptr(abar), _ptr(ys), flags,
                                   _ptr(work), work.numel(), _stream(stream))
    _check("adpar_vjp_scan_wide", st)
    return abar, ys


def adpar_vjp_hist_general(op, a, inds, m, hsbar_a, b=None, hsbar_b=None, abar=None, bbar=None, want_hs=False,
                           accumulate=False, work=None, stream=None):
    """reduce_by_index VJP by the general rule (C: adpar_vjp_hist_general).

    Returns (abar, bbar, hs_a, hs_b); bbar and hs_b only for linrec, the hs
    arrays only with ``want_hs``.
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = a.numel()
    dt = _dtype_code(a)
    it = _itype_code(inds)
    w = 2 if opc == OP_LINREC else 1
    if abar is None:
        abar = torch.zeros_like(a) if accumulate else torch.empty_like(a)
    if w == 2 and bbar is None:
        bbar = torch.zeros_like(a) if accumulate else torch.empty_like(a)
    for t in (b, abar, bbar):
        if t is not None and (t.dtype != a.dtype or t.numel() != n):
            raise ValueError("all element arrays must share dtype and length")
    if inds.numel() != n:
        raise ValueError("inds must have one index per element")
    hs_a = torch.empty(m, dtype=a.dtype, device=a.device) if want_hs else None
    hs_b = torch.empty(m, dtype=a.dtype, device=a.device) if want_hs and w == 2 else None
    need = adpar_workspace_size(RULE_HIST_GENERAL, opc, dt, n, m)
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    st = lib().adpar_vjp_hist_general(OpDesc(opc, dt, w), n, m, _ptr(a), _ptr(b), _ptr(inds), it, _ptr(hsbar_a),
                                      _ptr(hsbar_b), _ptr(abar), _ptr(bbar), _ptr(hs_a), _ptr(hs_b),
                                      ACCUMULATE if accumulate else 0, _ptr(work), work.numel(), _stream(stream))
    _check("adpar_vjp_hist_general", st)
    return abar, bbar, hs_a, hs_b


def adpar_vjp_scan_vec(op, a, ybar_a, b=None, ybar_b=None, abar=None, bbar=None, accumulate=False, work=None,
                       stream=None):
    """VJP of a scan over the rows of [n, d] arrays, column by column (C: adpar_vjp_scan_vec).
    Returns (abar, bbar, work)."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    if ybar_a.dim() != 2:
        raise ValueError("arrays must be [n, d]")
    n, d = ybar_a.shape
    dt = _dtype_code(ybar_a)
    w = 2 if opc == OP_LINREC else 1
    for t in (a, b, ybar_b, abar, bbar):
        if t is not None and (t.dtype != ybar_a.dtype or tuple(t.shape) != (n, d) or not t.is_contiguous()):
            raise ValueError("all arrays must be contiguous [n, d] of one dtype")
    if abar is None:
        abar = torch.zeros_like(ybar_a) if accumulate else torch.empty_like(ybar_a)
    if w == 2 and bbar is None:
        bbar = torch.zeros_like(ybar_a) if accumulate else torch.empty_like(ybar_a)
    need = adpar_workspace_size(RULE_SCAN_VEC, opc, dt, n, d)
    if work is None or work.numel() < need:
        work = workspace(need, ybar_a.device)
    st = lib().adpar_vjp_scan_vec(OpDesc(opc, dt, w), n, d, _ptr(a), _ptr(b), _ptr(ybar_a), _ptr(ybar_b),
                                  _ptr(abar), _ptr(bbar), ACCUMULATE if accumulate else 0, _ptr(work),
                                  work.numel(), _stream(stream))
    _check("adpar_vjp_scan_vec", st)
    return abar, bbar, work


def adpar_jvp_scan(op, a, adot, b=None, bdot=None, want_ys=False, ysdot_a=None, ysdot_b=None, work=None,
                   stream=None):
    """Forward-mode tangent of an inclusive scan (C: adpar_jvp_scan).

    Returns (ysdot_a, ysdot_b, ys_a, ys_b); the b parts for linrec only, the
    ys parts when ``want_ys``."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = a.numel()
    dt = _dtype_code(a)
    w = 2 if opc == OP_LINREC else 1
    for t in (adot, b, bdot, ysdot_a, ysdot_b):
        if t is not None and (t.dtype != a.dtype or t.numel() != n):
            raise ValueError("all scan arrays must share dtype and length")
    if ysdot_a is None:
        ysdot_a = torch.empty_like(a)
    if w == 2 and ysdot_b is None:
        ysdot_b = torch.empty_like(a)
    ys_a = torch.empty_like(a) if want_ys else None
    ys_b = torch.empty_like(a) if (want_ys and w == 2) else None
    need = adpar_workspace_size(RULE_SCAN | WS_MINIMAL, opc, dt, n)
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    st = lib().adpar_jvp_scan(OpDesc(opc, dt, w), n, _ptr(a), _ptr(b), _ptr(adot), _ptr(bdot), _ptr(ys_a),
                              _ptr(ys_b), _ptr(ysdot_a), _ptr(ysdot_b), _ptr(work), work.numel(), _stream(stream))
    _check("adpar_jvp_scan", st)
    return ysdot_a, ysdot_b, ys_a, ys_b


def adpar_scan(op, a, b=None, ys_a=None, ys_b=None, work=None, stream=None):
    """Primal inclusive scan (C: adpar_scan).  Returns (ys_a, ys_b, work)."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = a.numel()
    dt = _dtype_code(a)
    w = 2 if opc == OP_LINREC else 1
    if ys_a is None:
        ys_a = torch.empty_like(a)
    if w == 2 and ys_b is None:
        ys_b = torch.empty_like(a)
    need = adpar_workspace_size(RULE_SCAN | WS_MINIMAL, opc, dt, n)  # the forward scan needs no more
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    st = lib().adpar_scan(OpDesc(opc, dt, w), n, _ptr(a), _ptr(b), _ptr(ys_a), _ptr(ys_b),
                          _ptr(work), work.numel(), _stream(stream))
    _check("adpar_scan", st)
    return ys_a, ys_b, work


def adpar_vjp_scan_noalloc(op, a, ybar_a, b=None, ybar_b=None, abar=None, bbar=None, ys_a=None,
                           ys_b=None, accumulate=False, stream=None):
    """Scan VJP that allocates nothing in the library (C: adpar_vjp_scan_noalloc).

    For callers that cannot allocate device memory at the call site: the
    library uses its static device scratch instead of a workspace.  Output
    tensors must be passed in (none is allocated here either).  Returns
    (abar, bbar).  Calls that overlap on the GPU race on the shared scratch.
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    w = 2 if opc == OP_LINREC else 1
    if abar is None or (w == 2 and bbar is None):
        raise ValueError("pass the output adjoint tensors: this entry point allocates nothing")
    n = ybar_a.numel()
    dt = _dtype_code(ybar_a)
    # every array is read or written over n elements on the device: one of
    # another dtype or length, or one in host memory, would be overrun
    given = [(name, t) for name, t in (("a", a), ("b", b), ("ybar_a", ybar_a), ("ybar_b", ybar_b),
                                       ("abar", abar), ("bbar", bbar), ("ys_a", ys_a), ("ys_b", ys_b))
             if t is not None]
    for name, t in given:
        if t.dtype != ybar_a.dtype or t.numel() != n:
            raise ValueError("%s must have ybar_a's dtype and length (%s, %d), got (%s, %d)"
                             % (name, ybar_a.dtype, n, t.dtype, t.numel()))
    for name, t in given:
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA tensor" % name)
    st = lib().adpar_vjp_scan_noalloc(OpDesc(opc, dt, w), n, _ptr(a), _ptr(b), _ptr(ybar_a),
                                      _ptr(ybar_b), _ptr(abar), _ptr(bbar), _ptr(ys_a), _ptr(ys_b),
                                      ACCUMULATE if accumulate else 0, _stream(stream))
    _check("adpar_vjp_scan_noalloc", st)
    return abar, bbar


def adpar_noalloc_scratch_bytes():
    """Bytes of the static scratch behind adpar_vjp_scan_noalloc."""
    return lib().adpar_noalloc_scratch_bytes()


def adpar_noalloc_status(stream=None):
    """Device status word of the last adpar_vjp_scan_noalloc call on the
    current device (C: adpar_noalloc_status; synchronises the stream)."""
    st = C.c_int(0)
    _check("adpar_noalloc_status", lib().adpar_noalloc_status(_stream(stream), C.byref(st)))
    return st.value


def adpar_noalloc_selftest_timeout(stream=None):
    """Bounded-wait timeout diagnostic in the static scratch
    (C: adpar_noalloc_selftest_timeout)."""
    _check("adpar_noalloc_selftest_timeout", lib().adpar_noalloc_selftest_timeout(_stream(stream)))


def _scalar_dev(x, like):
    if isinstance(x, torch.Tensor):
        return x.reshape(1).to(device=like.device, dtype=like.dtype).contiguous()
    return torch.tensor([float(x)], dtype=like.dtype, device=like.device)


def adpar_vjp_reduce(op, a, ybar=1.0, abar=None, want_y=False, want_argidx=False, want_aux=False,
                     logdomain=False, want_sign=False, accumulate=False, work=None, stream=None):
    """VJP of reduce (C: adpar_vjp_reduce).

    Returns a dict with ``abar`` and, when asked for, ``y`` (device scalar),
    ``argidx`` (int64 device scalar), ``aux`` (ProdAux, read back to the
    host) and ``sign`` (int8 [n]).
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = a.numel()
    dt = _dtype_code(a)
    yb = _scalar_dev(ybar, a)
    if abar is None:
        abar = torch.zeros_like(a) if accumulate else torch.empty_like(a)
    y = torch.empty(1, dtype=a.dtype, device=a.device) if want_y else None
    arg = torch.empty(1, dtype=torch.int64, device=a.device) if want_argidx else None
    aux = torch.empty(PROD_AUX_BYTES, dtype=torch.uint8, device=a.device) if want_aux else None
    sg = torch.empty(n, dtype=torch.int8, device=a.device) if want_sign else None
    need = adpar_workspace_size(RULE_REDUCE, opc, dt, n)
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    flags = (ACCUMULATE if accumulate else 0) | (PROD_LOGDOMAIN if logdomain else 0)
    st = lib().adpar_vjp_reduce(OpDesc(opc, dt, 1), n, _ptr(a), _ptr(yb), _ptr(abar), _ptr(y), _ptr(arg),
                                _ptr(aux), _ptr(sg), flags, _ptr(work), work.numel(), _stream(stream))
    _check("adpar_vjp_reduce", st)
    out = {"abar": abar, "work": work}
    if want_y:
        out["y"] = y
    if want_argidx:
        out["argidx"] = arg
    if want_sign:
        out["sign"] = sg
    if want_aux:
        raw = aux.cpu().numpy().tobytes()
        out["aux"] = ProdAux.from_buffer_copy(raw)
    return out


def adpar_vjp_hist(op, inds, m, hsbar, vals=None, valsbar=None, want_hs=False, want_argidx=False,
                   want_aux=False, logdomain=False, want_sign=False, accumulate=False, work=None,
                   stream=None):
    """VJP of reduce_by_index (C: adpar_vjp_hist).

    Returns a dict with ``valsbar`` and, when asked for, ``hs`` [m],
    ``argidx`` [m] int64, ``aux`` (structured numpy array of ProdAux, [m])
    and ``sign`` [n] int8.
    """
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = inds.numel()
    ref = hsbar
    dt = _dtype_code(ref)
    it = _itype_code(inds)
    if valsbar is None:
        valsbar = (torch.zeros if accumulate else torch.empty)(n, dtype=ref.dtype, device=ref.device)
    hs = torch.empty(m, dtype=ref.dtype, device=ref.device) if want_hs else None
    arg = torch.empty(m, dtype=torch.int64, device=ref.device) if want_argidx else None
    aux = torch.empty(max(m, 1) * PROD_AUX_BYTES, dtype=torch.uint8, device=ref.device) if want_aux else None
    sg = torch.empty(n, dtype=torch.int8, device=ref.device) if want_sign else None
    need = adpar_workspace_size(RULE_HIST, opc, dt, n, m)
    if work is None or work.numel() < need:
        work = workspace(need, ref.device)
    flags = (ACCUMULATE if accumulate else 0) | (PROD_LOGDOMAIN if logdomain else 0)
    st = lib().adpar_vjp_hist(OpDesc(opc, dt, 1), n, m, _ptr(vals), _ptr(inds), it, _ptr(hsbar), _ptr(valsbar),
                              _ptr(hs), _ptr(arg), _ptr(aux), _ptr(sg), flags, _ptr(work), work.numel(),
                              _stream(stream))
    _check("adpar_vjp_hist", st)
    out = {"valsbar": valsbar, "work": work}
    if want_hs:
        out["hs"] = hs
    if want_argidx:
        out["argidx"] = arg
    if want_sign:
        out["sign"] = sg
    if want_aux:
        import numpy as np
        dtype = np.dtype([("nzero", "<i8"), ("first_zero", "<i8"), ("exp2", "<i8"), ("mant", "<f8"),
                          ("log_abs_nz", "<f8"), ("sign", "<i4"), ("reserved", "<i4")])
        out["aux"] = np.frombuffer(aux.cpu().numpy().tobytes(), dtype=dtype)[:m]
    return out


def adpar_vjp_scatter(is_, ysbar, vsbar=None, ys=None, xs_saved=None, accumulate=False, stream=None):
    """VJP of scatter (C: adpar_vjp_scatter).  ``ysbar`` becomes xsbar in place.

    Returns (xsbar, vsbar).  With ``ys`` and ``xs_saved`` the scattered
    positions of ``ys`` are restored too.
    """
    m = is_.numel()
    n = ysbar.numel()
    dt = _dtype_code(ysbar)
    it = _itype_code(is_)
    if vsbar is None:
        vsbar = (torch.zeros if accumulate else torch.empty)(m, dtype=ysbar.dtype, device=ysbar.device)
    flags = (ACCUMULATE if accumulate else 0) | (SCATTER_RESTORE if ys is not None else 0)
    st = lib().adpar_vjp_scatter(dt, n, m, _ptr(is_), it, _ptr(ysbar), _ptr(vsbar), _ptr(ys), _ptr(xs_saved),
                                 flags, _stream(stream))
    _check("adpar_vjp_scatter", st)
    return ysbar, vsbar


def adpar_vjp_map_acc(g, as_, is_, xsbar, ws=None, width=1, asbar=None, wsbar=None, want_wsbar=False,
                      accumulate=False, stream=None):
    """VJP of map with a free array (C: adpar_vjp_map_acc).  Returns (asbar, wsbar)."""
    gc = GFUNS[g] if isinstance(g, str) else int(g)
    nj = is_.numel()
    na = as_.numel() // width
    dt = _dtype_code(as_)
    it = _itype_code(is_)
    if asbar is None:
        asbar = torch.zeros_like(as_) if accumulate else torch.empty_like(as_)
    if want_wsbar and wsbar is None and ws is not None:
        wsbar = torch.zeros_like(ws) if accumulate else torch.empty_like(ws)
    st = lib().adpar_vjp_map_acc(gc, dt, nj, na, width, _ptr(as_), _ptr(is_), it, _ptr(ws), _ptr(xsbar),
                                 _ptr(asbar), _ptr(wsbar), ACCUMULATE if accumulate else 0, None, 0,
                                 _stream(stream))
    _check("adpar_vjp_map_acc", st)
    return asbar, wsbar


def adpar_kmeans_hessdiag(k, ybar, work, Hdiag=None, accumulate=False, stream=None):
    """Hessian diagonal [k, 32] of the k-means cost in C (C: adpar_kmeans_hessdiag), from the
    counts that the preceding adpar_kmeans_vjp call (gradient requested) left in ``work``."""
    dev = work.device
    yb = _scalar_dev(1.0 if ybar is None else ybar, torch.empty(0, device=dev))
    if Hdiag is None:
        Hdiag = (torch.zeros if accumulate else torch.empty)(k, 32, dtype=torch.float32, device=dev)
    st = lib().adpar_kmeans_hessdiag(int(k), _ptr(yb), _ptr(work), work.numel(), _ptr(Hdiag),
                                     ACCUMULATE if accumulate else 0, _stream(stream))
    _check("adpar_kmeans_hessdiag", st)
    return Hdiag


def adpar_kmeans_vjp(X, C, ybar=None, want_grad=True, want_argmin=False, Cbar=None, accumulate=False,
                     work=None, stream=None):
    """k-means loss and its gradient in C (C: adpar_kmeans_vjp).

    Returns a dict with ``loss`` (device FP32 scalar), ``Cbar`` [k, d] when
    ``want_grad`` and ``argmin`` [N] int32 when asked for.
    """
    N, d = X.shape
    k = C.shape[0]
    if X.dtype != torch.float32 or C.dtype != torch.float32:
        raise TypeError("k-means takes FP32 X and C")
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    arg = torch.empty(N, dtype=torch.int32, device=X.device) if want_argmin else None
    yb = None
    if want_grad:
        yb = _scalar_dev(1.0 if ybar is None else ybar, X)
        if Cbar is None:
            Cbar = torch.zeros_like(C) if accumulate else torch.empty_like(C)
    else:
        Cbar = None
    need = adpar_workspace_size(RULE_KMEANS, 0, F32, N, k)
    if work is None or work.numel() < need:
        work = workspace(need, X.device)
    st = lib().adpar_kmeans_vjp(N, d, k, _ptr(X), _ptr(C), _ptr(yb), _ptr(loss), _ptr(arg), _ptr(Cbar),
                                ACCUMULATE if accumulate else 0, _ptr(work), work.numel(), _stream(stream))
    _check("adpar_kmeans_vjp", st)
    out = {"loss": loss, "work": work}
    if want_grad:
        out["Cbar"] = Cbar
    if want_argmin:
        out["argmin"] = arg
    return out


def adpar_reduce(op, a, want_argidx=False, work=None, stream=None):
    """Primal reduce (C: adpar_reduce).  Returns (y [1], argidx [1] or None)."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = a.numel()
    dt = _dtype_code(a)
    y = torch.empty(1, dtype=a.dtype, device=a.device)
    arg = torch.empty(1, dtype=torch.int64, device=a.device) if want_argidx else None
    need = adpar_workspace_size(RULE_REDUCE, opc, dt, n)
    if work is None or work.numel() < need:
        work = workspace(need, a.device)
    _check("adpar_reduce", lib().adpar_reduce(OpDesc(opc, dt, 1), n, _ptr(a), _ptr(y), _ptr(arg), None,
                                              _ptr(work), work.numel(), _stream(stream)))
    return y, arg


def adpar_hist(op, vals, inds, m, want_argidx=False, work=None, stream=None):
    """Primal reduce_by_index (C: adpar_hist).  Returns (hs [m], argidx [m] or None)."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = inds.numel()
    dt = _dtype_code(vals)
    hs = torch.empty(m, dtype=vals.dtype, device=vals.device)
    arg = torch.empty(m, dtype=torch.int64, device=vals.device) if want_argidx else None
    need = adpar_workspace_size(RULE_HIST, opc, dt, n, m)
    if work is None or work.numel() < need:
        work = workspace(need, vals.device)
    _check("adpar_hist", lib().adpar_hist(OpDesc(opc, dt, 1), n, m, _ptr(vals), _ptr(inds), _itype_code(inds),
                                          _ptr(hs), _ptr(arg), None, _ptr(work), work.numel(), _stream(stream)))
    return hs, arg


def adpar_scatter(is_, vs, ys_inout, xs_saved=None, stream=None):
    """Primal scatter in place (C: adpar_scatter).  Returns ys_inout."""
    _check("adpar_scatter", lib().adpar_scatter(_dtype_code(vs), ys_inout.numel(), is_.numel(), _ptr(is_),
                                                _itype_code(is_), _ptr(vs), _ptr(ys_inout), _ptr(xs_saved),
                                                _stream(stream)))
    return ys_inout


def adpar_map_acc(g, as_, is_, ws=None, width=1, stream=None):
    """Primal map with a free array (C: adpar_map_acc).  Returns xs [nj]."""
    gc = GFUNS[g] if isinstance(g, str) else int(g)
    nj = is_.numel()
    xs = torch.empty(nj, dtype=as_.dtype, device=as_.device)
    _check("adpar_map_acc", lib().adpar_map_acc(gc, _dtype_code(as_), nj, as_.numel() // width, width, _ptr(as_),
                                                _ptr(is_), _itype_code(is_), _ptr(ws), _ptr(xs),
                                                _stream(stream)))
    return xs


def adpar_selftest_timeout(work=None, stream=None):
    """Run the bounded-wait timeout diagnostic; returns the workspace used."""
    if work is None:
        work = workspace(512)
    _check("adpar_selftest_timeout", lib().adpar_selftest_timeout(_ptr(work), work.numel(), _stream(stream)))
    return work


# ------------------------------------------------------------ forward mode
def _aux_records(buf, count):
    import numpy as np
    return np.frombuffer(buf.cpu().numpy().tobytes(), dtype=np.dtype(JVP_AUX_DTYPE))[:count]


def adpar_jvp_reduce(op, a, adot, want_y=False, want_aux=False, work=None, stream=None):
    """Forward mode of reduce (C: adpar_jvp_reduce).  Returns a dict with
    ``ydot`` (device scalar), ``y`` when asked for, and ``aux`` (ln|ydot|,
    sign; read back to the host) when asked for."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = adot.numel()
    dt = _dtype_code(adot)
    if a is not None and (a.dtype != adot.dtype or a.numel() != n):
        raise ValueError("a and adot must share dtype and length")
    ydot = torch.empty(1, dtype=adot.dtype, device=adot.device)
    y = torch.empty(1, dtype=adot.dtype, device=adot.device) if want_y else None
    aux = torch.empty(JVP_AUX_BYTES, dtype=torch.uint8, device=adot.device) if want_aux else None
    need = adpar_workspace_size(RULE_JVP_REDUCE, opc, dt, n)
    if work is None or work.numel() < need:
        work = workspace(need, adot.device)
    _check("adpar_jvp_reduce", lib().adpar_jvp_reduce(OpDesc(opc, dt, 1), n, _ptr(a), _ptr(adot), _ptr(y),
                                                      _ptr(ydot), _ptr(aux), _ptr(work), work.numel(),
                                                      _stream(stream)))
    out = {"ydot": ydot}
    if want_y:
        out["y"] = y
    if want_aux:
        out["aux"] = _aux_records(aux, 1)[0]
    return out


def adpar_jvp_hist(op, vals, vdot, inds, m, want_hs=False, want_aux=False, work=None, stream=None):
    """Forward mode of reduce_by_index (C: adpar_jvp_hist).  Returns a dict
    with ``hsdot`` [m], ``hs`` [m] when asked for, and ``aux`` (structured
    numpy array of ln|hsdot|, sign; * only) when asked for."""
    opc = OPS[op] if isinstance(op, str) else int(op)
    n = inds.numel()
    dt = _dtype_code(vdot)
    for t in (vals, vdot):
        if t is not None and (t.dtype != vdot.dtype or t.numel() != n):
            raise ValueError("vals, vdot and inds must share length (and vals, vdot dtype)")
    hsdot = torch.empty(m, dtype=vdot.dtype, device=vdot.device)
    hs = torch.empty(m, dtype=vdot.dtype, device=vdot.device) if want_hs else None
    aux = torch.empty(max(m, 1) * JVP_AUX_BYTES, dtype=torch.uint8, device=vdot.device) if want_aux else None
    need = adpar_workspace_size(RULE_JVP_HIST, opc, dt, n, m)
    if work is None or work.numel() < need:
        work = workspace(need, vdot.device)
    _check("adpar_jvp_hist", lib().adpar_jvp_hist(OpDesc(opc, dt, 1), n, m, _ptr(vals), _ptr(vdot), _ptr(inds),
                                                  _itype_code(inds), _ptr(hs), _ptr(hsdot), _ptr(aux), _ptr(work),
                                                  work.numel(), _stream(stream)))
    out = {"hsdot": hsdot}
    if want_hs:
        out["hs"] = hs
    if want_aux:
        out["aux"] = _aux_records(aux, m)
    return out


def adpar_jvp_scatter(is_, vsdot, ysdot_inout, stream=None):
    """Forward mode of scatter (C: adpar_jvp_scatter): ``ysdot_inout`` holds
    xsdot on entry and ysdot on return."""
    if vsdot.dtype != ysdot_inout.dtype or vsdot.numel() != is_.numel():
        raise ValueError("vsdot must match is_ in length and ysdot in dtype")
    _check("adpar_jvp_scatter", lib().adpar_jvp_scatter(_dtype_code(vsdot), ysdot_inout.numel(), is_.numel(),
                                                        _ptr(is_), _itype_code(is_), _ptr(vsdot), _ptr(ysdot_inout),
                                                        _stream(stream)))
    return ysdot_inout


def adpar_jvp_map_acc(g, as_, is_, asdot, ws=None, wsdot=None, width=1, stream=None):
    """Forward mode of map with a free array (C: adpar_jvp_map_acc).  Returns xsdot [nj]."""
    gc = GFUNS[g] if isinstance(g, str) else int(g)
    nj = is_.numel()
    if asdot.dtype != as_.dtype or asdot.numel() != as_.numel():
        raise ValueError("asdot must match as_")
    for t in (ws, wsdot):
        if t is not None and (t.dtype != as_.dtype or t.numel() != nj * width):
            raise ValueError("ws and wsdot must hold nj * width values of as_'s dtype")
    xsdot = torch.empty(nj, dtype=as_.dtype, device=as_.device)
    _check("adpar_jvp_map_acc", lib().adpar_jvp_map_acc(gc, _dtype_code(as_), nj, as_.numel() // width, width,
                                                        _ptr(as_), _ptr(is_), _itype_code(is_), _ptr(ws),
                                                        _ptr(asdot), _ptr(wsdot), _ptr(xsdot), _stream(stream)))
    return xsdot


def adpar_kmeans_fwd_rev(X, C_, Cdot, ybar=1.0, Cbardot=None, accumulate=False, work=None, stream=None):
    """Forward over reverse for the k-means cost (C: adpar_kmeans_fwd_rev):
    the tangent along Cdot of the gradient in C (a Hessian-vector product)
    and of the loss.  Returns (ydot device scalar, Cbardot [k, d])."""
    N, d = X.shape
    k = C_.shape[0]
    for t in (X, C_, Cdot):
        if t.dtype != torch.float32:
            raise TypeError("k-means takes FP32 X, C and Cdot")
    if Cdot.shape != C_.shape:
        raise ValueError("Cdot must have C's shape")
    yb = _scalar_dev(ybar, C_)
    ydot = torch.empty(1, dtype=torch.float32, device=C_.device)
    if Cbardot is None:
        Cbardot = torch.zeros_like(C_) if accumulate else torch.empty_like(C_)
    need = adpar_workspace_size(RULE_KMEANS_FWD_REV, 0, F32, N, k)
    if work is None or work.numel() < need:
        work = workspace(need, C_.device)
    _check("adpar_kmeans_fwd_rev", lib().adpar_kmeans_fwd_rev(N, d, k, _ptr(X), _ptr(C_), _ptr(Cdot), _ptr(yb),
                                                              _ptr(ydot), _ptr(Cbardot),
                                                              ACCUMULATE if accumulate else 0, _ptr(work),
                                                              work.numel(), _stream(stream)))
    return ydot, Cbardot


def adpar_kmeans_hessdiag_fwd_rev(X, C_, ybar=1.0, stream=None):
    """Hessian diagonal of the k-means cost in C by forward over reverse: the
    cost's Hessian is diagonal, so H 1 is its diagonal."""
    _, H = adpar_kmeans_fwd_rev(X, C_, torch.ones_like(C_), ybar=ybar, stream=stream)
    return H
