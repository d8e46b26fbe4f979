/*
 * adpar.h -- C ABI of libadpar: tape-free reverse-mode adjoints (VJPs) of
 * bulk-parallel operators, after "AD for an Array Language with Nested
 * Parallelism" (arXiv 2202.10297), as hand-written CUDA kernels for GB300
 * (sm_103a).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.    Every array argument is a DEVICE pointer unless it is marked
 *            "host".  The caller allocates and owns every buffer; the
 *            library allocates nothing.  Arrays are dense and contiguous
 *            (structure of arrays for multi-component elements) and must
 *            start on a 16-byte boundary (ADPAR_ERR_ALIGN otherwise).
 * Streams.   `stream` is a cudaStream_t passed as void* (NULL = legacy
 *            default stream).  Every call only enqueues work on it and
 *            returns; nothing synchronises the host.
 * Workspace. Calls that take (work, work_bytes) need scratch device memory
 *            of at least adpar_workspace_size(...) bytes, 256-byte aligned.
 *            Its contents need no initialisation and are clobbered; two
 *            calls in flight at once must not share one workspace.
 * Adjoints.  Output adjoints are overwritten (x_bar = contribution) unless
 *            flags has ADPAR_ACCUMULATE, in which case the contribution is
 *            added (x_bar += contribution), as in Eq. rewrite-adj (Sec. 2).
 * Recompute. Every rule re-executes the primal from its inputs (Sec. 4's
 *            redundant execution); nothing saved by an earlier call (no
 *            tape) is read.  Within one call a pass may leave the
 *            re-executed forward result in the workspace for the next
 *            pass (the FP64 scan, see adpar_vjp_scan).
 * Errors.    Argument errors are detected on the host and returned before
 *            anything is enqueued.  Device-side give-ups (a bounded wait
 *            that ran out) are recorded in the workspace and read back with
 *            adpar_workspace_status().  Kernel launch failures return
 *            ADPAR_ERR_CUDA.
 * NaN/inf.   Inputs holding NaN or infinities are outside the contract:
 *            results are unspecified, but no kernel faults or hangs.
 */
#ifndef ADPAR_H
#define ADPAR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* element types of values and of indices */
typedef enum { ADPAR_F32 = 0, ADPAR_F64 = 1 } adpar_dtype;
typedef enum { ADPAR_I32 = 0, ADPAR_I64 = 1 } adpar_itype;

/* associative operators (Sec. 5.1 and 5.2).  LINREC is the pair operator
 * (a1,b1) (.) (a2,b2) = (a2*a1, a2*b1 + b2) of a first-order linear
 * recurrence; its elements are two arrays a, b (width 2). */
typedef enum {
    ADPAR_OP_ADD = 0,
    ADPAR_OP_MUL = 1,
    ADPAR_OP_MIN = 2,
    ADPAR_OP_MAX = 3,
    ADPAR_OP_LINREC = 4,
    ADPAR_OP_MATREC2 = 5   /* 2x2 matrix linear recurrence: adpar_vjp_scan_wide only */
} adpar_op;

/* map bodies g for adpar_vjp_map_acc (Sec. 5.4) */
typedef enum {
    ADPAR_G_GATHER = 0,     /* x_j = as[is_j]                               */
    ADPAR_G_SCALE = 1,      /* x_j = as[is_j] * ws_j                        */
    ADPAR_G_SQDIST_ROW = 2  /* x_j = sum_k (ws[j,k] - as[is_j,k])^2, rows of width */
} adpar_gfun;

/* rules, for adpar_workspace_size */
typedef enum {
    ADPAR_RULE_REDUCE = 0,
    ADPAR_RULE_SCAN = 1,
    ADPAR_RULE_HIST = 2,
    ADPAR_RULE_SCATTER = 3,
    ADPAR_RULE_MAP_ACC = 4,
    ADPAR_RULE_KMEANS = 5,
    ADPAR_RULE_REDUCE_GENERAL = 6,
    ADPAR_RULE_SCAN_VEC = 7,  /* m = the vector length d */
    ADPAR_RULE_HIST_GENERAL = 8,
    ADPAR_RULE_SCAN_WIDE = 9,
    ADPAR_RULE_JVP_REDUCE = 10,     /* adpar_jvp_reduce                       */
    ADPAR_RULE_JVP_HIST = 11,       /* adpar_jvp_hist; m = bins               */
    ADPAR_RULE_KMEANS_FWD_REV = 12  /* adpar_kmeans_fwd_rev; n = points, m = centroids */
} adpar_rule;

/* or'ed into the rule of adpar_workspace_size: the smallest workspace the
 * call accepts instead of the size that runs it at full speed (the two
 * differ only for the FP64 MUL and LINREC scans) */
#define ADPAR_WS_MINIMAL 0x100

typedef enum {
    ADPAR_OK = 0,
    ADPAR_ERR_INVALID = 1,     /* null pointer, negative size, bad enum value   */
    ADPAR_ERR_UNSUPPORTED = 2, /* valid combination this library does not do    */
    ADPAR_ERR_ALIGN = 3,       /* an array does not start on a 16-byte boundary */
    ADPAR_ERR_WORKSPACE = 4,   /* work is NULL, misaligned or too small         */
    ADPAR_ERR_CUDA = 5,        /* a CUDA call or kernel launch failed           */
    ADPAR_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up            */
    ADPAR_ERR_TOO_LARGE = 7    /* needs more than the static no-allocation scratch */
} adpar_status;

/* flags */
#define ADPAR_ACCUMULATE      0x1u /* x_bar += contribution (else x_bar = contribution) */
#define ADPAR_PROD_LOGDOMAIN  0x4u /* * rules: write ln|contribution| and its sign      */
#define ADPAR_SCATTER_RESTORE 0x8u /* scatter: also restore ys[is_j] = xs_saved[j]      */
#define ADPAR_FULL_LIN_O      0x10u /* wide scans: the return sweep on full d x d lin_o   */

/* operator descriptor: op (adpar_op), dtype (adpar_dtype) of the values,
 * width = number of arrays per element (1, or 2 for ADPAR_OP_LINREC). */
typedef struct {
    int32_t op;
    int32_t dtype;
    int32_t width;
} adpar_opdesc;

/* Result of the recomputed product forward sweep of Sec. 5.1.1: the
 * number of zeros, the lowest zero index, and the product of the nonzero
 * elements in scaled form  p_nz = mant * 2^exp2  (0.5 <= |mant| < 1, or
 * mant = 0 when there are no elements), with ln|p_nz| and sign(p_nz). */
typedef struct {
    int64_t nzero;
    int64_t first_zero;  /* -1 when there is no zero */
    int64_t exp2;
    double mant;
    double log_abs_nz;
    int32_t sign;        /* -1, 0 or +1 */
    int32_t reserved;
} adpar_prod_aux;

/* ------------------------------------------------------------------ */
/* Library                                                             */
/* ------------------------------------------------------------------ */

/* Human-readable name of a status code (static storage, never NULL). */
const char *adpar_status_string(int status);

/* Version string of the library (static storage). */
const char *adpar_version(void);

/* Bytes of workspace needed by `rule` for an operator `desc` over n
 * elements (m = number of bins for HIST, of destination elements for
 * SCATTER, of accumulator rows for MAP_ACC; for KMEANS n = points, m =
 * centroids).  Returns 0 when the rule needs none, and (size_t)-1 for an
 * invalid request.  With ADPAR_WS_MINIMAL or'ed into rule: the smallest
 * size the call accepts. */
size_t adpar_workspace_size(int rule, adpar_opdesc desc, int64_t n, int64_t m);

/* Waits for `stream`, then reads the device-side status word that the
 * last call using `work` left there (ADPAR_OK, or ADPAR_ERR_TIMEOUT when
 * a bounded wait inside a kernel gave up).  *device_status receives it
 * (host pointer).  Returns ADPAR_ERR_CUDA if the read itself fails. */
int adpar_workspace_status(const void *work, void *stream, int *device_status);

/* Diagnostic of the failure detection (no counterpart in the paper):
 * enqueues one kernel whose bounded wait on a flag that nothing sets runs
 * out (after about a second), so adpar_workspace_status(work) then reports
 * ADPAR_ERR_TIMEOUT while the CUDA context stays usable.  work: at least
 * 512 bytes, 256-byte aligned. */
int adpar_selftest_timeout(void *work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* reduce (Sec. 5.1 and 5.1.1)                                         */
/* ------------------------------------------------------------------ */
/* y = a_0 (.) a_1 (.) ... (.) a_{n-1} and its adjoint a_bar, for
 * op = ADD, MUL, MIN, MAX (width 1), dtype F32 or F64.
 *   ADD:  a_bar_i = y_bar                                   (Sec. 5.1.1)
 *   MUL:  the three cases of Sec. 5.1.1 on the zero count z:
 *         z = 0: a_bar_i = p_nz / a_i * y_bar;  z = 1: a_bar_{i0} = p_nz *
 *         y_bar (p_nz = product of the nonzero elements), all others 0;
 *         z >= 2: all 0.  The forward sweep is re-executed as a map-reduce
 *         of (zero count, lowest zero index, scaled nonzero product), so
 *         no intermediate underflows.
 *   MIN/MAX: (y, i_y) = argmin/argmax with the LOWEST index on ties
 *         (Sec. 5.1.1, "(first) index"); a_bar_{i_y} = y_bar, others 0.
 * Arguments:
 *   n          number of elements (0 allowed: y = neutral element).
 *   a          [n] input values, dtype.
 *   ybar       device scalar (dtype): the cotangent of y.
 *   abar       [n] output adjoint, dtype.  With ADPAR_PROD_LOGDOMAIN (MUL
 *              only) it receives ln|contribution| (-inf where it is 0).
 *   y_out      nullable device scalar (dtype): the recomputed y (MUL: the
 *              product rounded to dtype, 0 or subnormal on underflow).
 *   argidx_out nullable device int64 scalar: i_y (MIN/MAX; -1 if n == 0).
 *   aux_out    nullable device adpar_prod_aux (MUL only).
 *   abar_sign  nullable device int8 [n]: sign of each contribution
 *              (MUL with ADPAR_PROD_LOGDOMAIN only).
 * Flags: ADPAR_ACCUMULATE (not with LOGDOMAIN), ADPAR_PROD_LOGDOMAIN.
 * Workspace: adpar_workspace_size(ADPAR_RULE_REDUCE, desc, n, 0). */
int adpar_vjp_reduce(adpar_opdesc desc, int64_t n, const void *a, const void *ybar,
                     void *abar, void *y_out, int64_t *argidx_out,
                     adpar_prod_aux *aux_out, int8_t *abar_sign, uint32_t flags,
                     void *work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* scan (Sec. 5.2)                                                     */
/* ------------------------------------------------------------------ */
/* Inclusive scan rs_i = rs_{i-1} (.) as_i and its adjoint, for op = ADD,
 * MUL, MIN, MAX (width 1) and LINREC (width 2: arrays a, b), dtype F32 or
 * F64.  The return sweep is the one of Sec. 5.2: with
 *   J_left(i) = d(rs_{i-1} (.) as_i)/d rs_{i-1}   and
 *   J_right(i) = d(rs_{i-1} (.) as_i)/d as_i,
 * rs_bar_i = ys_bar_i + J_left(i+1)^T rs_bar_{i+1} (a backward linear
 * recurrence solved by a scan with the lin_o operator of Sec. 5.2) and
 * as_bar_i = J_right(i)^T rs_bar_i, as_bar_0 = rs_bar_0.  MAX/MIN keep the
 * gradient with the earlier element on ties.
 * Arguments:
 *   n            number of elements (0 allowed: nothing is written).
 *   a, b         [n] inputs (b only for LINREC, else NULL).
 *   ybar_a/_b    [n] cotangents of the outputs (ybar_b only for LINREC).
 *   abar, bbar   [n] output adjoints (bbar only for LINREC).
 *   ys_a, ys_b   nullable [n]: the recomputed primal outputs.
 * Flags: ADPAR_ACCUMULATE.
 * Workspace: adpar_workspace_size(ADPAR_RULE_SCAN, desc, n, 0).  For the
 * F64 MUL and LINREC scans that size includes room for the re-executed
 * forward result in factored form (each thread's local prefixes and its
 * carry, about 8 * width bytes per element), which saves the return sweep
 * a third of its FP64 arithmetic; any workspace of at least the
 * ADPAR_WS_MINIMAL size is accepted, and with less than the full size the
 * return sweep re-forms the primal prefixes itself (same results up to
 * rounding). */
int adpar_vjp_scan(adpar_opdesc desc, int64_t n, const void *a, const void *b,
                   const void *ybar_a, const void *ybar_b, void *abar, void *bbar,
                   void *ys_a, void *ys_b, uint32_t flags, void *work,
                   size_t work_bytes, void *stream);

/* VJP of an inclusive scan whose element is a vector of D scalars, by the
 * general lin_o of Sec. 5.2: J_left and J_right are D x D matrices and the
 * return sweep's recurrence rs_bar_i = ybar_i + J_left(i+1)^T rs_bar_{i+1}
 * is a reverse scan of affine maps (d, C) whose combine multiplies two
 * D x D matrices (neutral element (0, I)); then
 *   as_bar_i (+)= J_right(i)^T rs_bar_i (i >= 1),  as_bar_0 (+)= rs_bar_0.
 * Operators (desc.op, desc.width = D):
 *   ADPAR_OP_LINREC  D = 2: the element (a, b); the same recurrence as
 *                    adpar_vjp_scan's LINREC, through full 2x2 Jacobians.
 *   ADPAR_OP_MATREC2 D = 6: the element (M, v), M a row-major 2x2 matrix in
 *                    the first four scalars and v a 2-vector in the last
 *                    two; (M1, v1) (.) (M2, v2) = (M2 M1, M2 v1 + v2), the
 *                    affine maps h -> M h + v composed in scan order (the
 *                    second entry of ys_i is h_i = M_i h_{i-1} + v_i with
 *                    h_{-1} = 0; companion matrices give second-order
 *                    recurrences).
 * Arguments:
 *   n        elements (0 allowed).
 *   a        [n][D] row-major elements, dtype.
 *   ybar     [n][D] cotangent of the inclusive scan ys.
 *   abar     [n][D] output adjoint (overwritten, or += with ADPAR_ACCUMULATE).
 *   ys_out   nullable [n][D]: the recomputed inclusive scan.
 * The 2x2 matrix recurrence's J_left is I_3 (x) M (M acts on the two
 * columns of the matrix part and on the vector part alike), so by default
 * its return sweep carries C = I_3 (x) N with N a 2x2 matrix (10 scalars a
 * state instead of 42); ADPAR_FULL_LIN_O forces the full d x d lin_o for
 * either operator (same results up to rounding).
 * Every non-null array must start on a 16-byte boundary (ADPAR_ERR_ALIGN).
 * Flags: ADPAR_ACCUMULATE, ADPAR_FULL_LIN_O.
 * Workspace: adpar_workspace_size(ADPAR_RULE_SCAN_WIDE, desc, n, 0) (the
 * full lin_o's size, which covers both forms). */
int adpar_vjp_scan_wide(adpar_opdesc desc, int64_t n, const void *a, const void *ybar, void *abar,
                        void *ys_out, uint32_t flags, void *work, size_t work_bytes, void *stream);

/* Reduce by the GENERAL rule of Sec. 5.1, for any operator of this
 * library (ADD, MUL, MIN, MAX, and LINREC, which has no special rule):
 *   y = a_0 (.) a_1 (.) ... (.) a_{n-1},
 *   a_bar_i (+)= d(l_i (.) a_i (.) r_i)/d a_i ^T y_bar,
 * with l_i = a_0 (.) ... (.) a_{i-1} and r_i = a_{i+1} (.) ... (.) a_{n-1}
 * from a forward and a reverse exclusive scan (the neutral element at the
 * ends).  For LINREC that is (abar, bbar)_i = (rA (lA ybar_A + lB ybar_B),
 * rA ybar_B); for MUL the product of all other elements (no division, so
 * zeros are safe; values may underflow where adpar_vjp_reduce's scaled
 * rule would not: with factors of magnitude about 1/2..3/2 an FP32 product
 * underflows beyond a few thousand factors and an FP64 one beyond about
 * 16000, and every adjoint then rounds to 0; use adpar_vjp_reduce for long
 * products); for MIN/MAX the lowest index of the extremum.  Two
 * single-pass kernels: the forward carries, then the reverse pass.  LINREC
 * with the full workspace runs on per-thread runs (a carry pass storing
 * run carries and products, then a reverse pass forming rA from the runs'
 * products); with the ADPAR_WS_MINIMAL size, on the scan engine.
 * Arguments (as for adpar_vjp_scan; b, ybar_b, bbar, y_out_b for LINREC):
 *   n            number of elements (0 allowed: y = neutral element).
 *   a, b         [n] inputs.
 *   ybar_a/_b    device scalars (dtype): the cotangent of y.
 *   abar, bbar   [n] output adjoints.
 *   y_out_a/_b   nullable device scalars: the recomputed y.
 * Flags: ADPAR_ACCUMULATE.
 * Workspace: adpar_workspace_size(ADPAR_RULE_REDUCE_GENERAL, desc, n, 0)
 * (or with ADPAR_WS_MINIMAL: the smaller size, the engine's path). */
int adpar_vjp_reduce_general(adpar_opdesc desc, int64_t n, const void *a, const void *b,
                             const void *ybar_a, const void *ybar_b, void *abar, void *bbar,
                             void *y_out_a, void *y_out_b, uint32_t flags, void *work,
                             size_t work_bytes, void *stream);

/* VJP of a scan over d-vectors with an elementwise operator (Sec. 5.2, the
 * vectorised case): the arrays are row-major [n][d] and
 *   scan (map (.)) e xs = transpose xs |> map (scan (.) e) |> transpose,
 * i.e. d independent scans down the columns (for LINREC: d channels of the
 * recurrence h_t = a_t h_{t-1} + b_t).  Outputs as adpar_vjp_scan, column
 * by column; no transpose is materialised.
 * Arguments: n rows, d columns; a, b, ybar_a, ybar_b, abar, bbar [n][d]
 * (b, ybar_b, bbar for LINREC only; a may be NULL for ADD).
 * Flags: ADPAR_ACCUMULATE.
 * Workspace: adpar_workspace_size(ADPAR_RULE_SCAN_VEC, desc, n, d). */
int adpar_vjp_scan_vec(adpar_opdesc desc, int64_t n, int64_t d, const void *a, const void *b,
                       const void *ybar_a, const void *ybar_b, void *abar, void *bbar, uint32_t flags,
                       void *work, size_t work_bytes, void *stream);

/* Forward mode (JVP) of the inclusive scan: the tangent ysdot = d ys(as)
 * [asdot] of ys = scan (.) as, i.e. the forward-mode rule of the scan in the
 * sense of Sec. 3 (dual numbers carried through the operator):
 *   ys_i = ys_{i-1} (.) as_i,
 *   ysdot_i = J_left(i) ysdot_{i-1} + J_right(i) asdot_i,
 * computed as one single-pass scan of (value, tangent) pairs.  MIN/MAX give
 * the tangent of the running record (the earlier element on ties).
 * Arguments (b, bdot, ys_b, ysdot_b for LINREC only):
 *   n              number of elements (0 allowed).
 *   a, b           [n] inputs;  adot, bdot [n] their tangents.
 *   ys_a, ys_b     nullable [n]: the primal outputs.
 *   ysdot_a/_b     [n] the output tangents.
 * Workspace: as for adpar_scan (ADPAR_RULE_SCAN | ADPAR_WS_MINIMAL). */
int adpar_jvp_scan(adpar_opdesc desc, int64_t n, const void *a, const void *b, const void *adot,
                   const void *bdot, void *ys_a, void *ys_b, void *ysdot_a, void *ysdot_b, void *work,
                   size_t work_bytes, void *stream);

/* Log-domain form of a tangent whose value may leave the FP64 range (the
 * * rules below): ln|tangent| (-inf when it is 0) and its sign. */
typedef struct {
    double log_abs;
    int32_t sign;      /* -1, 0 or +1 */
    int32_t reserved;
} adpar_jvp_aux;

/* Forward mode (JVP) of reduce, the tangent of y = reduce (.) a along adot
 * (Sec. 3's dual numbers through the operators of Sec. 5.1 and 5.1.1):
 *   ADD      ydot = sum_i adot_i;
 *   MIN/MAX  ydot = adot_{i_y}, i_y the recomputed argmin/argmax with the
 *            lowest index on ties (0 for n = 0);
 *   MUL      the product rule on the recomputed forward sweep (zero count z,
 *            lowest zero i0, scaled product p of the nonzeros):
 *            z = 0: ydot = p sum_i adot_i / a_i;  z = 1: ydot = p adot_i0;
 *            z >= 2: ydot = 0.
 * Arguments:
 *   n           number of elements (0 allowed: ydot = 0).
 *   a, adot     [n] inputs and their tangent (dtype); a may be NULL for ADD
 *               when y_out is NULL.
 *   y_out       nullable device scalar: the recomputed y.
 *   ydot_out    device scalar (dtype): the tangent, rounded to dtype (0 or
 *               subnormal when a long product underflows).
 *   ydot_aux    nullable device adpar_jvp_aux: ln|ydot| and its sign,
 *               exact where the value under- or overflows.
 * Workspace: adpar_workspace_size(ADPAR_RULE_JVP_REDUCE, desc, n, 0).
 * Errors: ADPAR_ERR_INVALID (bad op/dtype/width, n < 0, missing pointers),
 * ADPAR_ERR_ALIGN, ADPAR_ERR_WORKSPACE; nothing is enqueued on error. */
int adpar_jvp_reduce(adpar_opdesc desc, int64_t n, const void *a, const void *adot, void *y_out,
                     void *ydot_out, adpar_jvp_aux *ydot_aux, void *work, size_t work_bytes, void *stream);

/* Forward mode of reduce_by_index (Sec. 5.1.2 on dual numbers): per bin b
 * the tangent of hs[b] = reduce (.) {vals_i : inds_i = b} along vdot, with
 * the cases of adpar_jvp_reduce per bin (ADD is reduce_by_index + of vdot;
 * MIN/MAX the tangent of the bin's lowest-index extremum; MUL the product
 * rule on the bin's zero count, lowest zero and scaled product).  Indices
 * outside [0, m) are ignored.
 * Arguments:
 *   n, m          elements and bins.
 *   vals, vdot    [n] values and tangents (dtype); vals may be NULL for ADD
 *                 when hs_out is NULL.
 *   inds          [n] bin indices (itype).
 *   hs_out        nullable [m]: the recomputed bins.
 *   hsdot_out     [m] (dtype): the bins' tangents.
 *   hsdot_aux     nullable [m] adpar_jvp_aux, MUL only (else
 *                 ADPAR_ERR_UNSUPPORTED): ln|tangent| and sign per bin.
 * Workspace: adpar_workspace_size(ADPAR_RULE_JVP_HIST, desc, n, m). */
int adpar_jvp_hist(adpar_opdesc desc, int64_t n, int64_t m, const void *vals, const void *vdot,
                   const void *inds, int itype, void *hs_out, void *hsdot_out, adpar_jvp_aux *hsdot_aux,
                   void *work, size_t work_bytes, void *stream);

/* Forward mode of scatter (Sec. 5.3): ys = scatter xs is vs is linear in
 * (xs, vs), so ysdot = xsdot with ysdot[is_j] = vsdot_j.  ysdot_inout [n]
 * holds xsdot on entry and ysdot on return; vsdot [m]; indices outside
 * [0, n) are skipped; duplicate indices are a caller error.  No workspace. */
int adpar_jvp_scatter(int dtype, int64_t n, int64_t m, const void *is, int itype, const void *vsdot,
                      void *ysdot_inout, void *stream);

/* Forward mode of map with a free array (Sec. 5.4):
 *   xs_j = g(as[is_j, :], ws[j, :])  ->  xsdot_j = dg/da asdot[is_j, :] + dg/dw wsdot[j, :]
 *   GATHER      xsdot_j = asdot[is_j]
 *   SCALE       xsdot_j = asdot[is_j] ws_j + as[is_j] wsdot_j
 *   SQDIST_ROW  xsdot_j = sum_k 2 (ws[j,k] - as[is_j,k]) (wsdot[j,k] - asdot[is_j,k])
 * An index outside [0, na) gives xsdot_j = 0.  Arguments as for
 * adpar_map_acc, plus asdot [na*width] (required), wsdot [nj*width]
 * (nullable: no tangent on ws) and xsdot [nj] (output).  No workspace. */
int adpar_jvp_map_acc(int gfun, int dtype, int64_t nj, int64_t na, int width, const void *as, const void *is,
                      int itype, const void *ws, const void *asdot, const void *wsdot, void *xsdot, void *stream);

/* The primal forward scan ys = scan (.) as (Sec. 5.2's forward sweep), on
 * its own.  It is the baseline of the AD overhead ratio (VJP time / primal
 * time, Sec. 7).  Arguments as for adpar_vjp_scan; ys_a (and ys_b for
 * LINREC) are required outputs.  Workspace: as for adpar_vjp_scan. */
int adpar_scan(adpar_opdesc desc, int64_t n, const void *a, const void *b, void *ys_a,
               void *ys_b, void *work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* reduce_by_index (Sec. 5.1.2)                                        */
/* ------------------------------------------------------------------ */
/* hs = reduce_by_index (.) e inds vals, i.e. the loop
 *   hs = replicate m e;  for i: hs[inds_i] = hs[inds_i] (.) vals_i,
 * with indices outside [0, m) ignored, and its adjoint valsbar given hsbar:
 * the reduce rule of Sec. 5.1.1 per bin with ybar replaced by hsbar[inds_i].
 *   ADD      valsbar_i = hsbar[inds_i] (in range), else 0.
 *   MIN/MAX  per bin the extremum and its LOWEST index; that element gets
 *            hsbar_b, every other element 0.
 *   MUL      per bin (zero count, lowest zero index, scaled product of the
 *            nonzeros); the three cases of Sec. 5.1.1 per element.
 * Out-of-range elements get 0 (overwrite) or keep their value (accumulate).
 * Arguments:
 *   n, m         elements and bins.
 *   vals         [n] values, dtype (may be NULL for ADD without hs_out).
 *   inds         [n] bin indices, itype (adpar_itype).
 *   hsbar        [m] cotangent of hs, dtype.
 *   valsbar      [n] output adjoint, dtype (ln|contribution| with
 *                ADPAR_PROD_LOGDOMAIN, MUL only).
 *   hs_out       nullable [m]: the recomputed histogram (ADD: sums; MIN/MAX:
 *                extremum, +-inf for an empty bin; MUL: product rounded to
 *                dtype).
 *   argidx_out   nullable [m] int64 (MIN/MAX): the lowest index of the
 *                extremum of each bin, -1 for an empty bin.
 *   bin_aux_out  nullable [m] adpar_prod_aux (MUL).
 *   valsbar_sign nullable [n] int8 (MUL with ADPAR_PROD_LOGDOMAIN).
 * Limits: FP32 MIN/MAX keep 32-bit element indices (n <= 2^32).
 * Workspace: adpar_workspace_size(ADPAR_RULE_HIST, desc, n, m). */
int adpar_vjp_hist(adpar_opdesc desc, int64_t n, int64_t m, const void *vals, const void *inds,
                   int itype, const void *hsbar, void *valsbar, void *hs_out, int64_t *argidx_out,
                   adpar_prod_aux *bin_aux_out, int8_t *valsbar_sign, uint32_t flags, void *work,
                   size_t work_bytes, void *stream);

/* reduce_by_index by the GENERAL rule of Sec. 5.1.2, for any operator of
 * this library (ADD, MUL, MIN, MAX, and LINREC, which has no special rule):
 *   hs[k] = e (.) (a, b)_{i_1} (.) (a, b)_{i_2} (.) ...  over the elements
 *           with inds = k in increasing index order (so a bin of the
 *           non-commutative LINREC is the recurrence over its elements in
 *           index order; the paper states the rule for commutative
 *           operators, where the order does not matter),
 *   (abar, bbar)_i (+)= d(l_i (.) (a, b)_i (.) r_i)/d(a, b)_i ^T hsbar[inds_i]
 * with l_i and r_i the combination of the bin's elements before and after
 * i (the neutral element at the bin's ends).  Computed as Sec. 5.1.2
 * proposes: a stable radix sort of the elements by bin (the values travel
 * with the keys), a forward and a reverse segmented single-pass scan over
 * the sorted sequence, and the per-element map.  Indices outside [0, m)
 * are ignored: those elements get 0 (overwrite) or keep their adjoint
 * (ADPAR_ACCUMULATE).  MUL is the product of the bin's other elements
 * (no division, zeros safe, no extended exponent: it may underflow where
 * adpar_vjp_hist's scaled rule would not); MIN/MAX give hsbar to the
 * lowest index of the bin's extremum.
 * Arguments:
 *   desc         op, dtype and width (2 for LINREC, else 1).
 *   n, m         elements and bins; n < 2^32 - 2048 and m <= 2^31
 *                (ADPAR_ERR_UNSUPPORTED beyond).
 *   a, b         [n] element arrays, dtype (b: LINREC only).
 *   inds         [n] bin indices, itype.
 *   hsbar_a/_b   [m] cotangents of hs (the _b one for LINREC).
 *   abar, bbar   [n] output adjoints.
 *   hs_a, hs_b   nullable [m]: the recomputed bins (neutral element for an
 *                empty bin); both or neither for LINREC.
 * No alignment is required of the caller's arrays.
 * Flags: ADPAR_ACCUMULATE.
 * Workspace: adpar_workspace_size(ADPAR_RULE_HIST_GENERAL, desc, n, m):
 * about 2 * (8 + width * sizeof(dtype)) bytes per element (the sort's two
 * buffers) plus the scans' slots. */
int adpar_vjp_hist_general(adpar_opdesc desc, int64_t n, int64_t m, const void *a, const void *b,
                           const void *inds, int itype, const void *hsbar_a, const void *hsbar_b,
                           void *abar, void *bbar, void *hs_a, void *hs_b, uint32_t flags, void *work,
                           size_t work_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* scatter (Sec. 5.3)                                                  */
/* ------------------------------------------------------------------ */
/* ys = scatter xs is vs with `is` free of duplicates (a duplicate is a
 * caller error, not detected).  Return sweep of Sec. 5.3, O(m) work:
 *   vsbar[j] += ysbar[is_j];  ysbar[is_j] = 0 (ysbar becomes xsbar in
 *   place);  with ADPAR_SCATTER_RESTORE also ys[is_j] = xs_saved[j].
 * Indices outside [0, n) are skipped (vsbar_j gets 0, or keeps its value
 * with ADPAR_ACCUMULATE).
 * Arguments: dtype (adpar_dtype); n destination length; m = |is|; is [m]
 * (itype); ysbar_inout [n]; vsbar [m]; ys_restore [n] and xs_saved [m]
 * (only with ADPAR_SCATTER_RESTORE).  No workspace. */
int adpar_vjp_scatter(int dtype, int64_t n, int64_t m, const void *is, int itype, void *ysbar_inout,
                      void *vsbar, void *ys_restore, const void *xs_saved, uint32_t flags, void *stream);

/* ------------------------------------------------------------------ */
/* map with a free array (Sec. 5.4)                                    */
/* ------------------------------------------------------------------ */
/* xs[j] = g(as[is_j, :], ws[j, :]) for j < nj, with as a free array of na
 * rows of `width` values.  Each read of as becomes an accumulation into
 * asbar at the same index (Sec. 5.4's accumulators):
 *   GATHER      (width 1)  asbar[is_j] += xsbar_j
 *   SCALE       (width 1)  asbar[is_j] += ws_j xsbar_j;  wsbar_j = as[is_j] xsbar_j
 *   SQDIST_ROW  (width d)  asbar[is_j,k] += -2 (ws[j,k] - as[is_j,k]) xsbar_j;
 *                          wsbar[j,k] = 2 (ws[j,k] - as[is_j,k]) xsbar_j
 * Indices outside [0, na) are skipped.  asbar starts from zero unless
 * ADPAR_ACCUMULATE; wsbar (nullable) is overwritten or accumulated likewise.
 * Arguments: gfun (adpar_gfun), dtype, nj, na, width; as [na*width]; is
 * [nj] (itype); ws [nj*width] (not for GATHER); xsbar [nj]; asbar
 * [na*width]; wsbar [nj*width].  work/work_bytes: unused (may be NULL). */
int adpar_vjp_map_acc(int gfun, int dtype, int64_t nj, int64_t na, int width, const void *as,
                      const void *is, int itype, const void *ws, const void *xsbar, void *asbar,
                      void *wsbar, uint32_t flags, void *work, size_t work_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* k-means cost and its gradient (Sec. 7.4)                            */
/* ------------------------------------------------------------------ */
/* loss = sum_i min_k ||x_i - c_k||^2 over N points x_i (rows of X, d = 32
 * FP32) and k centroids (rows of C), and its VJP in C:
 *   Cbar[k] = 2 ybar (cnt_k c_k - sum_{i: argmin_i = k} x_i),
 * the min-reduce rule of Sec. 5.1.1 followed by the accumulator of
 * Sec. 5.4 on the free array C.  Distances come from a TF32 tensor-core
 * GEMM X C^T; the argmin is certified (every centroid within the TF32 error
 * bound of the minimum is recomputed exactly, FP64 breaking what FP32
 * cannot), so it equals the FP64 argmin with the lowest k on ties, and the
 * loss sums the exactly recomputed distances.
 * Arguments:
 *   N, d, k      points, dimension (32) and centroids (multiple of 32, <= 256).
 *   X [N*32], C [k*32]   row-major FP32 inputs.
 *   ybar         device FP32 scalar, required when Cbar is given.
 *   loss_out     nullable device FP32 scalar.
 *   argmin_out   nullable device int32 [N].
 *   Cbar         nullable [k*32] FP32: the gradient (forward only if NULL).
 * Flags: ADPAR_ACCUMULATE (Cbar += ...).
 * Workspace: adpar_workspace_size(ADPAR_RULE_KMEANS, desc, N, k). */
int adpar_kmeans_vjp(int64_t N, int d, int k, const float *X, const float *C, const float *ybar,
                     float *loss_out, int32_t *argmin_out, float *Cbar, uint32_t flags, void *work,
                     size_t work_bytes, void *stream);

/* Hessian diagonal of the same cost in C, the second-order information of
 * Sec. 7.4, in closed form from the counts (adpar_kmeans_fwd_rev below
 * obtains it by forward mode nested over the VJP): with every point's
 * argmin held fixed (the cost is piecewise quadratic in C),
 *   Hdiag[k][j] = d^2 loss / dc_kj^2 = 2 ybar cnt_k,
 * cnt_k the number of points whose argmin is k.  It reads the counts that
 * the preceding adpar_kmeans_vjp call (Cbar requested) left in its
 * workspace: call it on the same stream with the same workspace, before
 * the workspace is reused.
 * Arguments: k (as for adpar_kmeans_vjp); ybar device FP32 scalar; work,
 * work_bytes that call's workspace; Hdiag [k*32] FP32 output.
 * Flags: ADPAR_ACCUMULATE (Hdiag += ...). */
int adpar_kmeans_hessdiag(int k, const float *ybar, const void *work, size_t work_bytes, float *Hdiag,
                          uint32_t flags, void *stream);

/* Forward over reverse for the same cost (Sec. 7.4 nests forward mode over
 * the VJP): the reverse sweep of adpar_kmeans_vjp run on dual numbers along
 * a tangent Cdot of the centroids.  With k*_i the certified argmin of point
 * i (recomputed by adpar_kmeans_vjp's forward part; it has no tangent):
 *   ydot     = sum_i sum_j 2 (c_{k*_i j} - x_ij) cdot_{k*_i j}   (loss tangent)
 *   Cbardot[k] = sum_{i: k*_i = k} ybar (-2)(0 - cdot_k) = 2 ybar cnt_k cdot_k,
 * the tangent of the gradient Cbar, i.e. the Hessian-vector product H Cdot.
 * The cost's Hessian in C is diagonal (2 ybar cnt_k on centroid k's
 * coordinates), so Cdot = 1 gives the Hessian diagonal.
 * Arguments: N, d, k, X, C as for adpar_kmeans_vjp; Cdot [k*32] FP32;
 * ybar device FP32 scalar; ydot_out nullable device FP32 scalar; Cbardot
 * [k*32] FP32 output.  Flags: ADPAR_ACCUMULATE (Cbardot += ...).
 * Workspace: adpar_workspace_size(ADPAR_RULE_KMEANS_FWD_REV, desc, N, k). */
int adpar_kmeans_fwd_rev(int64_t N, int d, int k, const float *X, const float *C, const float *Cdot,
                         const float *ybar, float *ydot_out, float *Cbardot, uint32_t flags, void *work,
                         size_t work_bytes, void *stream);

/* ------------------------------------------------------------------ */
/* batched VJPs: many instances in one persistent launch               */
/* ------------------------------------------------------------------ */
/* Not in the paper (a serving form of its rules).  Each segment is an
 * independent instance of: the product-reduce VJP of Sec. 5.1.1 over x
 * (cotangent ybar_prod), and the linear-recurrence scan VJP of Sec. 5.2
 * over (a, b) with cotangents (ybar_a, ybar_b).  All pointers are device
 * pointers of the segment's dtype; outputs are overwritten. */
typedef struct {
    const void *x;        /* [len] product-reduce input               */
    void *xbar;           /* [len] its adjoint                        */
    const void *a;        /* [len] linear-recurrence inputs           */
    const void *b;
    const void *ybar_a;   /* [len] cotangents of the scan outputs     */
    const void *ybar_b;
    void *abar;           /* [len] adjoints of a and b                */
    void *bbar;
    adpar_prod_aux *aux;  /* nullable: the recomputed product sweep   */
    double ybar_prod;     /* cotangent of the product                 */
    int64_t len;
    int32_t dtype;        /* ADPAR_F32 or ADPAR_F64                   */
    int32_t reserved;
} adpar_batch_segment;

/* Launch shape chosen by the autotuner: variant = compiled tile shapes
 * (0: 2048-element scan tiles, 8192-element product tiles; 1: 4096 /
 * 16384; 2: 1024 / 4096), ctas_per_sm = persistent blocks per SM (1..8),
 * order = 0 (as given) or 1 (longest segments first). */
typedef struct {
    int32_t variant;
    int32_t ctas_per_sm;
    int32_t order;
    int32_t reserved;
} adpar_batch_config;

/* Bytes of the plan image for nseg segments. */
size_t adpar_batch_plan_bytes(int nseg);

/* Host-side planning: writes the plan image (segments in scheduling order,
 * work-item numbering, per-segment state offsets) into plan_host (host
 * memory, adpar_batch_plan_bytes(nseg) bytes) and the workspace size the
 * launch needs into *work_bytes_out.  segs is host memory; cfg may be NULL
 * (variant 0, 2 blocks per SM, longest first).  The caller copies the plan
 * image to device memory once and keeps it (and every segment buffer)
 * alive while the batch may run. */
int adpar_batch_plan(const adpar_batch_segment *segs, int nseg, const adpar_batch_config *cfg,
                     void *plan_host, size_t plan_bytes, size_t *work_bytes_out);

/* One launch of the batch: a zero-fill of the workspace state and one
 * persistent kernel.  plan_host and plan_dev are the same image (host copy
 * for the launch shape, device copy for the kernel).  Only kernel launches
 * are enqueued, so the call can be captured in a CUDA graph and replayed. */
int adpar_vjp_batch(const void *plan_host, const void *plan_dev, void *work, size_t work_bytes,
                    void *stream);

/* ------------------------------------------------------------------ */
/* primal forward operators                                            */
/* ------------------------------------------------------------------ */
/* The forward operators on their own: the forward sweeps of Sec. 5 without
 * any adjoint.  They serve the autograd forward pass and are the baseline
 * of the AD overhead ratio (VJP time / primal time, Sec. 7).  Arguments,
 * layouts and workspaces are those of the matching VJP entry point. */

/* y = reduce (.) a; argidx_out (MIN/MAX) and aux_out (MUL) as for
 * adpar_vjp_reduce.  y_out is required. */
int adpar_reduce(adpar_opdesc desc, int64_t n, const void *a, void *y_out, int64_t *argidx_out,
                 adpar_prod_aux *aux_out, void *work, size_t work_bytes, void *stream);

/* hs = reduce_by_index (.) inds vals into hs_out [m] (required);
 * argidx_out and bin_aux_out as for adpar_vjp_hist. */
int adpar_hist(adpar_opdesc desc, int64_t n, int64_t m, const void *vals, const void *inds, int itype,
               void *hs_out, int64_t *argidx_out, adpar_prod_aux *bin_aux_out, void *work,
               size_t work_bytes, void *stream);

/* ys = scatter ys is vs in place (ys_inout [n] holds xs on entry), saving
 * the overwritten values xs_saved_out[j] = xs[is_j] first (nullable), the
 * forward sweep of Sec. 5.3.  Out-of-range indices are skipped. */
int adpar_scatter(int dtype, int64_t n, int64_t m, const void *is, int itype, const void *vs,
                  void *ys_inout, void *xs_saved_out, void *stream);

/* xs[j] = g(as[is_j, :], ws[j, :]) (0 for an index out of range). */
int adpar_map_acc(int gfun, int dtype, int64_t nj, int64_t na, int width, const void *as, const void *is,
                  int itype, const void *ws, void *xs_out, void *stream);

/* ------------------------------------------------------------------ */
/* scan VJP without any allocation                                     */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart of this entry point; it serves callers
 * that cannot allocate device memory when they need the gradient (code
 * inside an allocator or memory-manager hook that must not re-enter it,
 * loops that forbid allocation after start-up, hosts that hand over fixed
 * buffers only).  It computes exactly what adpar_vjp_scan computes, with
 * the same arguments minus (work, work_bytes): its scratch is one static
 * device array of adpar_noalloc_scratch_bytes() bytes (8 MiB), which every
 * GPU that loads the library holds until the process exits.  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   - Sizes whose scan workspace exceeds the array are refused with
 *     ADPAR_ERR_TOO_LARGE before anything is enqueued (up to 2^28 FP32
 *     elements of a width-1 operator and 2^26 FP64 LINREC pairs fit).
 *   - Every call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress).  The first lookup on a device also loads the
 *     library's module there; make that first call before any stream
 *     capture on the device.
 *   - All calls on one device share the array.  Each call clears the parts
 *     that must start at zero, but two calls that overlap on the GPU (on
 *     different streams, or from different threads) race on it and give
 *     wrong results: serialise them.
 *   - A device-side wait that gives up records ADPAR_ERR_TIMEOUT in the
 *     array's status word while the call itself has returned ADPAR_OK; read
 *     it with adpar_noalloc_status after the call.  The next call clears it. */
int adpar_vjp_scan_noalloc(adpar_opdesc desc, int64_t n, const void *a, const void *b,
                           const void *ybar_a, const void *ybar_b, void *abar, void *bbar,
                           void *ys_a, void *ys_b, uint32_t flags, void *stream);

/* Size in bytes of the static scratch array of adpar_vjp_scan_noalloc. */
size_t adpar_noalloc_scratch_bytes(void);

/* Device status of the last adpar_vjp_scan_noalloc call on the current
 * device, as adpar_workspace_status gives it for a caller workspace: waits
 * for `stream` (cudaStreamSynchronize), then copies the status word out of
 * the static array into *device_status (ADPAR_OK, or ADPAR_ERR_TIMEOUT when
 * a bounded wait gave up and the adjoints are wrong).  Allocates nothing.
 * Returns ADPAR_ERR_INVALID for a null device_status, ADPAR_ERR_CUDA when
 * the synchronisation or the copy fails. */
int adpar_noalloc_status(void *stream, int *device_status);

/* Failure-detection self-test on the static array: the same bounded wait on
 * a flag that nothing sets as adpar_selftest_timeout, run in the static
 * array instead of a caller workspace, so that adpar_noalloc_status then
 * reports ADPAR_ERR_TIMEOUT.  Takes about a second on the GPU; the GPU
 * context stays usable.  Allocates nothing. */
int adpar_noalloc_selftest_timeout(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ADPAR_H */
