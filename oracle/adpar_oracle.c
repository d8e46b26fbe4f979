/*
 * adpar oracle: a plain, slow, single-threaded FP64 statement of the
 * reverse-mode (VJP) rules for bulk-parallel operators of
 * "AD for an Array Language with Nested Parallelism" (arXiv 2202.10297).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant with the
 * CUDA library; the two meet only at the seeded synthetic inputs.
 *
 * Every rule here is the plain definition of the gradient, obtained the
 * way Sec. 2 (Eq. rewrite-adj) obtains it for a straight-line program: the
 * primal is run as a sequential loop that records a tape of every value
 * that feeds an operator, and the adjoint is the reverse sweep over that
 * tape, adding dF/d(input) * adjoint(output) into each input's adjoint.
 * No case analysis of the parallel rules (zero counting, argmin, lin_o
 * scans, privatisation) is used, so agreement with the CUDA path checks
 * that analysis independently.
 *
 * Products (reduce and reduce_by_index with *) leave the FP64 exponent
 * range on realistic sizes, so their sweeps run in an extended-exponent
 * number "xd" = m * 2^e with m in [0.5,1) (or 0) and a 64-bit e.  Every
 * multiplication of two xd values rounds once, exactly as an FP64 multiply
 * would, so the xd sweep is the FP64 sweep without overflow/underflow.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* operator codes of this file (deliberately not shared with the library) */
enum { O_ADD = 0, O_MUL = 1, O_MIN = 2, O_MAX = 3, O_LINREC = 4 };
/* map_acc functions g */
enum { G_GATHER = 0, G_SCALE = 1, G_SQDIST_ROW = 2 };

/* ---------------------------------------------------------------------
 * Extended-exponent FP64 numbers.
 * ------------------------------------------------------------------- */
typedef struct { double m; int64_t e; } xd;

static xd xd_make(double v)
{
    xd r;
    int e = 0;
    r.m = frexp(v, &e);
    r.e = (r.m == 0.0) ? 0 : (int64_t)e;
    return r;
}

static xd xd_mul(xd a, xd b)
{
    xd r;
    int e = 0;
    if (a.m == 0.0 || b.m == 0.0) { r.m = 0.0; r.e = 0; return r; }
    r.m = frexp(a.m * b.m, &e);
    r.e = a.e + b.e + e;
    return r;
}

/* value rounded to FP64 (0 or subnormal when the exponent is very small) */
static double xd_value(xd a)
{
    if (a.m == 0.0) return 0.0;
    if (a.e > 2000) return copysign(INFINITY, a.m);
    if (a.e < -2000) return copysign(0.0, a.m);
    return ldexp(a.m, (int)a.e);
}

/* natural log of |a| (-inf for 0) */
static double xd_log(xd a)
{
    if (a.m == 0.0) return -INFINITY;
    return log(fabs(a.m)) + (double)a.e * 0.69314718055994530942;
}

static int xd_sign(xd a) { return (a.m > 0.0) - (a.m < 0.0); }

/* ---------------------------------------------------------------------
 * Reduce with +, min, max (Sec. 5.1).  The primal is the loop
 *   t_0 = e;  t_{i+1} = t_i (.) a_i;  y = t_n
 * and its reverse sweep, starting from g = ybar, is
 *   abar_i += d(t_i (.) a_i)/d a_i * g;   g = d(t_i (.) a_i)/d t_i * g.
 * For max the derivative of max(t,a) goes to t on ties (t >= a), i.e. to
 * the earlier element, which is the "(first) index" of Sec. 5.1.1.
 * argidx_out receives the index whose adjoint the sweep touched with a
 * unit chain factor (min/max only; -1 when n == 0).
 * ------------------------------------------------------------------- */
static double neutral_of(int op)
{
    switch (op) {
    case O_ADD: return 0.0;
    case O_MUL: return 1.0;
    case O_MIN: return INFINITY;
    case O_MAX: return -INFINITY;
    }
    return 0.0;
}

static double combine(int op, double t, double a)
{
    switch (op) {
    case O_ADD: return t + a;
    case O_MUL: return t * a;
    case O_MIN: return (a < t) ? a : t;
    case O_MAX: return (a > t) ? a : t;
    }
    return 0.0;
}

/* partial derivatives of t (.) a with respect to a and to t */
static double d_da(int op, double t, double a)
{
    switch (op) {
    case O_ADD: return 1.0;
    case O_MUL: return t;
    case O_MIN: return (a < t) ? 1.0 : 0.0;
    case O_MAX: return (a > t) ? 1.0 : 0.0;
    }
    return 0.0;
}

static double d_dt(int op, double t, double a)
{
    switch (op) {
    case O_ADD: return 1.0;
    case O_MUL: return a;
    case O_MIN: return (t <= a) ? 1.0 : 0.0;
    case O_MAX: return (t >= a) ? 1.0 : 0.0;
    }
    return 0.0;
}

int oracle_reduce_vjp(int op, int64_t n, const double *a, double ybar,
                      double *y_out, double *abar, int64_t *argidx_out)
{
    if (op != O_ADD && op != O_MIN && op != O_MAX && op != O_MUL) return 1;
    double *t = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    if (!t) return 2;
    t[0] = neutral_of(op);
    for (int64_t i = 0; i < n; ++i) t[i + 1] = combine(op, t[i], a[i]);
    if (y_out) *y_out = t[n];

    double g = ybar;
    double chain = 1.0; /* product of d/dt factors, without ybar */
    int64_t arg = -1;
    for (int64_t i = n - 1; i >= 0; --i) {
        double fa = d_da(op, t[i], a[i]);
        double ft = d_dt(op, t[i], a[i]);
        abar[i] += fa * g;
        if (arg < 0 && chain != 0.0 && fa != 0.0 && (op == O_MIN || op == O_MAX))
            arg = i;
        g = ft * g;
        chain = ft * chain;
    }
    if (argidx_out) *argidx_out = arg;
    free(t);
    return 0;
}

/* ---------------------------------------------------------------------
 * Reduce with * (Sec. 5.1.1) in extended-exponent FP64.  Same tape sweep
 * as above (abar_i += t_i * g; g = a_i * g), which needs no division and
 * no case analysis of the zeros.  Outputs per element:
 *   abar_val[i]  += the contribution rounded to FP64,
 *   abar_log[i]   = ln|contribution| (-inf when it is zero),
 *   abar_sign[i]  = sign of the contribution (-1, 0, +1).
 * aux receives, by a separate plain loop over the definition:
 *   aux_i[0] = number of zeros, aux_i[1] = lowest zero index (-1 if none),
 *   aux_d[0] = ln|product of the nonzero elements|, aux_d[1] = its sign,
 *   aux_d[2] = y = the full product rounded to FP64.
 * ------------------------------------------------------------------- */
int oracle_prod_reduce_vjp(int64_t n, const double *a, double ybar,
                           double *abar_val, double *abar_log, int8_t *abar_sign,
                           int64_t *aux_i, double *aux_d)
{
    xd *t = (xd *)malloc(sizeof(xd) * (size_t)(n + 1));
    if (!t) return 2;
    t[0] = xd_make(1.0);
    for (int64_t i = 0; i < n; ++i) t[i + 1] = xd_mul(t[i], xd_make(a[i]));

    xd g = xd_make(ybar);
    for (int64_t i = n - 1; i >= 0; --i) {
        xd c = xd_mul(t[i], g);
        if (abar_val) abar_val[i] += xd_value(c);
        if (abar_log) abar_log[i] = xd_log(c);
        if (abar_sign) abar_sign[i] = (int8_t)xd_sign(c);
        g = xd_mul(xd_make(a[i]), g);
    }

    int64_t nz = 0, first = -1;
    xd p = xd_make(1.0);
    for (int64_t i = 0; i < n; ++i) {
        if (a[i] == 0.0) {
            if (first < 0) first = i;
            ++nz;
        } else {
            p = xd_mul(p, xd_make(a[i]));
        }
    }
    if (aux_i) { aux_i[0] = nz; aux_i[1] = first; }
    if (aux_d) {
        aux_d[0] = xd_log(p);
        aux_d[1] = (double)xd_sign(p);
        aux_d[2] = xd_value(t[n]);
    }
    free(t);
    return 0;
}

/* ---------------------------------------------------------------------
 * Inclusive scan (Sec. 5.2).  The primal is the loop
 *   rs_0 = as_0;  rs_i = rs_{i-1} (.) as_i
 * and its reverse sweep is the unrolled loop of Sec. 5.2 before the loop
 * distribution: starting from rsbar = ysbar,
 *   for i = n-1 .. 1:
 *     rsbar_{i-1} += J_left(i)^T  rsbar_i,
 *     asbar_i     += J_right(i)^T rsbar_i,
 *   asbar_0 += rsbar_0,
 * with J_left(i) = d(rs_{i-1} (.) as_i)/d rs_{i-1} and
 *      J_right(i) = d(rs_{i-1} (.) as_i)/d as_i.
 * Elements are vectors of width w (1, or 2 for LINREC) and the Jacobians
 * are full w x w matrices, applied transposed.
 *
 * LINREC: (a1,b1) (.) (a2,b2) = (a2*a1, a2*b1 + b2).  With rs = (A,B),
 *   J_left  = [[a_i, 0], [0, a_i]],
 *   J_right = [[A_{i-1}, 0], [B_{i-1}, 1]]   (rows: A,B; columns: a,b).
 * ------------------------------------------------------------------- */
typedef struct { double v[2][2]; } mat2;

/* y = M^T x  (x, y of width w) */
static void mat_t_vec(const mat2 *M, const double *x, double *y, int w)
{
    for (int c = 0; c < w; ++c) {
        double s = 0.0;
        for (int r = 0; r < w; ++r) s += M->v[r][c] * x[r];
        y[c] = s;
    }
}

static void scan_combine(int op, const double *l, const double *r, double *out)
{
    if (op == O_LINREC) {
        double A = r[0] * l[0];
        double B = r[0] * l[1] + r[1];
        out[0] = A;
        out[1] = B;
    } else {
        out[0] = combine(op, l[0], r[0]);
    }
}

static void scan_jacobians(int op, const double *prev, const double *x,
                           mat2 *Jl, mat2 *Jr)
{
    memset(Jl, 0, sizeof(*Jl));
    memset(Jr, 0, sizeof(*Jr));
    if (op == O_LINREC) {
        Jl->v[0][0] = x[0];
        Jl->v[1][1] = x[0];
        Jr->v[0][0] = prev[0];
        Jr->v[1][0] = prev[1];
        Jr->v[1][1] = 1.0;
    } else {
        Jl->v[0][0] = d_dt(op, prev[0], x[0]);
        Jr->v[0][0] = d_da(op, prev[0], x[0]);
    }
}

/* as: w arrays of n (as0 = a, as1 = b for LINREC); ysbar likewise;
 * asbar are accumulated; ys_out (nullable) receive the primal. */
int oracle_scan_vjp(int op, int64_t n,
                    const double *as0, const double *as1,
                    const double *ysbar0, const double *ysbar1,
                    double *asbar0, double *asbar1,
                    double *ys0, double *ys1)
{
    int w = (op == O_LINREC) ? 2 : 1;
    if (op < O_ADD || op > O_LINREC) return 1;
    if (n == 0) return 0;
    double *rs = (double *)malloc(sizeof(double) * (size_t)n * (size_t)w);
    double *rsbar = (double *)calloc((size_t)n * (size_t)w, sizeof(double));
    if (!rs || !rsbar) { free(rs); free(rsbar); return 2; }
    const double *as[2] = { as0, as1 };
    const double *ysb[2] = { ysbar0, ysbar1 };
    double *asb[2] = { asbar0, asbar1 };

    for (int c = 0; c < w; ++c) rs[c] = as[c][0];
    for (int64_t i = 1; i < n; ++i) {
        double x[2], out[2];
        for (int c = 0; c < w; ++c) x[c] = as[c][i];
        scan_combine(op, &rs[(i - 1) * w], x, out);
        for (int c = 0; c < w; ++c) rs[i * w + c] = out[c];
    }
    if (ys0) for (int64_t i = 0; i < n; ++i) ys0[i] = rs[i * w];
    if (ys1 && w == 2) for (int64_t i = 0; i < n; ++i) ys1[i] = rs[i * w + 1];

    for (int64_t i = 0; i < n; ++i)
        for (int c = 0; c < w; ++c) rsbar[i * w + c] = ysb[c][i];

    for (int64_t i = n - 1; i >= 1; --i) {
        double x[2], dl[2], dr[2];
        mat2 Jl, Jr;
        for (int c = 0; c < w; ++c) x[c] = as[c][i];
        scan_jacobians(op, &rs[(i - 1) * w], x, &Jl, &Jr);
        mat_t_vec(&Jl, &rsbar[i * w], dl, w);
        mat_t_vec(&Jr, &rsbar[i * w], dr, w);
        for (int c = 0; c < w; ++c) {
            rsbar[(i - 1) * w + c] += dl[c];
            asb[c][i] += dr[c];
        }
    }
    for (int c = 0; c < w; ++c) asb[c][0] += rsbar[c];
    free(rs);
    free(rsbar);
    return 0;
}

/* ---------------------------------------------------------------------
 * Forward mode (JVP) of the inclusive scan: the primal loop carried with
 * dual numbers, rs_i = rs_{i-1} (.) as_i and
 *   rsdot_i = J_left(i) rsdot_{i-1} + J_right(i) asdot_i,
 * with the same per-operator Jacobians as the reverse sweep above (applied
 * forward, not transposed) and rs_0 = as_0, rsdot_0 = asdot_0.
 * ------------------------------------------------------------------- */
static void mat_vec(const mat2 *M, const double *x, double *y, int w)
{
    for (int i = 0; i < w; ++i) {
        double s = 0.0;
        for (int j = 0; j < w; ++j) s += M->v[i][j] * x[j];
        y[i] = s;
    }
}

int oracle_scan_jvp(int op, int64_t n,
                    const double *as0, const double *as1,
                    const double *ad0, const double *ad1,
                    double *ys0, double *ys1, double *yd0, double *yd1)
{
    if (op < O_ADD || op > O_LINREC) return 1;
    int w = (op == O_LINREC) ? 2 : 1;
    if (n == 0) return 0;
    const double *as[2] = { as0, as1 };
    const double *ad[2] = { ad0, ad1 };
    double *ys[2] = { ys0, ys1 };
    double *yd[2] = { yd0, yd1 };
    double rs[2], rd[2];
    for (int c = 0; c < w; ++c) { rs[c] = as[c][0]; rd[c] = ad[c][0]; }
    for (int c = 0; c < w; ++c) { ys[c][0] = rs[c]; yd[c][0] = rd[c]; }
    for (int64_t i = 1; i < n; ++i) {
        double x[2], xd[2], out[2], t1[2], t2[2];
        mat2 Jl, Jr;
        for (int c = 0; c < w; ++c) { x[c] = as[c][i]; xd[c] = ad[c][i]; }
        scan_jacobians(op, rs, x, &Jl, &Jr);
        mat_vec(&Jl, rd, t1, w);
        mat_vec(&Jr, xd, t2, w);
        scan_combine(op, rs, x, out);
        for (int c = 0; c < w; ++c) {
            rs[c] = out[c];
            rd[c] = t1[c] + t2[c];
            ys[c][i] = rs[c];
            yd[c][i] = rd[c];
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------
 * Reduce with an arbitrary associative operator (Sec. 5.1.1, the general
 * rule), any width: y = e (.) a_0 (.) ... (.) a_{n-1}.  Plain tape sweep:
 * the forward loop records t_i = e (.) a_0 (.) ... (.) a_{i-1}; the reverse
 * loop keeps g = adjoint of t_{i+1} (starting at ybar) and does
 *   asbar_i += J_right(t_i, a_i)^T g;   g = J_left(t_i, a_i)^T g
 * with the same per-operator Jacobians as the scan sweep above.  The rule
 * the library implements (l_i and r_i from two exclusive scans, then
 * d(l_i (.) a_i (.) r_i)/d a_i) is not used here.
 * ------------------------------------------------------------------- */
int oracle_reduce_general_vjp(int op, int64_t n,
                              const double *as0, const double *as1,
                              double ybar0, double ybar1,
                              double *asbar0, double *asbar1,
                              double *y_out)
{
    if (op < O_ADD || op > O_LINREC) return 1;
    int w = (op == O_LINREC) ? 2 : 1;
    double *t = (double *)malloc(sizeof(double) * (size_t)(n + 1) * (size_t)w);
    if (!t) return 2;
    const double *as[2] = { as0, as1 };
    double *asb[2] = { asbar0, asbar1 };
    /* the neutral element */
    if (op == O_LINREC) { t[0] = 1.0; t[1] = 0.0; }
    else t[0] = neutral_of(op);
    for (int64_t i = 0; i < n; ++i) {
        double x[2];
        for (int c = 0; c < w; ++c) x[c] = as[c][i];
        scan_combine(op, &t[i * w], x, &t[(i + 1) * w]);
    }
    if (y_out) for (int c = 0; c < w; ++c) y_out[c] = t[n * w + c];
    double g[2] = { ybar0, ybar1 };
    for (int64_t i = n - 1; i >= 0; --i) {
        double x[2], dl[2], dr[2];
        mat2 Jl, Jr;
        for (int c = 0; c < w; ++c) x[c] = as[c][i];
        scan_jacobians(op, &t[i * w], x, &Jl, &Jr);
        mat_t_vec(&Jr, g, dr, w);
        mat_t_vec(&Jl, g, dl, w);
        for (int c = 0; c < w; ++c) {
            asb[c][i] += dr[c];
            g[c] = dl[c];
        }
    }
    free(t);
    return 0;
}

/* ---------------------------------------------------------------------
 * reduce_by_index with +, min, max (Sec. 5.1.2).  The primal is the
 * semantic loop
 *   hs = replicate m e;  for i: hs[inds[i]] = hs[inds[i]] (.) vals[i]
 * with a tape t_i of the bin's running value before element i.  Indices
 * outside [0, m) are skipped (their element does not take part).  The
 * reverse sweep keeps one adjoint g[b] per bin, starting at hsbar[b]:
 *   for i = n-1..0 (b = inds[i] in range):
 *     valsbar_i += d(t_i (.) v_i)/dv_i * g[b];  g[b] = d(...)/dt_i * g[b].
 * argidx_out[b] = the element that received bin b's adjoint with a unit
 * chain factor (min/max only; -1 for an empty bin).
 * ------------------------------------------------------------------- */
int oracle_hist_vjp(int op, int64_t n, int64_t m, const double *vals,
                    const int64_t *inds, const double *hsbar,
                    double *valsbar, double *hs_out, int64_t *argidx_out)
{
    if (op != O_ADD && op != O_MIN && op != O_MAX) return 1;
    double *hs = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *t = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *g = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *chain = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!hs || !t || !g || !chain) { free(hs); free(t); free(g); free(chain); return 2; }
    for (int64_t b = 0; b < m; ++b) hs[b] = neutral_of(op);
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) continue;
        t[i] = hs[b];
        hs[b] = combine(op, hs[b], vals[i]);
    }
    if (hs_out) for (int64_t b = 0; b < m; ++b) hs_out[b] = hs[b];
    for (int64_t b = 0; b < m; ++b) {
        g[b] = hsbar ? hsbar[b] : 0.0;
        chain[b] = 1.0;
        if (argidx_out) argidx_out[b] = -1;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) continue;
        double fa = d_da(op, t[i], vals[i]);
        double ft = d_dt(op, t[i], vals[i]);
        valsbar[i] += fa * g[b];
        if (argidx_out && argidx_out[b] < 0 && chain[b] != 0.0 && fa != 0.0 &&
            (op == O_MIN || op == O_MAX))
            argidx_out[b] = i;
        g[b] = ft * g[b];
        chain[b] = ft * chain[b];
    }
    free(hs); free(t); free(g); free(chain);
    return 0;
}

/* reduce_by_index with * in extended-exponent FP64: the same tape sweep
 * (valsbar_i += t_i * g[b]; g[b] = vals_i * g[b]).  Per element outputs as
 * for oracle_prod_reduce_vjp; per bin (m entries each):
 *   bin_nzero[b], bin_first_zero[b] (-1 if none),
 *   bin_lognz[b] = ln|product of nonzeros|, bin_signnz[b] = its sign. */
int oracle_hist_prod_vjp(int64_t n, int64_t m, const double *vals,
                         const int64_t *inds, const double *hsbar,
                         double *valsbar_val, double *valsbar_log, int8_t *valsbar_sign,
                         int64_t *bin_nzero, int64_t *bin_first_zero,
                         double *bin_lognz, double *bin_signnz)
{
    xd *hs = (xd *)malloc(sizeof(xd) * (size_t)(m > 0 ? m : 1));
    xd *t = (xd *)malloc(sizeof(xd) * (size_t)(n > 0 ? n : 1));
    xd *g = (xd *)malloc(sizeof(xd) * (size_t)(m > 0 ? m : 1));
    xd *pnz = (xd *)malloc(sizeof(xd) * (size_t)(m > 0 ? m : 1));
    if (!hs || !t || !g || !pnz) { free(hs); free(t); free(g); free(pnz); return 2; }
    for (int64_t b = 0; b < m; ++b) hs[b] = xd_make(1.0);
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) continue;
        t[i] = hs[b];
        hs[b] = xd_mul(hs[b], xd_make(vals[i]));
    }
    for (int64_t b = 0; b < m; ++b) g[b] = xd_make(hsbar[b]);
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) {
            if (valsbar_log) valsbar_log[i] = -INFINITY;
            if (valsbar_sign) valsbar_sign[i] = 0;
            continue;
        }
        xd c = xd_mul(t[i], g[b]);
        if (valsbar_val) valsbar_val[i] += xd_value(c);
        if (valsbar_log) valsbar_log[i] = xd_log(c);
        if (valsbar_sign) valsbar_sign[i] = (int8_t)xd_sign(c);
        g[b] = xd_mul(xd_make(vals[i]), g[b]);
    }
    for (int64_t b = 0; b < m; ++b) {
        pnz[b] = xd_make(1.0);
        if (bin_nzero) bin_nzero[b] = 0;
        if (bin_first_zero) bin_first_zero[b] = -1;
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) continue;
        if (vals[i] == 0.0) {
            if (bin_nzero) bin_nzero[b] += 1;
            if (bin_first_zero && bin_first_zero[b] < 0) bin_first_zero[b] = i;
        } else {
            pnz[b] = xd_mul(pnz[b], xd_make(vals[i]));
        }
    }
    for (int64_t b = 0; b < m; ++b) {
        if (bin_lognz) bin_lognz[b] = xd_log(pnz[b]);
        if (bin_signnz) bin_signnz[b] = (double)xd_sign(pnz[b]);
    }
    free(hs); free(t); free(g); free(pnz);
    return 0;
}

/* ---------------------------------------------------------------------
 * Scatter (Sec. 5.3): ys = scatter xs is vs, with is free of duplicates.
 * Return sweep, in the order the section gives it:
 *   vsbar[j] += ysbar[is[j]]           (gather)
 *   xsbar     = ysbar with ysbar[is[j]] = 0   (done in place)
 *   optionally ys[is[j]] = xs_saved[j] (restore xs)
 * Indices outside [0, n) are skipped.
 * ------------------------------------------------------------------- */
int oracle_scatter_vjp(int64_t n, int64_t m, const int64_t *is,
                       double *ysbar_inout, double *vsbar,
                       double *ys_restore, const double *xs_saved)
{
    for (int64_t j = 0; j < m; ++j) {
        int64_t k = is[j];
        if (k < 0 || k >= n) continue;
        vsbar[j] += ysbar_inout[k];
    }
    for (int64_t j = 0; j < m; ++j) {
        int64_t k = is[j];
        if (k < 0 || k >= n) continue;
        ysbar_inout[k] = 0.0;
    }
    if (ys_restore && xs_saved) {
        for (int64_t j = 0; j < m; ++j) {
            int64_t k = is[j];
            if (k < 0 || k >= n) continue;
            ys_restore[k] = xs_saved[j];
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------
 * map with a free array variable (Sec. 5.4): xs[j] = g(as[is[j], :], ws[j, :])
 * Every read of the free array as becomes an accumulation into asbar at
 * the same index (the accumulator of Sec. 5.4), and ws is an ordinary
 * mapped input:
 *   GATHER      (width 1): x = a            asbar[i] += xbar
 *   SCALE       (width 1): x = a * w        asbar[i] += w * xbar, wsbar[j] += a * xbar
 *   SQDIST_ROW  (width d): x = sum_k (w_k - a_k)^2
 *               asbar[i,k] += -2 (w_k - a_k) xbar, wsbar[j,k] += 2 (w_k - a_k) xbar
 * Indices outside [0, na) are skipped.  asbar and wsbar are accumulated.
 * ------------------------------------------------------------------- */
int oracle_map_acc_vjp(int gfun, int64_t nj, int64_t na, int width,
                       const double *as, const int64_t *is, const double *ws,
                       const double *xsbar, double *asbar, double *wsbar)
{
    for (int64_t j = 0; j < nj; ++j) {
        int64_t i = is[j];
        if (i < 0 || i >= na) continue;
        double xb = xsbar[j];
        if (gfun == G_GATHER) {
            asbar[i] += xb;
        } else if (gfun == G_SCALE) {
            asbar[i] += ws[j] * xb;
            if (wsbar) wsbar[j] += as[i] * xb;
        } else if (gfun == G_SQDIST_ROW) {
            for (int k = 0; k < width; ++k) {
                double diff = ws[j * width + k] - as[i * width + k];
                asbar[i * width + k] += -2.0 * diff * xb;
                if (wsbar) wsbar[j * width + k] += 2.0 * diff * xb;
            }
        } else {
            return 1;
        }
    }
    return 0;
}

/* ---------------------------------------------------------------------
 * k-means cost (Sec. 7.4, with the squared distance):
 *   loss = sum_i min_k sum_j (x_ij - c_kj)^2.
 * Forward: all distances in FP64, argmin with the lowest k on ties
 * (the min-reduce rule of Sec. 5.1.1).  Reverse: the min-reduce adjoint
 * goes to the argmin only, and the map body's read of the free array C
 * accumulates into Cbar (Sec. 5.4):
 *   Cbar[k*, j] += ybar * d/dc (x_ij - c_j)^2 = ybar * (-2) (x_ij - c_k*j).
 * ------------------------------------------------------------------- */
int oracle_kmeans(int64_t N, int d, int k, const double *X, const double *C,
                  double ybar, double *loss_out, int64_t *argmin_out,
                  double *mind_out, double *Cbar)
{
    double loss = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double best = INFINITY;
        int64_t arg = -1;
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) {
                double diff = X[i * d + j] - C[(int64_t)c * d + j];
                s += diff * diff;
            }
            if (s < best) { best = s; arg = c; }
        }
        if (argmin_out) argmin_out[i] = arg;
        if (mind_out) mind_out[i] = best;
        loss += best;
        if (Cbar && arg >= 0)
            for (int j = 0; j < d; ++j)
                Cbar[arg * d + j] += ybar * (-2.0) * (X[i * d + j] - C[arg * d + j]);
    }
    if (loss_out) *loss_out = loss;
    return 0;
}

/* ---------------------------------------------------------------------
 * reduce_by_index with any operator of this file, any width (Sec. 5.1.2,
 * the general rule; LINREC included): the semantic loop
 *   hs = replicate m e;  for i: hs[inds[i]] = hs[inds[i]] (.) vals[i]
 * taken in increasing i, so an operator that does not commute combines
 * each bin's elements in index order.  Tape: tp_i = the bin's running
 * value before element i.  Reverse sweep with one adjoint per bin,
 * starting at hsbar[bin]:
 *   for i = n-1..0 (bin k = inds[i] in range):
 *     valsbar_i += J_right(tp_i, v_i)^T gk;   gk = J_left(tp_i, v_i)^T gk
 * with the per-operator Jacobians of the scan sweep.  Indices outside
 * [0, m) are skipped.  vals0/vals1, hsbar0/hsbar1, vbar0/vbar1 and
 * hs_out0/hs_out1 are the width components (the *1 ones for LINREC only);
 * vbar is accumulated, hs_out (nullable) receives the primal.
 * ------------------------------------------------------------------- */
int oracle_hist_general_vjp(int op, int64_t n, int64_t m,
                            const double *vals0, const double *vals1,
                            const int64_t *inds,
                            const double *hsbar0, const double *hsbar1,
                            double *vbar0, double *vbar1,
                            double *hs_out0, double *hs_out1)
{
    if (op < O_ADD || op > O_LINREC) return 1;
    int w = (op == O_LINREC) ? 2 : 1;
    size_t mm = (size_t)(m > 0 ? m : 1), nn = (size_t)(n > 0 ? n : 1);
    double *bins = (double *)malloc(sizeof(double) * mm * (size_t)w);
    double *tp = (double *)malloc(sizeof(double) * nn * (size_t)w);
    double *gb = (double *)malloc(sizeof(double) * mm * (size_t)w);
    if (!bins || !tp || !gb) { free(bins); free(tp); free(gb); return 2; }
    const double *vs[2] = { vals0, vals1 };
    const double *hb[2] = { hsbar0, hsbar1 };
    double *vb[2] = { vbar0, vbar1 };
    double *ho[2] = { hs_out0, hs_out1 };
    for (int64_t k = 0; k < m; ++k) {
        if (op == O_LINREC) { bins[k * 2] = 1.0; bins[k * 2 + 1] = 0.0; }
        else bins[k] = neutral_of(op);
    }
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = inds[i];
        if (k < 0 || k >= m) continue;
        double x[2], out[2];
        for (int c = 0; c < w; ++c) {
            x[c] = vs[c][i];
            tp[i * w + c] = bins[k * w + c];
        }
        scan_combine(op, &tp[i * w], x, out);
        for (int c = 0; c < w; ++c) bins[k * w + c] = out[c];
    }
    for (int64_t k = 0; k < m; ++k)
        for (int c = 0; c < w; ++c) {
            if (ho[c]) ho[c][k] = bins[k * w + c];
            gb[k * w + c] = hb[c] ? hb[c][k] : 0.0;
        }
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t k = inds[i];
        if (k < 0 || k >= m) continue;
        double x[2], to_v[2], to_t[2];
        mat2 Jl, Jr;
        for (int c = 0; c < w; ++c) x[c] = vs[c][i];
        scan_jacobians(op, &tp[i * w], x, &Jl, &Jr);
        mat_t_vec(&Jr, &gb[k * w], to_v, w);
        mat_t_vec(&Jl, &gb[k * w], to_t, w);
        for (int c = 0; c < w; ++c) {
            vb[c][i] += to_v[c];
            gb[k * w + c] = to_t[c];
        }
    }
    free(bins); free(tp); free(gb);
    return 0;
}

/* ---------------------------------------------------------------------
 * Scan VJP with an element of d scalars and full d x d Jacobians (Sec. 5.2,
 * the generalisation to any element type linearised to a vector: J_left
 * and J_right become d x d matrices, lin_o multiplies matrices).  The
 * element i is the row a[i*d .. i*d+d).  Operators:
 *   O_LINREC  (d = 2)  (a1, b1) (.) (a2, b2) = (a2 a1, a2 b1 + b2)
 *   O_MATREC2 (d = 6)  a 2x2 matrix M (row-major, 4 entries) and a 2-vector
 *                      v: (M1, v1) (.) (M2, v2) = (M2 M1, M2 v1 + v2), the
 *                      affine maps x -> M x + v composed in scan order.
 * The tape sweep is the unrolled loop of Sec. 5.2: rs_0 = a_0,
 * rs_i = rs_{i-1} (.) a_i; then rsbar = ybar and, for i = n-1..1,
 *   rsbar_{i-1} += J_left(i)^T rsbar_i;  abar_i += J_right(i)^T rsbar_i,
 * and abar_0 += rsbar_0.  abar is accumulated; ys (nullable) gets rs.
 * ------------------------------------------------------------------- */
enum { O_MATREC2 = 5 };
#define WIDE_MAX 6

typedef struct { double v[WIDE_MAX][WIDE_MAX]; } matw;

static int wide_width(int op)
{
    return op == O_LINREC ? 2 : (op == O_MATREC2 ? 6 : 0);
}

static void wide_combine(int op, const double *l, const double *r, double *out)
{
    if (op == O_LINREC) {
        out[0] = r[0] * l[0];
        out[1] = r[0] * l[1] + r[1];
        return;
    }
    /* r's matrix times l's matrix, r's matrix times l's vector plus r's vector */
    for (int j = 0; j < 2; ++j) {
        for (int k = 0; k < 2; ++k)
            out[2 * j + k] = r[2 * j + 0] * l[0 + k] + r[2 * j + 1] * l[2 + k];
        out[4 + j] = r[2 * j + 0] * l[4] + r[2 * j + 1] * l[5] + r[4 + j];
    }
}

/* J_left = d(prev (.) x)/d prev and J_right = d(prev (.) x)/d x, rows are
 * the output components, columns the input ones */
static void wide_jacobians(int op, const double *prev, const double *x, matw *Jl, matw *Jr)
{
    memset(Jl, 0, sizeof(*Jl));
    memset(Jr, 0, sizeof(*Jr));
    if (op == O_LINREC) {
        /* (A, B) -> (x0 A, x0 B + x1) */
        const double jr[2][2] = { { prev[0], 0.0 }, { prev[1], 1.0 } };
        for (int r = 0; r < 2; ++r) {
            Jl->v[r][r] = x[0];
            for (int c = 0; c < 2; ++c) Jr->v[r][c] = jr[r][c];
        }
        return;
    }
    /* out P[j][k] = sum_m X[j][m] P[m][k];  out h[j] = sum_m X[j][m] h[m] + xv[j] */
    for (int j = 0; j < 2; ++j) {
        for (int k = 0; k < 2; ++k)
            for (int m = 0; m < 2; ++m) {
                Jl->v[2 * j + k][2 * m + k] = x[2 * j + m];   /* d out P[j][k] / d P[m][k] */
                Jr->v[2 * j + k][2 * j + m] = prev[2 * m + k]; /* d out P[j][k] / d X[j][m] */
            }
        for (int m = 0; m < 2; ++m) {
            Jl->v[4 + j][4 + m] = x[2 * j + m];     /* d out h[j] / d h[m] */
            Jr->v[4 + j][2 * j + m] = prev[4 + m];  /* d out h[j] / d X[j][m] */
        }
        Jr->v[4 + j][4 + j] = 1.0;                 /* d out h[j] / d xv[j] */
    }
}

/* y = M^T x for d x d M */
static void matw_t_vec(const matw *M, const double *x, double *y, int d)
{
    for (int c = 0; c < d; ++c) {
        double s = 0.0;
        for (int r = 0; r < d; ++r) s += M->v[r][c] * x[r];
        y[c] = s;
    }
}

int oracle_scan_wide_vjp(int op, int64_t n, int d, const double *a, const double *ybar,
                         double *abar, double *ys)
{
    if (wide_width(op) == 0 || d != wide_width(op)) return 1;
    if (n == 0) return 0;
    double *rs = (double *)malloc(sizeof(double) * (size_t)n * (size_t)d);
    double *rsb = (double *)malloc(sizeof(double) * (size_t)n * (size_t)d);
    if (!rs || !rsb) { free(rs); free(rsb); return 2; }
    for (int c = 0; c < d; ++c) rs[c] = a[c];
    for (int64_t i = 1; i < n; ++i) wide_combine(op, &rs[(i - 1) * d], &a[i * d], &rs[i * d]);
    if (ys) memcpy(ys, rs, sizeof(double) * (size_t)n * (size_t)d);
    memcpy(rsb, ybar, sizeof(double) * (size_t)n * (size_t)d);
    for (int64_t i = n - 1; i >= 1; --i) {
        matw Jl, Jr;
        double back[WIDE_MAX], into[WIDE_MAX];
        wide_jacobians(op, &rs[(i - 1) * d], &a[i * d], &Jl, &Jr);
        matw_t_vec(&Jl, &rsb[i * d], back, d);
        matw_t_vec(&Jr, &rsb[i * d], into, d);
        for (int c = 0; c < d; ++c) {
            rsb[(i - 1) * d + c] += back[c];
            abar[i * d + c] += into[c];
        }
    }
    for (int c = 0; c < d; ++c) abar[c] += rsb[c];
    free(rs); free(rsb);
    return 0;
}

/* ---------------------------------------------------------------------
 * Hessian diagonal of the k-means cost in C (Sec. 7.4, the second-order
 * information the paper obtains by nesting forward mode over the VJP):
 * with every point's argmin held fixed (the cost is piecewise quadratic in
 * C and the argmin changes only on measure-zero ties),
 *   d^2/dc_kj^2 ybar sum_{i: argmin_i = k} (x_ij - c_kj)^2 = 2 ybar |{i: argmin_i = k}|.
 * The argmin is the one oracle_kmeans takes (FP64, lowest k on ties).
 * H is [k*d], overwritten.
 * ------------------------------------------------------------------- */
int oracle_kmeans_hessdiag(int64_t N, int d, int k, const double *X, const double *C,
                           double ybar, double *H)
{
    int64_t *cnt = (int64_t *)calloc((size_t)(k > 0 ? k : 1), sizeof(int64_t));
    if (!cnt) return 2;
    for (int64_t i = 0; i < N; ++i) {
        double best = INFINITY;
        int64_t arg = -1;
        for (int c = 0; c < k; ++c) {
            double s = 0.0;
            for (int j = 0; j < d; ++j) {
                double diff = X[i * d + j] - C[(int64_t)c * d + j];
                s += diff * diff;
            }
            if (s < best) { best = s; arg = c; }
        }
        if (arg >= 0) ++cnt[arg];
    }
    for (int c = 0; c < k; ++c)
        for (int j = 0; j < d; ++j) H[(int64_t)c * d + j] = 2.0 * ybar * (double)cnt[c];
    free(cnt);
    return 0;
}

/* =====================================================================
 * Forward mode (Sec. 3): dual numbers.  Every value of the primal loop
 * carries a tangent, and each operation is followed by its derivative
 * applied to the tangents of its arguments:
 *   t (.) a  ->  tdot' = d(t (.) a)/dt * tdot + d(t (.) a)/da * adot.
 * The primal loops and the partial derivatives (combine, d_dt, d_da) are
 * the ones of the reverse sweeps above, so the duality
 *   <ybar, J xdot> = <J^T ybar, xdot>
 * against the reverse sweeps checks the two directions against each other.
 * ===================================================================== */

/* extended-exponent addition, rounded once like an FP64 add */
static xd xd_add(xd a, xd b)
{
    if (a.m == 0.0) return b;
    if (b.m == 0.0) return a;
    if (a.e < b.e) { xd t = a; a = b; b = t; }
    int64_t d = a.e - b.e;
    if (d > 1100) return a; /* b lies far below half an ulp of a */
    xd r;
    int e = 0;
    r.m = frexp(a.m + ldexp(b.m, (int)(-d)), &e);
    r.e = (r.m == 0.0) ? 0 : a.e + e;
    return r;
}

/* reduce with +, min, max:  t_0 = e, tdot_0 = 0;
 *   tdot_{i+1} = d_dt(t_i, a_i) tdot_i + d_da(t_i, a_i) adot_i,
 *   t_{i+1}    = t_i (.) a_i.
 * For max the tangent follows t on ties (t >= a): the first index. */
int oracle_reduce_jvp(int op, int64_t n, const double *a, const double *adot,
                      double *y_out, double *ydot_out)
{
    if (op != O_ADD && op != O_MIN && op != O_MAX) return 1;
    double t = neutral_of(op), td = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double ft = d_dt(op, t, a[i]), fa = d_da(op, t, a[i]);
        td = (ft != 0.0 ? ft * td : 0.0) + (fa != 0.0 ? fa * adot[i] : 0.0);
        t = combine(op, t, a[i]);
    }
    if (y_out) *y_out = t;
    if (ydot_out) *ydot_out = td;
    return 0;
}

/* reduce with * in extended exponent: the product rule on dual numbers,
 *   tdot_{i+1} = a_i tdot_i + t_i adot_i,   t_{i+1} = t_i a_i,
 * with no division and no case analysis of the zeros.  Outputs the tangent
 * of y rounded to FP64, ln|ydot| (-inf when 0) and its sign. */
int oracle_prod_reduce_jvp(int64_t n, const double *a, const double *adot,
                           double *ydot_val, double *ydot_log, int8_t *ydot_sign)
{
    xd t = xd_make(1.0), td = xd_make(0.0);
    for (int64_t i = 0; i < n; ++i) {
        xd ai = xd_make(a[i]);
        td = xd_add(xd_mul(ai, td), xd_mul(t, xd_make(adot[i])));
        t = xd_mul(t, ai);
    }
    if (ydot_val) *ydot_val = xd_value(td);
    if (ydot_log) *ydot_log = xd_log(td);
    if (ydot_sign) *ydot_sign = (int8_t)xd_sign(td);
    return 0;
}

/* reduce_by_index with +, min, max: the semantic loop of Sec. 5.1.2 on dual
 * numbers, one (value, tangent) per bin, elements taken in index order;
 * out-of-range indices are skipped.  hs_out (nullable) and hsdot_out [m]. */
int oracle_hist_jvp(int op, int64_t n, int64_t m, const double *vals, const double *vdot,
                    const int64_t *inds, double *hs_out, double *hsdot_out)
{
    if (op != O_ADD && op != O_MIN && op != O_MAX) return 1;
    double *hs = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *hd = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!hs || !hd) { free(hs); free(hd); return 2; }
    for (int64_t b = 0; b < m; ++b) { hs[b] = neutral_of(op); hd[b] = 0.0; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) continue;
        double t = hs[b];
        double ft = d_dt(op, t, vals[i]), fa = d_da(op, t, vals[i]);
        hd[b] = (ft != 0.0 ? ft * hd[b] : 0.0) + (fa != 0.0 ? fa * vdot[i] : 0.0);
        hs[b] = combine(op, t, vals[i]);
    }
    for (int64_t b = 0; b < m; ++b) {
        if (hs_out) hs_out[b] = hs[b];
        hsdot_out[b] = hd[b];
    }
    free(hs); free(hd);
    return 0;
}

/* reduce_by_index with * in extended exponent: per bin the product rule on
 * dual numbers; per bin the tangent rounded to FP64, its log and sign. */
int oracle_hist_prod_jvp(int64_t n, int64_t m, const double *vals, const double *vdot,
                         const int64_t *inds, double *hsdot_val, double *hsdot_log,
                         int8_t *hsdot_sign)
{
    xd *t = (xd *)malloc(sizeof(xd) * (size_t)(m > 0 ? m : 1));
    xd *td = (xd *)malloc(sizeof(xd) * (size_t)(m > 0 ? m : 1));
    if (!t || !td) { free(t); free(td); return 2; }
    for (int64_t b = 0; b < m; ++b) { t[b] = xd_make(1.0); td[b] = xd_make(0.0); }
    for (int64_t i = 0; i < n; ++i) {
        int64_t b = inds[i];
        if (b < 0 || b >= m) continue;
        xd vi = xd_make(vals[i]);
        td[b] = xd_add(xd_mul(vi, td[b]), xd_mul(t[b], xd_make(vdot[i])));
        t[b] = xd_mul(t[b], vi);
    }
    for (int64_t b = 0; b < m; ++b) {
        if (hsdot_val) hsdot_val[b] = xd_value(td[b]);
        if (hsdot_log) hsdot_log[b] = xd_log(td[b]);
        if (hsdot_sign) hsdot_sign[b] = (int8_t)xd_sign(td[b]);
    }
    free(t); free(td);
    return 0;
}

/* scatter (Sec. 5.3) on dual numbers: ys = xs with ys[is_j] = vs_j, so
 * ysdot = xsdot with ysdot[is_j] = vsdot_j (in place over xsdot; indices
 * outside [0, n) are skipped). */
int oracle_scatter_jvp(int64_t n, int64_t m, const int64_t *is, const double *vsdot,
                       double *xsdot_inout)
{
    for (int64_t j = 0; j < m; ++j) {
        int64_t k = is[j];
        if (k < 0 || k >= n) continue;
        xsdot_inout[k] = vsdot[j];
    }
    return 0;
}

/* map with a free array (Sec. 5.4) on dual numbers:
 *   xs_j = g(as[is_j], ws_j)  ->  xsdot_j = dg/da asdot[is_j] + dg/dw wsdot_j,
 *   GATHER: xsdot_j = asdot_i;  SCALE: asdot_i w_j + a_i wsdot_j;
 *   SQDIST_ROW: sum_k 2 (w_jk - a_ik)(wsdot_jk - asdot_ik).
 * An index out of range gives xs_j = 0 and a zero tangent.  wsdot may be
 * NULL (no tangent on ws). */
int oracle_map_acc_jvp(int gfun, int64_t nj, int64_t na, int width,
                       const double *as, const int64_t *is, const double *ws,
                       const double *asdot, const double *wsdot, double *xsdot)
{
    for (int64_t j = 0; j < nj; ++j) {
        int64_t i = is[j];
        if (i < 0 || i >= na) { xsdot[j] = 0.0; continue; }
        if (gfun == G_GATHER) {
            xsdot[j] = asdot[i];
        } else if (gfun == G_SCALE) {
            xsdot[j] = asdot[i] * ws[j] + (wsdot ? as[i] * wsdot[j] : 0.0);
        } else if (gfun == G_SQDIST_ROW) {
            double s = 0.0;
            for (int k = 0; k < width; ++k) {
                double diff = ws[j * width + k] - as[i * width + k];
                double dd = (wsdot ? wsdot[j * width + k] : 0.0) - asdot[i * width + k];
                s += 2.0 * diff * dd;
            }
            xsdot[j] = s;
        } else {
            return 1;
        }
    }
    return 0;
}

/* Forward over reverse for the k-means cost (Sec. 7.4 nests forward mode
 * over the VJP for the Hessian diagonal): the forward and reverse sweeps of
 * oracle_kmeans run on dual numbers whose tangent is Cdot (X and ybar carry
 * none).  Per point: the distances and their tangents
 *   s_c = sum_j (x_ij - c_cj)^2,   sdot_c = sum_j 2 (c_cj - x_ij) cdot_cj,
 * the min (lowest k on ties; the argmin itself has no tangent), the loss
 * and its tangent ydot += sdot_k*; then the reverse step
 *   Cbar[k*, j] += ybar (-2)(x_ij - c_k*j)
 * whose tangent is  Cbardot[k*, j] += ybar (-2)(0 - cdot_k*j).
 * Cbardot [k*d] is overwritten; ydot_out (nullable) receives the loss's
 * tangent. */
int oracle_kmeans_fwd_rev(int64_t N, int d, int k, const double *X, const double *C,
                          const double *Cdot, double ybar, double *ydot_out, double *Cbardot)
{
    double ydot = 0.0;
    for (int64_t q = 0; q < (int64_t)k * d; ++q) Cbardot[q] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        double best = INFINITY, bestdot = 0.0;
        int64_t arg = -1;
        for (int c = 0; c < k; ++c) {
            double s = 0.0, sd = 0.0;
            for (int j = 0; j < d; ++j) {
                double diff = X[i * d + j] - C[(int64_t)c * d + j];
                s += diff * diff;
                sd += 2.0 * (-diff) * Cdot[(int64_t)c * d + j];
            }
            if (s < best) { best = s; bestdot = sd; arg = c; }
        }
        ydot += bestdot;
        if (arg >= 0)
            for (int j = 0; j < d; ++j)
                Cbardot[arg * d + j] += ybar * (-2.0) * (0.0 - Cdot[arg * d + j]);
    }
    if (ydot_out) *ydot_out = ydot;
    return 0;
}
