/*
 * tds_oracle.c -- plain CPU FP64 reference for batched compact finite-difference
 * derivatives (the oracle).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library.  The GPU product path shares no
 * code, header, table or constant with it.
 *
 * What it computes, per line of n points (the plain definition D f = A^{-1} (B f)):
 *   1. d = B f, the explicit right-hand side of the compact scheme (Eq. cfds, Sec. 4.2),
 *      written row by row from the stencil definition;
 *   2. A u = d solved by the Thomas algorithm (Algorithm 1, Sec. 2.1) for closed lines,
 *      or by the periodic Thomas algorithm (Sherman-Morrison, Sec. 2.1, last paragraph)
 *      for cyclic lines;
 *   3. the adjoint x = B^T (A^{-T} g): the same solvers applied to the explicitly
 *      transposed band, then the explicitly transposed right-hand-side matrix.
 *
 * Schemes (order 1 from Eq. cfds; order 2 and the closed-boundary closures are the
 * standard Lele-family Pade schemes stated below, since the paper prints none):
 *   order 1 interior: alpha=1/3, a=14/9, b=1/9 on (f[i+1]-f[i-1])/2h and (f[i+2]-f[i-2])/4h
 *   order 2 interior: alpha=2/11, a=12/11, b=3/11 on (f[i+1]-2f[i]+f[i-1])/h^2 and
 *                     (f[i+2]-2f[i]+f[i-2])/4h^2
 *   closed, order 1:  i=0:  f'0 + 2 f'1 = (-5 f0 + 4 f1 + f2)/2h
 *                     i=1:  f'0/4 + f'1 + f'2/4 = (3/2)(f2 - f0)/2h
 *                     i=n-2, n-1: mirror images with the right-hand side negated
 *   closed, order 2:  i=0:  f''0 + 11 f''1 = (13 f0 - 27 f1 + 15 f2 - f3)/h^2
 *                     i=1:  f''0/10 + f''1 + f''2/10 = (6/5)(f0 - 2 f1 + f2)/h^2
 *                     i=n-2, n-1: mirror images
 *
 * Other compact operators of the same tridiagonal form (the paper notes that compact schemes
 * also give interpolations and filters, citing Lele 1992; it prints neither, so these are
 * the standard members of Lele's families, stated here in full).  The slot h then carries
 * the operator's parameter:
 *   order 3, filter (Lele 1992, App. C.2, tridiagonal fourth-order member), h = alpha_f with
 *     |alpha_f| < 1/2:
 *       alpha_f g[i-1] + g[i] + alpha_f g[i+1]
 *         = a0 f[i] + (a1/2)(f[i+1] + f[i-1]) + (a2/2)(f[i+2] + f[i-2]),
 *       a0 = 5/8 + 3 alpha_f/4, a1 = 1/2 + alpha_f, a2 = -1/8 + alpha_f/4
 *     (transfer function 1 at k = 0, 0 at the grid's odd-even mode); closed lines keep the
 *     end values (g[0] = f[0], g[n-1] = f[n-1]) and use the second-order member at rows 1
 *     and n-2 (a0 = a1 = 1/2 + alpha_f, a2 = 0);
 *   order 4, mid-point interpolation (Lele 1992, App. C.1, sixth-order member), h unused:
 *     g[i] approximates f at x[i] + h/2,
 *       alpha g[i-1] + g[i] + alpha g[i+1] = (a/2)(f[i] + f[i+1]) + (b/2)(f[i-1] + f[i+2]),
 *       alpha = 3/10, a = 3/2, b = 1/10;
 *     its transpose (the adjoint) is the interpolation from mid-points back to the nodes.
 *     Closed lines have n - 1 mid-points g[0..n-2]; row n-1 is a zero row (g[n-1] = 0, no
 *     coupling), so that n points map to n.  The first mid-point uses the compact closure with
 *     four nodes that is exact for polynomials through degree 4 (the unique such row with one
 *     coupling g[1]: five conditions, five coefficients),
 *       g[0] + (5/3) g[1] = (5/24) f[0] + (15/8) f[1] + (5/8) f[2] - (1/24) f[3],
 *     and row n-2 its mirror image, (5/3) g[n-3] + g[n-2] = (5/24) f[n-1] + (15/8) f[n-2]
 *     + (5/8) f[n-3] - (1/24) f[n-4]; rows 1 .. n-3 are interior rows.
 *
 * Band convention: row i of A is a[i]*u[i-1] + b[i]*u[i] + c[i]*u[i+1]; for cyclic
 * lines a[0] multiplies u[n-1] and c[n-1] multiplies u[0].  Row i of B is stored as 7
 * taps B7[7*i + 3 + o] multiplying f[i+o], o = -3..3 (indices taken modulo n on cyclic
 * lines).  Everything is double precision; compiled with -ffp-contract=off.
 */
#include <stdlib.h>
#include <string.h>

#define TAPS 7
#define MID 3

/* The filter and the mid-point interpolation (orders 3 and 4 above). */
static int other_bands(int n, int order, int periodic, double param,
                       double *a, double *b, double *c, double *B7)
{
    if (order == 3) {
        const double af = param;
        if (!(af > -0.5 && af < 0.5)) return -1;
        const double a0 = 5.0 / 8.0 + 0.75 * af, a1 = 0.5 + af, a2 = -1.0 / 8.0 + 0.25 * af;
        for (int i = 0; i < n; ++i) {
            a[i] = af; b[i] = 1.0; c[i] = af;
            double *r = B7 + (size_t)TAPS * i + MID;
            r[-2] = 0.5 * a2; r[-1] = 0.5 * a1; r[0] = a0; r[1] = 0.5 * a1; r[2] = 0.5 * a2;
        }
        if (periodic) return 0;
        for (int e = 0; e < 2; ++e) {
            const int i0 = e ? n - 1 : 0, i1 = e ? n - 2 : 1;
            double *r0 = B7 + (size_t)TAPS * i0 + MID, *r1 = B7 + (size_t)TAPS * i1 + MID;
            for (int o = -MID; o <= MID; ++o) { r0[o] = 0.0; r1[o] = 0.0; }
            a[i0] = 0.0; c[i0] = 0.0;
            r0[0] = 1.0;
            r1[-1] = 0.5 * (0.5 + af); r1[0] = 0.5 + af; r1[1] = 0.5 * (0.5 + af);
        }
        return 0;
    }
    /* order 4 */
    const double alpha = 3.0 / 10.0, ha = 0.5 * 1.5, hb = 0.5 * (1.0 / 10.0);
    for (int i = 0; i < n; ++i) {
        a[i] = alpha; b[i] = 1.0; c[i] = alpha;
        double *r = B7 + (size_t)TAPS * i + MID;
        r[-1] = hb; r[0] = ha; r[1] = ha; r[2] = hb;
    }
    if (periodic) return 0;
    /* closed: mid-points 0 .. n-2, the closure rows 0 and n-2, the zero row n-1 */
    double *r0 = B7 + MID, *rm = B7 + (size_t)TAPS * (n - 2) + MID, *rl = B7 + (size_t)TAPS * (n - 1) + MID;
    for (int o = -MID; o <= MID; ++o) { r0[o] = 0.0; rm[o] = 0.0; rl[o] = 0.0; }
    a[0] = 0.0; b[0] = 1.0; c[0] = 5.0 / 3.0;
    r0[0] = 5.0 / 24.0; r0[1] = 15.0 / 8.0; r0[2] = 5.0 / 8.0; r0[3] = -1.0 / 24.0;
    a[n - 2] = 5.0 / 3.0; b[n - 2] = 1.0; c[n - 2] = 0.0;
    rm[1] = 5.0 / 24.0; rm[0] = 15.0 / 8.0; rm[-1] = 5.0 / 8.0; rm[-2] = -1.0 / 24.0;
    a[n - 1] = 0.0; b[n - 1] = 1.0; c[n - 1] = 0.0;
    return 0;
}

/* Interior and closure coefficients: order 1 or 2 with grid spacing h, or the operators of
 * orders 3 and 4 with their parameter in h.  Returns 0 on success, -1 on invalid arguments. */
int tdso_bands(int n, int order, int periodic, double h,
               double *a, double *b, double *c, double *B7)
{
    if (n < 5 || order < 1 || order > 4) return -1;
    memset(B7, 0, sizeof(double) * (size_t)TAPS * (size_t)n);
    if (order >= 3) return other_bands(n, order, periodic, h, a, b, c, B7);
    if (!(h > 0.0)) return -1;
    double alpha, t1, t2, t0;
    if (order == 1) {
        /* Eq. cfds: a/(2h) on f[i+1]-f[i-1], b/(4h) on f[i+2]-f[i-2] */
        alpha = 1.0 / 3.0;
        t1 = (14.0 / 9.0) / (2.0 * h);
        t2 = (1.0 / 9.0) / (4.0 * h);
        t0 = 0.0;
    } else {
        alpha = 2.0 / 11.0;
        t1 = (12.0 / 11.0) / (h * h);
        t2 = (3.0 / 11.0) / (4.0 * h * h);
        t0 = -2.0 * t1 - 2.0 * t2;
    }
    for (int i = 0; i < n; ++i) {
        a[i] = alpha; b[i] = 1.0; c[i] = alpha;
        double *r = B7 + (size_t)TAPS * i + MID;
        if (order == 1) { r[-2] = -t2; r[-1] = -t1; r[0] = t0; r[1] = t1; r[2] = t2; }
        else            { r[-2] =  t2; r[-1] =  t1; r[0] = t0; r[1] = t1; r[2] = t2; }
    }
    if (periodic) return 0;

    /* closed lines: boundary rows replaced by the one-sided closures */
    double *r0 = B7 + MID, *r1 = B7 + TAPS + MID;
    double *rm = B7 + (size_t)TAPS * (n - 2) + MID, *rl = B7 + (size_t)TAPS * (n - 1) + MID;
    for (int o = -MID; o <= MID; ++o) { r0[o] = 0; r1[o] = 0; rm[o] = 0; rl[o] = 0; }
    a[0] = 0.0; c[n - 1] = 0.0;
    if (order == 1) {
        b[0] = 1.0; c[0] = 2.0;
        r0[0] = -5.0 / (2.0 * h); r0[1] = 4.0 / (2.0 * h); r0[2] = 1.0 / (2.0 * h);
        a[1] = 0.25; b[1] = 1.0; c[1] = 0.25;
        r1[-1] = -1.5 / (2.0 * h); r1[1] = 1.5 / (2.0 * h);
        a[n - 2] = 0.25; b[n - 2] = 1.0; c[n - 2] = 0.25;
        rm[-1] = -1.5 / (2.0 * h); rm[1] = 1.5 / (2.0 * h);
        a[n - 1] = 2.0; b[n - 1] = 1.0;
        rl[0] = 5.0 / (2.0 * h); rl[-1] = -4.0 / (2.0 * h); rl[-2] = -1.0 / (2.0 * h);
    } else {
        double h2 = h * h;
        b[0] = 1.0; c[0] = 11.0;
        r0[0] = 13.0 / h2; r0[1] = -27.0 / h2; r0[2] = 15.0 / h2; r0[3] = -1.0 / h2;
        a[1] = 0.1; b[1] = 1.0; c[1] = 0.1;
        r1[-1] = 1.2 / h2; r1[0] = -2.4 / h2; r1[1] = 1.2 / h2;
        a[n - 2] = 0.1; b[n - 2] = 1.0; c[n - 2] = 0.1;
        rm[-1] = 1.2 / h2; rm[0] = -2.4 / h2; rm[1] = 1.2 / h2;
        a[n - 1] = 11.0; b[n - 1] = 1.0;
        rl[0] = 13.0 / h2; rl[-1] = -27.0 / h2; rl[-2] = 15.0 / h2; rl[-3] = -1.0 / h2;
    }
    return 0;
}

/* d = B f for one line (step 1). */
static void apply_B(int n, int periodic, const double *B7, const double *f, double *d)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int o = -MID; o <= MID; ++o) {
            double coef = B7[(size_t)TAPS * i + MID + o];
            if (coef == 0.0) continue;
            int j = i + o;
            if (periodic) j = ((j % n) + n) % n;
            else if (j < 0 || j >= n) continue;
            s += coef * f[j];
        }
        d[i] = s;
    }
}

/* x = B^T y for one line: every tap of row i scatters into column i+o. */
static void apply_BT(int n, int periodic, const double *B7, const double *y, double *x)
{
    for (int j = 0; j < n; ++j) x[j] = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int o = -MID; o <= MID; ++o) {
            double coef = B7[(size_t)TAPS * i + MID + o];
            if (coef == 0.0) continue;
            int j = i + o;
            if (periodic) j = ((j % n) + n) % n;
            else if (j < 0 || j >= n) continue;
            x[j] += coef * y[i];
        }
    }
}

/* Thomas algorithm (Algorithm 1).  a[0] and c[n-1] are ignored.  cp is scratch (n). */
static void thomas(int n, const double *a, const double *b, const double *c,
                   const double *d, double *u, double *cp)
{
    u[0] = d[0] / b[0];
    cp[0] = c[0] / b[0];
    for (int i = 1; i < n; ++i) {
        double w = 1.0 / (b[i] - a[i] * cp[i - 1]);
        u[i] = w * (d[i] - a[i] * u[i - 1]);
        cp[i] = w * c[i];
    }
    for (int i = n - 2; i >= 0; --i) u[i] = u[i] - cp[i] * u[i + 1];
}

/* Periodic Thomas via Sherman-Morrison: A = T + u v^T with gamma = -b[0],
 * T(0,0) = b[0] - gamma, T(n-1,n-1) = b[n-1] - a[0] c[n-1] / gamma,
 * u = (gamma, 0, ..., 0, c[n-1]), v = (1, 0, ..., 0, a[0] / gamma).
 * Solve T y = d and T q = u, then x = y - (v.y)/(1 + v.q) q.  work: 5n doubles. */
static void periodic_thomas(int n, const double *a, const double *b, const double *c,
                            const double *d, double *x, double *work)
{
    double *bb = work, *uu = work + n, *y = work + 2 * n, *q = work + 3 * n, *cp = work + 4 * n;
    double gamma = -b[0];
    for (int i = 0; i < n; ++i) { bb[i] = b[i]; uu[i] = 0.0; }
    bb[0] = b[0] - gamma;
    bb[n - 1] = b[n - 1] - a[0] * c[n - 1] / gamma;
    uu[0] = gamma;
    uu[n - 1] = c[n - 1];
    thomas(n, a, bb, c, d, y, cp);
    thomas(n, a, bb, c, uu, q, cp);
    double vy = y[0] + (a[0] / gamma) * y[n - 1];
    double vq = q[0] + (a[0] / gamma) * q[n - 1];
    double beta = vy / (1.0 + vq);
    for (int i = 0; i < n; ++i) x[i] = y[i] - beta * q[i];
}

/* General tridiagonal solve of one system (cyclic if periodic != 0).  Exposed so the
 * solver can be checked against dense LU on arbitrary diagonally dominant bands. */
int tdso_tridiag_solve(int n, int periodic, const double *a, const double *b,
                       const double *c, const double *d, double *x)
{
    if (n < 3) return -1;
    double *work = (double *)malloc(sizeof(double) * 5 * (size_t)n);
    if (!work) return -2;
    if (periodic) periodic_thomas(n, a, b, c, d, x, work);
    else thomas(n, a, b, c, d, x, work);
    free(work);
    return 0;
}

/* Transposed band of a tridiagonal A (cyclic corners swapped as well). */
static void transpose_band(int n, int periodic, const double *a, const double *b,
                           const double *c, double *at, double *bt, double *ct)
{
    for (int i = 0; i < n; ++i) {
        bt[i] = b[i];
        at[i] = (i > 0) ? c[i - 1] : (periodic ? c[n - 1] : 0.0);
        ct[i] = (i < n - 1) ? a[i + 1] : (periodic ? a[0] : 0.0);
    }
}

/* Derivative of nlines contiguous lines of n points: out = A^{-1} B in, per line. */
int tdso_deriv_lines(int n, long nlines, int order, int periodic, double h,
                     const double *in, double *out)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)n * (3 + TAPS + 6));
    if (!a) return -2;
    double *b = a + n, *c = b + n, *B7 = c + n, *d = B7 + (size_t)TAPS * n, *work = d + n;
    if (tdso_bands(n, order, periodic, h, a, b, c, B7) != 0) { free(a); return -1; }
    for (long l = 0; l < nlines; ++l) {
        const double *f = in + (size_t)l * n;
        double *u = out + (size_t)l * n;
        apply_B(n, periodic, B7, f, d);
        if (periodic) periodic_thomas(n, a, b, c, d, u, work);
        else thomas(n, a, b, c, d, u, work);
    }
    free(a);
    return 0;
}

/* Adjoint of the derivative: out = B^T A^{-T} g, per line. */
int tdso_deriv_adjoint_lines(int n, long nlines, int order, int periodic, double h,
                             const double *g, double *out)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)n * (6 + TAPS + 7));
    if (!a) return -2;
    double *b = a + n, *c = b + n, *at = c + n, *bt = at + n, *ct = bt + n;
    double *B7 = ct + n, *y = B7 + (size_t)TAPS * n, *work = y + n;
    if (tdso_bands(n, order, periodic, h, a, b, c, B7) != 0) { free(a); return -1; }
    transpose_band(n, periodic, a, b, c, at, bt, ct);
    for (long l = 0; l < nlines; ++l) {
        const double *gl = g + (size_t)l * n;
        if (periodic) periodic_thomas(n, at, bt, ct, gl, y, work);
        else thomas(n, at, bt, ct, gl, y, work);
        apply_BT(n, periodic, B7, y, out + (size_t)l * n);
    }
    free(a);
    return 0;
}

/* Right-hand side only (d = B f), per line; used to pin the stencil separately. */
int tdso_rhs_lines(int n, long nlines, int order, int periodic, double h,
                   const double *in, double *out)
{
    double *a = (double *)malloc(sizeof(double) * (size_t)n * (3 + TAPS));
    if (!a) return -2;
    double *b = a + n, *c = b + n, *B7 = c + n;
    if (tdso_bands(n, order, periodic, h, a, b, c, B7) != 0) { free(a); return -1; }
    for (long l = 0; l < nlines; ++l)
        apply_B(n, periodic, B7, in + (size_t)l * n, out + (size_t)l * n);
    free(a);
    return 0;
}
