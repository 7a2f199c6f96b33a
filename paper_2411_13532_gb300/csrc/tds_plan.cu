// tds_plan.cu -- host-side operator preprocessing (Algorithm 4, Sec. 4.2), in FP64.
//
// For one derivative operator the planner produces
//   * the tridiagonal band of A and the stencil taps of B (Eq. cfds and its closures), or a
//     caller-given band (band plans: the solve alone),
//   * per chunk class the Algorithm 4 arrays f, r, w, s^a, s^c and the row-0 normaliser, the
//     folded forward records and the rows whose records are constant,
//   * the reduced chunk-end system and its factorisation (cyclic: Sherman-Morrison),
// for A^{-1} B, its transpose B^T A^{-T} and A^{-1}, on the plan's chunks and (SEGMENTED) on the
// segment partition.  Everything is uploaded once to the device; the kernels only read it.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "tds_internal.h"

namespace tds {
namespace {

// Band of A over the whole line: row J is a[J] u[J-1] + b[J] u[J] + c[J] u[J+1]; on cyclic
// lines a[0] multiplies u[n-1] and c[n-1] multiplies u[0].  Stencil of B as taps[J][o+3].
struct LineOperator {
    std::vector<double> a, b, c;
    std::vector<double> taps;  // n * kTaps
};

void scheme_line(int n, int order, bool periodic, double h, LineOperator &L) {
    L.a.assign(n, 0.0); L.b.assign(n, 1.0); L.c.assign(n, 0.0);
    L.taps.assign((size_t)n * kTaps, 0.0);
    double alpha, t0, t1, t2;
    if (order == 1) {          // Eq. cfds: alpha = 1/3, a = 14/9 over 2h, b = 1/9 over 4h
        alpha = 1.0 / 3.0;
        t1 = (14.0 / 9.0) / (2.0 * h);
        t2 = (1.0 / 9.0) / (4.0 * h);
        t0 = 0.0;
    } else {                   // sixth-order second derivative: 2/11, 12/11 over h^2, 3/11 over 4h^2
        alpha = 2.0 / 11.0;
        t1 = (12.0 / 11.0) / (h * h);
        t2 = (3.0 / 11.0) / (4.0 * h * h);
        t0 = -2.0 * (t1 + t2);
    }
    const double sgn = (order == 1) ? -1.0 : 1.0;  // weight of the mirrored point
    for (int J = 0; J < n; ++J) {
        L.a[J] = alpha; L.c[J] = alpha;
        double *t = &L.taps[(size_t)J * kTaps + 3];
        t[-2] = sgn * t2; t[-1] = sgn * t1; t[0] = t0; t[1] = t1; t[2] = t2;
    }
    if (periodic) return;
    auto row = [&](int J) {
        double *t = &L.taps[(size_t)J * kTaps + 3];
        for (int o = -3; o <= 3; ++o) t[o] = 0.0;
        return t;
    };
    L.a[0] = 0.0; L.c[n - 1] = 0.0;
    double *r0 = row(0), *r1 = row(1), *rm = row(n - 2), *rl = row(n - 1);
    if (order == 1) {
        // f'0 + 2 f'1 = (-5 f0 + 4 f1 + f2)/2h  and  f'0/4 + f'1 + f'2/4 = (3/2)(f2 - f0)/2h
        L.c[0] = 2.0;
        r0[0] = -2.5 / h; r0[1] = 2.0 / h; r0[2] = 0.5 / h;
        L.a[1] = 0.25; L.c[1] = 0.25;
        r1[-1] = -0.75 / h; r1[1] = 0.75 / h;
        L.a[n - 2] = 0.25; L.c[n - 2] = 0.25;
        rm[-1] = -0.75 / h; rm[1] = 0.75 / h;
        L.a[n - 1] = 2.0;
        rl[0] = 2.5 / h; rl[-1] = -2.0 / h; rl[-2] = -0.5 / h;
    } else {
        // f''0 + 11 f''1 = (13 f0 - 27 f1 + 15 f2 - f3)/h^2 and
        // f''0/10 + f''1 + f''2/10 = (6/5)(f0 - 2 f1 + f2)/h^2
        const double ih2 = 1.0 / (h * h);
        L.c[0] = 11.0;
        r0[0] = 13.0 * ih2; r0[1] = -27.0 * ih2; r0[2] = 15.0 * ih2; r0[3] = -1.0 * ih2;
        L.a[1] = 0.1; L.c[1] = 0.1;
        r1[-1] = 1.2 * ih2; r1[0] = -2.4 * ih2; r1[1] = 1.2 * ih2;
        L.a[n - 2] = 0.1; L.c[n - 2] = 0.1;
        rm[-1] = 1.2 * ih2; rm[0] = -2.4 * ih2; rm[1] = 1.2 * ih2;
        L.a[n - 1] = 11.0;
        rl[0] = 13.0 * ih2; rl[-1] = -27.0 * ih2; rl[-2] = 15.0 * ih2; rl[-3] = -1.0 * ih2;
    }
}

// The other compact operators of the same tridiagonal form (the paper notes that compact
// schemes give interpolations and filters too, after Lele 1992, without printing them; these
// are the standard members of Lele's families):
//   order 3, filter with parameter alpha_f (|alpha_f| < 1/2), the fourth-order tridiagonal
//     member: alpha_f g[i-1] + g[i] + alpha_f g[i+1] = a0 f[i] + (a1/2)(f[i+1] + f[i-1])
//     + (a2/2)(f[i+2] + f[i-2]), a0 = 5/8 + 3 alpha_f/4, a1 = 1/2 + alpha_f,
//     a2 = -1/8 + alpha_f/4; closed lines keep the end values and use the second-order member
//     (a0 = a1 = 1/2 + alpha_f) at rows 1 and n-2;
//   order 4, interpolation from the nodes to the mid-points x_i + h/2, the sixth-order member:
//     3/10 g[i-1] + g[i] + 3/10 g[i+1] = 3/4 (f[i] + f[i+1]) + 1/20 (f[i-1] + f[i+2]); a closed
//     line has n-1 mid-points: the first and last use the compact closure exact through degree 4,
//     g[0] + 5/3 g[1] = 5/24 f[0] + 15/8 f[1] + 5/8 f[2] - 1/24 f[3] and its mirror image, and
//     row n-1 is a zero row (g[n-1] = 0) so that the layout maps n points to n.
void other_line(int n, int order, bool periodic, double alpha_f, LineOperator &L) {
    L.a.assign(n, 0.0); L.b.assign(n, 1.0); L.c.assign(n, 0.0);
    L.taps.assign((size_t)n * kTaps, 0.0);
    for (int J = 0; J < n; ++J) {
        double *t = &L.taps[(size_t)J * kTaps + 3];
        if (order == 3) {
            const double a0 = 5.0 / 8.0 + 0.75 * alpha_f, a1 = 0.5 + alpha_f, a2 = -1.0 / 8.0 + 0.25 * alpha_f;
            L.a[J] = alpha_f; L.c[J] = alpha_f;
            t[-2] = 0.5 * a2; t[-1] = 0.5 * a1; t[0] = a0; t[1] = 0.5 * a1; t[2] = 0.5 * a2;
        } else {
            L.a[J] = 0.3; L.c[J] = 0.3;
            t[-1] = 0.05; t[0] = 0.75; t[1] = 0.75; t[2] = 0.05;
        }
    }
    if (periodic) return;
    if (order == 4) {
        double *t0 = &L.taps[3], *tm = &L.taps[(size_t)(n - 2) * kTaps + 3], *tl = &L.taps[(size_t)(n - 1) * kTaps + 3];
        for (int o = -3; o <= 3; ++o) { t0[o] = 0.0; tm[o] = 0.0; tl[o] = 0.0; }
        L.a[0] = 0.0; L.c[0] = 5.0 / 3.0;
        t0[0] = 5.0 / 24.0; t0[1] = 15.0 / 8.0; t0[2] = 5.0 / 8.0; t0[3] = -1.0 / 24.0;
        L.a[n - 2] = 5.0 / 3.0; L.c[n - 2] = 0.0;
        tm[1] = 5.0 / 24.0; tm[0] = 15.0 / 8.0; tm[-1] = 5.0 / 8.0; tm[-2] = -1.0 / 24.0;
        L.a[n - 1] = 0.0; L.c[n - 1] = 0.0;
        return;
    }
    for (int e = 0; e < 2; ++e) {
        const int J0 = e ? n - 1 : 0, J1 = e ? n - 2 : 1;
        double *t0 = &L.taps[(size_t)J0 * kTaps + 3], *t1 = &L.taps[(size_t)J1 * kTaps + 3];
        for (int o = -3; o <= 3; ++o) { t0[o] = 0.0; t1[o] = 0.0; }
        L.a[J0] = 0.0; L.c[J0] = 0.0;
        t0[0] = 1.0;
        t1[-1] = 0.5 * (0.5 + alpha_f); t1[0] = 0.5 + alpha_f; t1[1] = 0.5 * (0.5 + alpha_f);
    }
}

// A caller-given band (a, b, c of n rows each): no stencil (the solve alone).  On closed lines
// a[0] and c[n-1] couple to nothing and are dropped.
void band_line(int n, bool periodic, const double *band, LineOperator &L) {
    L.a.assign(band, band + n);
    L.b.assign(band + n, band + 2 * n);
    L.c.assign(band + 2 * n, band + 3 * n);
    if (!periodic) { L.a[0] = 0.0; L.c[n - 1] = 0.0; }
    L.taps.assign((size_t)n * kTaps, 0.0);
}

// A^T and B^T of a line operator: (A^T)_{J,J-1} = c[J-1], (A^T)_{J,J+1} = a[J+1], and the tap
// of B^T at offset o in row J is B's tap at offset -o in row J+o.
void transpose_line(int n, bool periodic, const LineOperator &L, LineOperator &T) {
    T.a.assign(n, 0.0); T.b = L.b; T.c.assign(n, 0.0);
    T.taps.assign((size_t)n * kTaps, 0.0);
    for (int J = 0; J < n; ++J) {
        T.a[J] = (J > 0) ? L.c[J - 1] : (periodic ? L.c[n - 1] : 0.0);
        T.c[J] = (J < n - 1) ? L.a[J + 1] : (periodic ? L.a[0] : 0.0);
        for (int o = -3; o <= 3; ++o) {
            int I = J + o;
            if (periodic) I = ((I % n) + n) % n;
            else if (I < 0 || I >= n) continue;
            T.taps[(size_t)J * kTaps + 3 + o] = L.taps[(size_t)I * kTaps + 3 - o];
        }
    }
}

// Algorithm 4 on one chunk of m rows with local band (a, b, c): a[0] couples to the previous
// chunk's last unknown, c[m-1] to the next chunk's first.  Returns false on a zero pivot.
bool preprocess_chunk(int m, const double *a, const double *b, const double *c,
                      double *f, double *r, double *w, double *sa, double *sc, double *n1,
                      double *saf, double *scf, double *pi) {
    for (int j = 0; j < 2; ++j) {          // rows 1 and 2 of the paper: normalise only
        if (b[j] == 0.0) return false;
        sa[j] = a[j] / b[j];
        sc[j] = c[j] / b[j];
        w[j] = sc[j];
        f[j] = 1.0 / b[j];
        r[j] = 0.0;   // rows 1 and 2 are not eliminated: d_j = f_j (s_j - r_j d_{j-1}) with r_j = 0
    }
    for (int j = 2; j < m; ++j) {          // forward elimination against row j-1
        const double den = b[j] - a[j] * sc[j - 1];
        if (den == 0.0 || !std::isfinite(den)) return false;
        f[j] = 1.0 / den;
        r[j] = a[j];
        sa[j] = -f[j] * a[j] * sa[j - 1];
        sc[j] = f[j] * c[j];
        w[j] = 0.0;
    }
    // forward-pass couplings, and the weights of the forward values in the back-swept row 1
    for (int j = 0; j < m; ++j) { saf[j] = sa[j]; scf[j] = sc[j]; pi[j] = 0.0; }
    pi[1] = 1.0;
    for (int j = 2; j <= m - 2; ++j) pi[j] = -pi[j - 1] * scf[j - 1];
    for (int j = m - 3; j >= 1; --j) {     // backward elimination against row j+1
        sa[j] = sa[j] - sc[j] * sa[j + 1];
        w[j] = sc[j];
        sc[j] = -sc[j] * sc[j + 1];
    }
    const double den = 1.0 - sc[0] * sa[1];  // row 1 of the paper eliminates u_2
    if (den == 0.0 || !std::isfinite(den)) return false;
    *n1 = 1.0 / den;
    sa[0] = *n1 * sa[0];
    sc[0] = -*n1 * sc[0] * sc[1];
    // w[0] keeps c_0/b_0 for the final row-0 step of the sweep
    return true;
}

} // namespace

// Build one operator (A^{-1}B if which == 0, B^T A^{-T} if which == 1, A^{-1} if which == 2)
// into host buffers.
// On periodic lines A and B are circulant, so they commute and A is symmetric:
// B^T A^{-T} = A^{-1} B^T, the forward form with the transposed stencil (L is then the
// transposed line operator, whose band equals A's); op.adjoint is set only for closed lines,
// whose adjoint runs the transposed solve followed by the transposed stencil.
static tds_status build_operator(const tds_plan *p, int P, int m, const LineOperator &L, int which,
                                 DevOp &op, std::vector<double> &rows,
                                 std::vector<double> &n1s, std::vector<double> &red,
                                 std::vector<double> &sub, std::vector<double> &sup,
                                 std::vector<double> &fwd, std::vector<double> &bwd,
                                 std::vector<double> &ifw, std::vector<double> &ifw32,
                                 std::vector<float> &fwdd, std::vector<float> &bwdd,
                                 std::vector<float> &ifwd) {
    const int n = p->n;
    const bool periodic = (p->bc == TDS_BC_PERIODIC);
    std::memset(&op, 0, sizeof(op));
    op.n = n; op.m = m; op.P = P; op.nlines = p->nlines; op.ngroups = p->nlines / kSZ;
    const bool fwd_form = (which == 0) || (which == 1 && periodic);
    op.periodic = periodic; op.adjoint = fwd_form ? 0 : which;
    if (op.adjoint == 1 && m >= 16) {
        // FP32 sweeps fold x = B^T y into the back-substitution (measured at 512^3, P = 8, D1^T /
        // D2^T: 0.249 / 0.265 -> 0.235 / 0.262 ms); FP64 sweeps, bound by the FP64 pipe, keep the
        // separate pass (folded 2.38 / 2.53 -> 2.47 / 2.70 ms).  TDS_ADJOINT_FOLD = 0 / 1 forces
        // either form (tuning).
        const char *e = std::getenv("TDS_ADJOINT_FOLD");
        op.bt_fold = (e && (e[0] == '0' || e[0] == '1')) ? (e[0] == '1') : (p->dtype == TDS_F32);
    }
    // interior stencil form: the interpolation's transpose pairs its taps about -1/2; the
    // second derivative's taps (vanishing sum) may be applied to second differences
    op.symmetric = (p->order == 1) ? -1 : (p->order == 4) ? (which == 1 ? 3 : 2) : (p->order == 2 ? 4 : 1);

    // chunk classes: cyclic lines have one; closed lines distinguish first / interior / last.
    // A caller's band whose chunks differ beyond that (variable coefficients along the line)
    // makes every chunk its own class: Algorithm 4 runs per chunk on that chunk's rows.
    std::vector<int> reps;
    if (periodic || P == 1) { op.ncls = 1; reps = {0}; op.cls_first = op.cls_mid = op.cls_last = 0; }
    else if (P == 2) { op.ncls = 2; reps = {0, 1}; op.cls_first = 0; op.cls_mid = 0; op.cls_last = 1; }
    else { op.ncls = 3; reps = {0, 1, P - 1}; op.cls_first = 0; op.cls_mid = 1; op.cls_last = 2; }
    {
        auto same = [&](int k, int r) {   // chunks k and r carry the same band
            for (int j = 0; j < m; ++j) {
                const size_t x = (size_t)k * m + j, y = (size_t)r * m + j;
                if (L.a[x] != L.a[y] || L.b[x] != L.b[y] || L.c[x] != L.c[y]) return false;
            }
            return true;
        };
        bool uniform = true;
        for (int k = 0; k < P && uniform; ++k) {
            const int cl = (k == 0) ? op.cls_first : (k == P - 1 ? op.cls_last : op.cls_mid);
            uniform = same(k, reps[cl]);
        }
        if (!uniform) {
            op.ncls = P;
            op.cls_each = 1;
            reps.resize(P);
            for (int k = 0; k < P; ++k) reps[k] = k;
        }
    }
    auto class_of = [&](int k) {
        return op.cls_each ? k : (k == 0) ? op.cls_first : (k == P - 1 ? op.cls_last : op.cls_mid);
    };

    const int nc = op.ncls;
    rows.assign((size_t)kNumRowArrays * nc * m, 0.0);
    n1s.assign(nc, 0.0);
    fwd.assign((size_t)nc * m * 4, 0.0);
    bwd.assign((size_t)nc * m * 2, 0.0);
    std::vector<double> saf(m), scf(m), pi(m);
    for (int cl = 0; cl < nc; ++cl) {
        const int k = reps[cl];
        double *f = &rows[((size_t)kF * nc + cl) * m], *r = &rows[((size_t)kR * nc + cl) * m];
        double *w = &rows[((size_t)kW * nc + cl) * m], *sa = &rows[((size_t)kSA * nc + cl) * m];
        double *sc = &rows[((size_t)kSC * nc + cl) * m];
        if (!preprocess_chunk(m, &L.a[(size_t)k * m], &L.b[(size_t)k * m], &L.c[(size_t)k * m],
                              f, r, w, sa, sc, &n1s[cl], saf.data(), scf.data(), pi.data()))
            return TDS_ERR_ARG;
        for (int j = 0; j < m; ++j) {
            double *fw = &fwd[((size_t)cl * m + j) * 4], *bw = &bwd[((size_t)cl * m + j) * 2];
            fw[0] = f[j]; fw[1] = r[j]; fw[2] = pi[j]; fw[3] = 0.0;
            bw[0] = saf[j]; bw[1] = scf[j];
        }
    }
    // stencil taps: interior row (any row at least 4 from a closed end) and the edge rows
    const int mid = n / 2;
    for (int o = 0; o < kTaps; ++o) op.tap[o] = L.taps[(size_t)mid * kTaps + o];
    if (!periodic) {
        for (int e = 0; e < kEdgeRows; ++e)
            for (int o = 0; o < kTaps; ++o) {
                op.edge[e][o] = L.taps[(size_t)e * kTaps + o];
                op.edge[kEdgeRows + e][o] = L.taps[(size_t)(n - kEdgeRows + e) * kTaps + o];
            }
        for (int e = 0; e < 2 * kEdgeRows; ++e)
            for (int o = 0; o < kTaps; ++o) {
                const float hi = (float)op.edge[e][o];
                op.edge_pf[e][o][0] = hi;
                op.edge_pf[e][o][1] = (float)(op.edge[e][o] - (double)hi);
            }
    }
    // the form each edge row is evaluated in (DevOp::edge_form): moments of its taps
    for (int e = 0; e < 2 * kEdgeRows; ++e) {
        double m0 = 0.0, m1 = 0.0, mag = 0.0;
        for (int o = 0; o < kTaps; ++o) {
            m0 += op.edge[e][o];
            m1 += (o - 3) * op.edge[e][o];
            mag += std::fabs(op.edge[e][o]);
        }
        const double tol = 1e-12 * mag;
        op.edge_form[e] = (std::fabs(m0) <= tol) ? ((std::fabs(m1) <= 3.0 * tol) ? 2 : 1) : 0;
        // second-difference weights: d_k = sum_{o < k} (k - o) c_o (the taps' discrete second
        // antiderivative; it vanishes at k = 0 and k = 6 when both moments do)
        for (int k = 1; k <= 5; ++k) {
            double d = 0.0;
            for (int o = 0; o < k; ++o) d += (k - o) * op.edge[e][o];
            op.edge_dd[e][k - 1] = d;
        }
    }

    // symmetric interior taps: FP32 sweeps apply them as t1, t2 on second differences plus the tap
    // sum on the centre value -- exactly zero for a second derivative, so nothing cancels there
    const bool sym = (op.symmetric == 1 || op.symmetric == 4);
    op.tapsum = (op.symmetric == 4) ? 0.0 : op.tap[3] + 2.0 * (op.tap[4] + op.tap[5]);
    op.tapsum32 = (float)op.tapsum;
    for (int o = 0; o < kTaps; ++o) op.tap32[o] = (float)op.tap[o];
    for (int e = 0; e < 2 * kEdgeRows; ++e)
        for (int k = 0; k < 5; ++k) op.edge_dd32[e][k] = (float)op.edge_dd[e][k];

    // interior forward records with f folded in (FP32 records: the tap sum in place of t0 for
    // symmetric taps), and the cut-off rows of pi and s^a
    ifw.assign((size_t)nc * m * 4, 0.0);
    ifw32.assign((size_t)nc * m * 4, 0.0);
    for (int cl = 0; cl < nc; ++cl) {
        for (int j = 0; j < m; ++j) {
            const double f = fwd[((size_t)cl * m + j) * 4], r = fwd[((size_t)cl * m + j) * 4 + 1];
            double *c = &ifw[((size_t)cl * m + j) * 4], *c32 = &ifw32[((size_t)cl * m + j) * 4];
            if (fwd_form) { c[0] = f * op.tap[3]; c[1] = f * op.tap[4]; c[2] = f * op.tap[5]; }
            else { c[0] = f; c[1] = 0.0; c[2] = 0.0; }
            c[3] = f * r;
            for (int q = 0; q < 4; ++q) c32[q] = c[q];
            if (fwd_form && sym) c32[0] = f * op.tapsum;
        }
        auto cutoff = [&](int idx, double tol) {   // first row after which |x_j| <= tol
            int j0 = m;
            while (j0 > 0 && std::fabs(idx == 0 ? fwd[((size_t)cl * m + j0 - 1) * 4 + 2]
                                                : bwd[((size_t)cl * m + j0 - 1) * 2]) <= tol)
                --j0;
            return j0;
        };
        if (op.cls_each) {
            // one entry for all chunks: the latest cut-off of any chunk, and no constant runs
            // (the records of a variable band differ from row to row)
            if (cl == 0) {
                op.jpi64[0] = op.jsa64[0] = op.jpi32[0] = op.jsa32[0] = op.jpid[0] = op.jsad[0] = 0;
                op.kfl64[0] = op.kfh64[0] = op.kbl64[0] = op.kbh64[0] = 0;
                op.kfl32[0] = op.kfh32[0] = op.kbl32[0] = op.kbh32[0] = 0;
            }
            op.jpi64[0] = std::max(op.jpi64[0], cutoff(0, std::ldexp(1.0, -60)));
            op.jsa64[0] = std::max(op.jsa64[0], cutoff(1, std::ldexp(1.0, -60)));
            op.jpi32[0] = std::max(op.jpi32[0], cutoff(0, std::ldexp(1.0, -30)));
            op.jsa32[0] = std::max(op.jsa32[0], cutoff(1, std::ldexp(1.0, -30)));
            op.jpid[0] = std::max(op.jpid[0], cutoff(0, std::ldexp(1.0, -56)));
            op.jsad[0] = std::max(op.jsad[0], cutoff(1, std::ldexp(1.0, -56)));
            continue;
        }
        op.jpi64[cl] = cutoff(0, std::ldexp(1.0, -60));
        op.jsa64[cl] = cutoff(1, std::ldexp(1.0, -60));
        op.jpi32[cl] = cutoff(0, std::ldexp(1.0, -30));
        op.jsa32[cl] = cutoff(1, std::ldexp(1.0, -30));
        op.jpid[cl] = cutoff(0, std::ldexp(1.0, -56));
        op.jsad[cl] = cutoff(1, std::ldexp(1.0, -56));
        // the run of rows around row m-3 (interior in every class) whose records equal that
        // row's, bitwise in each precision
        const int ref = m - 3;
        auto run = [&](auto same, int &lo, int &hi) {
            lo = ref;
            while (lo > 0 && same(lo - 1)) --lo;
            hi = ref + 1;
            while (hi < m && same(hi)) ++hi;
        };
        const double *rf = &ifw[((size_t)cl * m + ref) * 4];
        auto fsame64 = [&](int j) {
            const double *x = &ifw[((size_t)cl * m + j) * 4];
            return x[0] == rf[0] && x[1] == rf[1] && x[2] == rf[2] && x[3] == rf[3];
        };
        const double *rf32 = &ifw32[((size_t)cl * m + ref) * 4];
        auto fsame32 = [&](int j) {
            const double *x = &ifw32[((size_t)cl * m + j) * 4];
            for (int q = 0; q < 4; ++q)
                if ((float)x[q] != (float)rf32[q]) return false;
            return true;
        };
        const double rb = bwd[((size_t)cl * m + ref) * 2 + 1];
        auto bsame64 = [&](int j) { return bwd[((size_t)cl * m + j) * 2 + 1] == rb; };
        auto bsame32 = [&](int j) { return (float)bwd[((size_t)cl * m + j) * 2 + 1] == (float)rb; };
        run(fsame64, op.kfl64[cl], op.kfh64[cl]);
        run(fsame32, op.kfl32[cl], op.kfh32[cl]);
        run(bsame64, op.kbl64[cl], op.kbh64[cl]);
        run(bsame32, op.kbl32[cl], op.kbh32[cl]);
        for (int q = 0; q < 4; ++q) {
            op.kf64[cl][q] = rf[q];
            op.kf32[cl][q] = (float)rf32[q];
        }
        op.kb64[cl] = rb;
        op.kb32[cl] = (float)rb;
    }

    // float-pair records of the split-precision FP64 sweeps (value = hi + lo, hi the float
    // nearest to the FP64 record, lo the float nearest to the rest): fwd {f, r, pi}, bwd
    // {s^a, s^c}, and the interior records in the form those sweeps evaluate the stencil --
    // antisymmetric taps {0, f t1, f t2, f r} on v[j+1] - v[j-1] and v[j+2] - v[j-2};
    // symmetric taps {f tapsum, f (t1 + 2 t2), f t2, f r} on v[j], the second difference
    // e_j = v[j+1] - 2 v[j] + v[j-1] and e_{j+1} + e_{j-1} (t1 e_j + t2 (v[j+2] - 2 v[j] + v[j-2])
    // with v[j+2] - 2 v[j] + v[j-2] = e_{j+1} + 2 e_j + e_{j-1})
    auto pair = [](double x, float *d) {
        d[0] = (float)x;
        d[1] = (float)(x - (double)d[0]);
    };
    fwdd.assign((size_t)nc * m * 8, 0.0f);
    bwdd.assign((size_t)nc * m * 4, 0.0f);
    ifwd.assign((size_t)nc * m * 8, 0.0f);
    for (int cl = 0; cl < nc; ++cl)
        for (int j = 0; j < m; ++j) {
            const size_t i = (size_t)cl * m + j;
            pair(fwd[i * 4], &fwdd[i * 8]);
            pair(fwd[i * 4 + 1], &fwdd[i * 8 + 2]);
            pair(fwd[i * 4 + 2], &fwdd[i * 8 + 4]);
            pair(bwd[i * 2], &bwdd[i * 4]);
            pair(bwd[i * 2 + 1], &bwdd[i * 4 + 2]);
            const double f = fwd[i * 4];
            double c[4] = {ifw[i * 4], ifw[i * 4 + 1], ifw[i * 4 + 2], ifw[i * 4 + 3]};
            if (fwd_form && sym) {
                c[0] = f * op.tapsum;
                c[1] = f * (op.tap[4] + 2.0 * op.tap[5]);
                c[2] = f * op.tap[5];
            } else if (fwd_form && op.symmetric < 0) {
                c[0] = 0.0;
            }
            for (int q = 0; q < 4; ++q) pair(c[q], &ifwd[i * 8 + 2 * q]);
        }
    for (int cl = 0; cl < (op.cls_each ? 0 : nc); ++cl) {
        // the constant runs of the FP64 records carry constant pair records too
        const size_t i = (size_t)cl * m + (m - 3);
        for (int q = 0; q < 8; ++q) op.kfd[cl][q] = ifwd[i * 8 + q];
        op.kbd[cl][0] = bwdd[i * 4 + 2];
        op.kbd[cl][1] = bwdd[i * 4 + 3];
    }

    // reduced chunk-end system, unknowns F_0, L_0, F_1, L_1, ... (2P)
    const int R = 2 * P;
    sub.assign(R, 0.0); sup.assign(R, 0.0);
    for (int k = 0; k < P; ++k) {
        const int cl = class_of(k);
        const double *sa = &rows[((size_t)kSA * nc + cl) * m];
        const double *sc = &rows[((size_t)kSC * nc + cl) * m];
        sub[2 * k] = sa[0];          // row F_k: coupling to L_{k-1}
        sup[2 * k] = sc[0];          //          coupling to its own L_k
        sub[2 * k + 1] = sa[m - 1];  // row L_k: coupling to its own F_k
        sup[2 * k + 1] = sc[m - 1];  //          coupling to F_{k+1}
        if (p->mode == TDS_REDUCED_PAPER_DROP) { sup[2 * k] = 0.0; sub[2 * k + 1] = 0.0; }
    }
    red.assign((size_t)kNumRedArrays * R, 0.0);
    double *rsub = &red[(size_t)kRedSub * R], *wf = &red[(size_t)kRedWf * R];
    double *cp = &red[(size_t)kRedCp * R], *q = &red[(size_t)kRedQ * R];
    std::vector<double> diag(R, 1.0);
    for (int i = 0; i < R; ++i) rsub[i] = sub[i];
    op.red_cyclic = periodic;
    double gamma = -1.0;
    if (periodic) {   // A = T' + u v^T, u = (gamma, 0.., sup_last), v = (1, 0.., sub_0/gamma)
        diag[0] = 1.0 - gamma;
        diag[R - 1] = 1.0 - sub[0] * sup[R - 1] / gamma;
        rsub[0] = 0.0;
    }
    for (int i = 0; i < R; ++i) {
        const double den = diag[i] - (i > 0 ? rsub[i] * cp[i - 1] : 0.0);
        if (den == 0.0 || !std::isfinite(den)) return TDS_ERR_ARG;
        wf[i] = 1.0 / den;
        cp[i] = (i < R - 1) ? wf[i] * sup[i] : 0.0;
    }
    // Decoupled form (the communication phase of Sec. 4.2 / Fig. alg): boundary k joins L_{k-1}
    // and F_k.  It is exact for P = 1 (both couplings of the single chunk's ends are kept, summed)
    // and for the paper-drop mode; for P >= 2 in exact mode it is used only when the couplings
    // it ignores (F_k <-> L_k within a chunk) are below kDecoupleTol.
    {
        double dropped = 0.0;
        for (int k = 0; k < P; ++k)
            dropped = std::fmax(dropped, std::fmax(std::fabs(sup[2 * k]), std::fabs(sub[2 * k + 1])));
        op.red_decoupled = (P == 1) || p->mode == TDS_REDUCED_PAPER_DROP || dropped <= kDecoupleTol;
        double *ba = &red[(size_t)kRedBa * R], *bc = &red[(size_t)kRedBc * R];
        double *binv = &red[(size_t)kRedBinv * R];
        for (int k = 0; k < P; ++k) {
            const int prev = (k - 1 + P) % P;
            double a = sub[2 * k], c = sup[2 * prev + 1];
            if (P == 1) { a += sup[0]; c += sub[1]; }
            const double det = 1.0 - a * c;
            if (op.red_decoupled && (det == 0.0 || !std::isfinite(det))) return TDS_ERR_ARG;
            ba[k] = a; bc[k] = c; binv[k] = 1.0 / det;
        }
    }
    if (periodic) {
        std::vector<double> u(R, 0.0);
        u[0] = gamma; u[R - 1] += sup[R - 1];
        for (int i = 0; i < R; ++i) q[i] = wf[i] * (u[i] - (i > 0 ? rsub[i] * q[i - 1] : 0.0));
        for (int i = R - 2; i >= 0; --i) q[i] -= cp[i] * q[i + 1];
        op.red_vlast = sub[0] / gamma;
        const double den = 1.0 + q[0] + op.red_vlast * q[R - 1];
        if (den == 0.0 || !std::isfinite(den)) return TDS_ERR_ARG;
        op.red_den_inv = 1.0 / den;
    }
    return TDS_OK;
}

// How much an FP32 rounding near a closed line's ends can grow in the solve: the largest |entry|
// of A^{-1} and of A^{-T} in the four columns at each end (Thomas solves of unit vectors in
// FP64).  Closures such as f''_0 + 11 f''_1 make it about 93, f'_0 + 2 f'_1 about 5, the filter's about 2.
static double end_gain(const LineOperator &L, int n) {
    std::vector<double> cp(n), x(n);
    double g = 0.0;
    for (int tr = 0; tr < 2; ++tr) {
        // band of A (tr = 0) or A^T (tr = 1): sub, diag, super of row J
        auto sub = [&](int J) { return tr ? (J > 0 ? L.c[J - 1] : 0.0) : (J > 0 ? L.a[J] : 0.0); };
        auto sup = [&](int J) { return tr ? (J < n - 1 ? L.a[J + 1] : 0.0) : (J < n - 1 ? L.c[J] : 0.0); };
        for (int k = 0; k < 2 * kEdgeRows; ++k) {
            const int col = (k < kEdgeRows) ? k : n - 2 * kEdgeRows + k;
            double den = L.b[0];
            if (den == 0.0) return 1e300;
            cp[0] = sup(0) / den;
            x[0] = (col == 0) ? 1.0 / den : 0.0;
            for (int J = 1; J < n; ++J) {
                den = L.b[J] - sub(J) * cp[J - 1];
                if (den == 0.0 || !std::isfinite(den)) return 1e300;
                cp[J] = sup(J) / den;
                x[J] = ((J == col ? 1.0 : 0.0) - sub(J) * x[J - 1]) / den;
            }
            for (int J = n - 2; J >= 0; --J) x[J] -= cp[J] * x[J + 1];
            for (int J = 0; J < n; ++J) g = std::fmax(g, std::fabs(x[J]));
        }
    }
    return g;
}

// Records of the plain Thomas algorithm on whole lines (Algorithm 1), stencil fused into the
// forward pass; cyclic lines (Sec. 2.1): Sherman-Morrison with A = A' + u v^T, gamma = -b_0,
// u = (gamma, 0, ..., 0, A[n-1][0]), v = (1, 0, ..., 0, A[0][n-1] / gamma), so that
// x = y - (v.y / (1 + v.z)) z with A' y = d and A' z = u.  Device layout in tds_plan::thomas_mem.
static tds_status build_thomas(tds_plan *p, const LineOperator &L, const DevOp &op) {
    const int n = p->n;
    const bool periodic = (p->bc == TDS_BC_PERIODIC);
    std::vector<double> a(L.a), b(L.b), c(L.c);
    double ratio = 0.0, gamma = 0.0;
    const double top = L.a[0], bot = L.c[n - 1];   // A[0][n-1], A[n-1][0] on cyclic lines
    if (periodic) {
        gamma = -b[0];
        if (gamma == 0.0) return TDS_ERR_ARG;
        b[0] -= gamma;
        b[n - 1] -= top * bot / gamma;
        ratio = top / gamma;
    }
    a[0] = 0.0;
    c[n - 1] = 0.0;
    std::vector<double> f(n), cp(n);
    for (int j = 0; j < n; ++j) {
        const double den = b[j] - (j > 0 ? a[j] * cp[j - 1] : 0.0);
        if (den == 0.0 || !std::isfinite(den)) return TDS_ERR_ARG;
        f[j] = 1.0 / den;
        cp[j] = c[j] * f[j];
    }
    std::vector<double> z;
    double inv_den = 0.0;
    if (periodic) {
        z.assign(n, 0.0);
        for (int j = 0; j < n; ++j) {
            const double u = (j == 0) ? gamma : (j == n - 1 ? bot : 0.0);
            z[j] = f[j] * (u - (j > 0 ? a[j] * z[j - 1] : 0.0));
        }
        for (int j = n - 2; j >= 0; --j) z[j] -= cp[j] * z[j + 1];
        const double den = 1.0 + z[0] + ratio * z[n - 1];
        if (den == 0.0 || !std::isfinite(den)) return TDS_ERR_ARG;
        inv_den = 1.0 / den;
    }
    const bool sym = (op.symmetric == 1 || op.symmetric == 4);
    const size_t nz = periodic ? (size_t)n : 0;
    // [rec64 n x 4][fc64 n x 2][z64 n][rec32 n x 4][fc32 n x 2][z32 n]
    const size_t bytes64 = ((size_t)n * 6 + nz) * sizeof(double), bytes32 = ((size_t)n * 6 + nz) * sizeof(float);
    const size_t off32 = (bytes64 + 255) & ~(size_t)255;
    std::vector<unsigned char> host(off32 + bytes32, 0);
    double *r64 = reinterpret_cast<double *>(host.data());
    float *r32 = reinterpret_cast<float *>(host.data() + off32);
    for (int j = 0; j < n; ++j) {
        const double rec[4] = {f[j] * op.tap[3], f[j] * op.tap[4], f[j] * op.tap[5], f[j] * a[j]};
        for (int q = 0; q < 4; ++q) {
            r64[4 * (size_t)j + q] = rec[q];
            r32[4 * (size_t)j + q] = (float)rec[q];
        }
        if (sym) r32[4 * (size_t)j] = (float)(f[j] * op.tapsum);
        r64[4 * (size_t)n + 2 * (size_t)j] = f[j];
        r64[4 * (size_t)n + 2 * (size_t)j + 1] = cp[j];
        r32[4 * (size_t)n + 2 * (size_t)j] = (float)f[j];
        r32[4 * (size_t)n + 2 * (size_t)j + 1] = (float)cp[j];
        if (periodic) {
            r64[6 * (size_t)n + j] = z[j];
            r32[6 * (size_t)n + j] = (float)z[j];
        }
    }
    void *d = nullptr;
    const cudaError_t e = cudaMalloc(&d, host.size());
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TDS_ERR_NOMEM : TDS_ERR_CUDA;
    }
    if (cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return TDS_ERR_CUDA;
    }
    p->thomas_mem = d;
    p->thomas_ratio = ratio;
    p->thomas_inv_den = inv_den;
    if (n >= 2 * kEdgeRows) {
        for (int t = 0; t < 2 * kEdgeRows; ++t) {
            const int j = (t < kEdgeRows) ? t : n - 2 * kEdgeRows + t;
            const double v[3] = {f[j], cp[j], f[j] * a[j]};
            for (int q = 0; q < 3; ++q) {
                const float hi = (float)v[q];
                p->thomas_end_pf[t][q][0] = hi;
                p->thomas_end_pf[t][q][1] = (float)(v[q] - (double)hi);
            }
        }
    }
    return TDS_OK;
}

tds_status build_plan(tds_plan *p) {
    const bool periodic = (p->bc == TDS_BC_PERIODIC);
    LineOperator L, LT;
    if (p->band) band_line(p->n, periodic, p->band, L);
    else if (p->order >= 3) other_line(p->n, p->order, periodic, p->h, L);
    else scheme_line(p->n, p->order, periodic, p->h, L);
    transpose_line(p->n, periodic, L, LT);

    // operators: [0] A^{-1} B, [1] B^T A^{-T} and [2] A^{-1} on the plan's P chunks; [3] A^{-1} B
    // on the segment partition of the SEGMENTED variant: segments of sg rows, 64 <= sg <= 32 KB of
    // one group's rows, sg dividing the chunk length (so segment boundaries include the chunk
    // boundaries), used only if every boundary system decouples; [4] on periodic lines the
    // adjoint on that partition (forward form, see build_operator)
    int sg = 0;
    {
        int cap = (p->dtype == TDS_F64) ? 128 : 256;
        if (const char *e = std::getenv("TDS_SEG_ROWS")) {   // longest segment (tuning)
            const int v = std::atoi(e);
            if (v >= 64 && v <= 4096) cap = v;
        }
        for (int d = (p->m < cap ? p->m : cap); d >= 64; --d)
            if (p->m % d == 0) { sg = d; break; }
    }
    const int nops = sg ? (periodic ? 5 : 4) : 3;
    std::vector<double> rows[5], n1s[5], red[5], sub[5], sup[5], fwd[5], bwd[5], ifw[5], ifw32[5];
    std::vector<float> fwdd[5], bwdd[5], ifwd[5];
    DevOp *ops[5] = {&p->op[0], &p->op[1], &p->op[2], &p->seg, &p->seg_adj};
    std::memset(&p->seg, 0, sizeof(p->seg));
    std::memset(&p->seg_adj, 0, sizeof(p->seg_adj));
    for (int w = 0; w < nops; ++w) {
        const int P = (w < 3) ? p->P : p->n / sg, m = (w < 3) ? p->m : sg;
        const int kind = (w == 1 || w == 4) ? 1 : (w == 2 ? 2 : 0);
        tds_status s = build_operator(p, P, m, kind == 1 ? LT : L, kind, *ops[w], rows[w], n1s[w],
                                      red[w], sub[w], sup[w], fwd[w], bwd[w], ifw[w], ifw32[w], fwdd[w],
                                      bwdd[w], ifwd[w]);
        if (s != TDS_OK) return s;
    }
    // FP32 and split-precision FP64 sweeps of closed lines take the closure rows in FP64 where the
    // solve magnifies an end row's rounding by more than 16 (FP32: 2^-24 x 16 ~ 1e-6; float
    // pairs: 2^-48 x 16 ~ 6e-14, against about 3e-13 at the gain of 93 of the second derivative's
    // closure); native FP64 sweeps ignore the flag
    const int e64 = (!periodic && end_gain(L, p->n) > 16.0) ? 1 : 0;
    for (int w = 0; w < nops; ++w) ops[w]->e64 = e64;
    if (nops >= 4 && (!p->seg.red_decoupled || (nops == 5 && !p->seg_adj.red_decoupled))) {
        std::memset(&p->seg, 0, sizeof(p->seg));
        std::memset(&p->seg_adj, 0, sizeof(p->seg_adj));
    }

    // one device allocation per plan, 256-byte aligned parts per operator:
    // [rows64 | rows32 | n1 | red | fwd64 | fwd32 | bwd64 | bwd32 | ifw64 | ifw32 | fwd, bwd and
    //  ifw float pairs]
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t off[5][13], total = 0;
    for (int w = 0; w < nops; ++w) {
        off[w][0] = total; total = align(total + rows[w].size() * sizeof(double));
        off[w][1] = total; total = align(total + rows[w].size() * sizeof(float));
        off[w][2] = total; total = align(total + n1s[w].size() * sizeof(double));
        off[w][3] = total; total = align(total + red[w].size() * sizeof(double));
        off[w][4] = total; total = align(total + fwd[w].size() * sizeof(double));
        off[w][5] = total; total = align(total + fwd[w].size() * sizeof(float));
        off[w][6] = total; total = align(total + bwd[w].size() * sizeof(double));
        off[w][7] = total; total = align(total + bwd[w].size() * sizeof(float));
        off[w][8] = total; total = align(total + ifw[w].size() * sizeof(double));
        off[w][9] = total; total = align(total + ifw[w].size() * sizeof(float));
        off[w][10] = total; total = align(total + fwdd[w].size() * sizeof(float));
        off[w][11] = total; total = align(total + bwdd[w].size() * sizeof(float));
        off[w][12] = total; total = align(total + ifwd[w].size() * sizeof(float));
    }
    std::vector<unsigned char> host(total, 0);
    auto put64 = [&](size_t o, const std::vector<double> &v) {
        std::memcpy(&host[o], v.data(), v.size() * sizeof(double));
    };
    auto put32 = [&](size_t o, const std::vector<double> &v) {
        float *d = reinterpret_cast<float *>(&host[o]);
        for (size_t i = 0; i < v.size(); ++i) d[i] = (float)v[i];
    };
    for (int w = 0; w < nops; ++w) {
        put64(off[w][0], rows[w]); put32(off[w][1], rows[w]);
        put64(off[w][2], n1s[w]); put64(off[w][3], red[w]);
        put64(off[w][4], fwd[w]); put32(off[w][5], fwd[w]);
        put64(off[w][6], bwd[w]); put32(off[w][7], bwd[w]);
        put64(off[w][8], ifw[w]); put32(off[w][9], ifw32[w]);
        std::memcpy(&host[off[w][10]], fwdd[w].data(), fwdd[w].size() * sizeof(float));
        std::memcpy(&host[off[w][11]], bwdd[w].data(), bwdd[w].size() * sizeof(float));
        std::memcpy(&host[off[w][12]], ifwd[w].data(), ifwd[w].size() * sizeof(float));
    }
    void *d = nullptr;
    const cudaError_t e = cudaMalloc(&d, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? TDS_ERR_NOMEM : TDS_ERR_CUDA;
    }
    if (cudaMemcpy(d, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        return TDS_ERR_CUDA;
    }
    p->dmem = d;
    unsigned char *base = static_cast<unsigned char *>(d);
    const int R = 2 * p->P;
    double *hm = static_cast<double *>(std::malloc(sizeof(double) * 4 * R));
    if (!hm) { cudaFree(d); p->dmem = nullptr; return TDS_ERR_NOMEM; }
    p->hmem = hm;
    for (int w = 0; w < nops; ++w) {
        DevOp &o = *ops[w];
        if (!o.P) continue;   // segment operator not used
        o.row64 = reinterpret_cast<const double *>(base + off[w][0]);
        o.row32 = reinterpret_cast<const float *>(base + off[w][1]);
        o.n1 = reinterpret_cast<const double *>(base + off[w][2]);
        o.red = reinterpret_cast<const double *>(base + off[w][3]);
        o.fwd64 = reinterpret_cast<const double *>(base + off[w][4]);
        o.fwd32 = reinterpret_cast<const float *>(base + off[w][5]);
        o.bwd64 = reinterpret_cast<const double *>(base + off[w][6]);
        o.bwd32 = reinterpret_cast<const float *>(base + off[w][7]);
        o.ifw64 = reinterpret_cast<const double *>(base + off[w][8]);
        o.ifw32 = reinterpret_cast<const float *>(base + off[w][9]);
        o.fwdd = reinterpret_cast<const float *>(base + off[w][10]);
        o.bwdd = reinterpret_cast<const float *>(base + off[w][11]);
        o.ifwd = reinterpret_cast<const float *>(base + off[w][12]);
    }
    for (int w = 0; w < 2; ++w) {
        p->red_sub_host[w] = hm + (size_t)(2 * w) * R;
        p->red_sup_host[w] = hm + (size_t)(2 * w + 1) * R;
        std::memcpy(p->red_sub_host[w], sub[w].data(), sizeof(double) * R);
        std::memcpy(p->red_sup_host[w], sup[w].data(), sizeof(double) * R);
    }
    // the whole-line Thomas records (tds_deriv_thomas); a zero pivot there only disables that call
    if (!p->band) {
        const tds_status ts = build_thomas(p, L, p->op[0]);
        if (ts == TDS_ERR_NOMEM || ts == TDS_ERR_CUDA) return ts;
    }
    return TDS_OK;
}

} // namespace tds
