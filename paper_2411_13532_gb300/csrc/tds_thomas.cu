// tds_thomas.cu -- the plain Thomas algorithm (Algorithm 1) on whole lines of the interleaved
// layout, the single-rank baseline the paper sets DistD2 against (Table BW): one thread per
// line, the 32 lines of a group in adjacent lanes so that every row access of a warp is one
// coalesced 128/256-byte transaction.
//
//   forward : the stencil right-hand side fused into the elimination, d_j = f_j s_j - f_j a_j
//             d_{j-1} (interior rows with f folded into the taps: one FMA on the recurrence),
//             d_j written to `out`;
//   backward: y_j = d_j - c'_j y_{j+1}, reading d back from `out`, in place;
//   cyclic lines (Sec. 2.1): the two passes run on the Sherman-Morrison matrix A', then a third
//             pass x_j = y_j - ((y_0 + (A[0][n-1] / gamma) y_{n-1}) / (1 + v.z)) z_j with
//             z = A'^{-1} u from the planner.
// `out` carries the forward values, so HBM sees the field read once and `out` written twice and
// read once (cyclic lines: once more each).  FP32 plans run every step in FP32, except where a
// closed line's closure makes its ends ill-conditioned (DevOp::e64: an FP32 rounding at row 1 or
// n-2 reaches the end row multiplied by about 100 for f''_0 + 11 f''_1 = ...): there the four
// rows at each end run both passes in float-pair arithmetic (about 48 bits, on the FP32 pipes) --
// right-hand sides from the exact FP32 inputs with the taps as pairs, forward steps with the
// planner's pair records, forward values kept in registers for the backward steps -- and only
// their final values are rounded to FP32.
#include <cstring>

#include "tds_device.cuh"
#include "tds_df.cuh"

namespace tds {
namespace {

struct ThomasArgs {
    DevOp op;
    const void *rec;   // [n] {f t0 (FP32 symmetric taps: f tapsum), f t1, f t2, f a}
    const void *fc;    // [n] {f, c'}
    const void *z;     // [n] z = A'^{-1} u (cyclic lines), else null
    double ratio, inv_den;
    float end_pf[2 * kEdgeRows][3][2];   // {f, c', f a} of the end rows as pairs (E64)
};

// Interior forms (window w[i] = v[J - 3 + i]), the coefficients folded with f:
//   0 antisymmetric, 1 symmetric (FP64: plain sums; FP32: second differences plus the tap sum),
//   2 pairs about +1/2, 3 pairs about -1/2.
template <typename T, int FORM>
__device__ __forceinline__ T interior(T c0, T c1, T c2, const T (&w)[kTaps]) {
    if constexpr (FORM == 1) {
        if constexpr (sizeof(T) == 8)
            return fma(c0, w[3], fma(c1, w[4] + w[2], c2 * (w[5] + w[1])));
        else
            return fmaf(c0, w[3], fmaf(c1, (w[4] - w[3]) - (w[3] - w[2]), c2 * ((w[5] - w[3]) - (w[3] - w[1]))));
    } else if constexpr (FORM == 2) {
        return c1 * (w[3] + w[4]) + c2 * (w[2] + w[5]);
    } else if constexpr (FORM == 3) {
        return c0 * (w[2] + w[3]) + c1 * (w[1] + w[4]);
    } else {
        return c1 * (w[4] - w[2]) + c2 * (w[5] - w[1]);
    }
}

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// sum_o c_o w_o over the taps of closure row e, c_o as float pairs, w_o floats (exact in a pair)
__device__ __forceinline__ DF edge_sum_pf(const DevOp &op, int e, const float (&w)[kTaps]) {
    float sh = 0.0f, se = 0.0f;
#pragma unroll
    for (int o = 0; o < kTaps; ++o) {
        const float ch = op.edge_pf[e][o][0], cl = op.edge_pf[e][o][1];
        const float p = __fmul_rn(ch, w[o]);
        float err = __fmaf_rn(ch, w[o], -p);
        err = __fmaf_rn(cl, w[o], err);
        const DF t = df_two(sh, p);
        sh = t.h;
        se = __fadd_rn(se, __fadd_rn(t.l, err));
    }
    return df_two(sh, se);
}

__device__ __forceinline__ float df_round(DF x) { return __fadd_rn(x.h, x.l); }

// E64: FP32 sweep of a closed line with the four rows at each end in float pairs (see the header).
template <typename T, int FORM, bool CYC, bool E64>
__global__ void __launch_bounds__(128) k_thomas(const __grid_constant__ ThomasArgs ta, const T *__restrict__ in,
                                                T *__restrict__ out) {
    using T2 = typename Vec2<T>::type;
    const DevOp &op = ta.op;
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= op.nlines) return;
    const int n = op.n;
    const size_t base = (size_t)(l / kSZ) * n * kSZ + (size_t)(l % kSZ);
    const T *src = in + base;
    T *dst = out + base;
    const T2 *rec = static_cast<const T2 *>(ta.rec);   // row j: rec[2j] = {c0, c1}, rec[2j+1] = {c2, g}
    const T2 *fc = static_cast<const T2 *>(ta.fc);

    T w[kTaps];
#pragma unroll
    for (int i = 0; i < kTaps; ++i) {
        const int r = line_row(op, i - 3);
        w[i] = (r >= 0) ? __ldg(src + (size_t)r * kSZ) : T(0);
    }
    auto slide = [&](int j) {
#pragma unroll
        for (int i = 0; i < kTaps - 1; ++i) w[i] = w[i + 1];
        const int r = line_row(op, j + 4);
        w[kTaps - 1] = (r >= 0) ? __ldg(src + (size_t)r * kSZ) : T(0);
    };
    // closure rows of a closed line: the plan's edge taps (generic stencil), then f
    auto edge_row = [&](int j, T d) {
        const T g = __ldg(&rec[2 * j + 1].y);
        const T f = __ldg(&fc[j].x);
        return fma(-g, d, f * stencil<T>(op, j, w));
    };
    // a closure row in pairs: d = f s - (f a) d with the taps on the (exact) inputs; t indexes the
    // end rows' pair records (0..3: rows 0..3, 4..7: rows n-4..n-1)
    auto edge_row_pf = [&](int t, int j, DF d) {
        if constexpr (E64) {
            const int e = (j < kEdgeRows) ? j : kEdgeRows + j - (n - kEdgeRows);
            const DF sum = edge_sum_pf(op, e, w);
            const DF f = df_make(ta.end_pf[t][0][0], ta.end_pf[t][0][1]);
            const DF g = df_make(ta.end_pf[t][2][0], ta.end_pf[t][2][1]);
            return dot2(f, sum, -g, d);
        } else {
            return d;
        }
    };
    auto cprime = [&](int t) { return df_make(ta.end_pf[t][1][0], ta.end_pf[t][1][1]); };
    const int e = CYC ? 0 : kEdgeRows;
    T d = T(0);
    DF dh[E64 ? kEdgeRows : 1], dt[E64 ? kEdgeRows : 1];   // forward values of the end rows
    if constexpr (E64) {
        DF x = df_make(0.0f, 0.0f);
#pragma unroll
        for (int j = 0; j < kEdgeRows; ++j) {
            x = edge_row_pf(j, j, x);
            dh[j] = x;
            slide(j);
        }
        d = df_round(x);
    } else {
        for (int j = 0; j < e; ++j) {
            d = edge_row(j, d);
            dst[(size_t)j * kSZ] = d;
            slide(j);
        }
    }
#pragma unroll 4
    for (int j = e; j < n - e; ++j) {
        const T2 c01 = __ldg(rec + 2 * j), c2g = __ldg(rec + 2 * j + 1);
        d = fma(-c2g.y, d, interior<T, FORM>(c01.x, c01.y, c2g.x, w));
        dst[(size_t)j * kSZ] = d;
        slide(j);
    }
    T y;
    if constexpr (E64) {
        // the last rows: forward in pairs from d_{n-5}, then their backward steps in pairs
        DF x = (n > 2 * kEdgeRows) ? df_make(d, 0.0f) : dh[kEdgeRows - 1];
#pragma unroll
        for (int t = 0; t < kEdgeRows; ++t) {
            x = edge_row_pf(kEdgeRows + t, n - kEdgeRows + t, x);
            dt[t] = x;
            slide(n - kEdgeRows + t);
        }
        dst[(size_t)(n - 1) * kSZ] = df_round(x);
#pragma unroll
        for (int t = kEdgeRows - 2; t >= 0; --t) {
            const int j = n - kEdgeRows + t;
            x = mad(-cprime(kEdgeRows + t), x, dt[t]);
            dst[(size_t)j * kSZ] = df_round(x);
        }
        // interior rows in FP32, in place
        y = df_round(x);
#pragma unroll 4
        for (int j = n - kEdgeRows - 1; j >= kEdgeRows; --j) {
            y = fma(-__ldg(&fc[j].y), y, dst[(size_t)j * kSZ]);
            dst[(size_t)j * kSZ] = y;
        }
        // the first rows in pairs from their forward values in registers
        x = (n > 2 * kEdgeRows) ? df_make(y, 0.0f) : x;
#pragma unroll
        for (int j = kEdgeRows - 1; j >= 0; --j) {
            x = mad(-cprime(j), x, dh[j]);
            dst[(size_t)j * kSZ] = df_round(x);
        }
    } else {
        for (int j = n - e; j < n; ++j) {
            d = edge_row(j, d);
            dst[(size_t)j * kSZ] = d;
            slide(j);
        }
        // backward pass, in place
        y = d;
#pragma unroll 4
        for (int j = n - 2; j >= 0; --j) {
            y = fma(-__ldg(&fc[j].y), y, dst[(size_t)j * kSZ]);
            dst[(size_t)j * kSZ] = y;
        }
    }
    const T ylast = d;
    if constexpr (CYC) {
        const T *z = static_cast<const T *>(ta.z);
        const T fac = (y + T(ta.ratio) * ylast) * T(ta.inv_den);
#pragma unroll 4
        for (int j = 0; j < n; ++j) dst[(size_t)j * kSZ] = fma(-fac, __ldg(z + j), dst[(size_t)j * kSZ]);
    }
}

template <typename T, bool CYC, bool E64>
tds_status launch_form(const ThomasArgs &ta, const void *in, void *out, cudaStream_t st) {
    const unsigned grid = (unsigned)((ta.op.nlines + 127) / 128);
    const T *i = static_cast<const T *>(in);
    T *o = static_cast<T *>(out);
    switch (ta.op.symmetric) {
    case 1:
    case 4: k_thomas<T, 1, CYC, E64><<<grid, 128, 0, st>>>(ta, i, o); break;
    case 2: k_thomas<T, 2, CYC, E64><<<grid, 128, 0, st>>>(ta, i, o); break;
    case 3: k_thomas<T, 3, CYC, E64><<<grid, 128, 0, st>>>(ta, i, o); break;
    default: k_thomas<T, 0, CYC, E64><<<grid, 128, 0, st>>>(ta, i, o); break;
    }
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

} // namespace

tds_status launch_thomas(const tds_plan *p, const void *in, void *out, cudaStream_t st) {
    if (!p->thomas_mem) return TDS_ERR_ARG;
    const bool cyc = (p->bc == TDS_BC_PERIODIC);
    const size_t n = (size_t)p->n, nz = cyc ? n : 0;
    const unsigned char *b = static_cast<const unsigned char *>(p->thomas_mem);
    const size_t off32 = ((n * 6 + nz) * sizeof(double) + 255) & ~(size_t)255;
    ThomasArgs ta;
    ta.op = p->op[0];
    ta.ratio = p->thomas_ratio;
    ta.inv_den = p->thomas_inv_den;
    const double *r64 = reinterpret_cast<const double *>(b);
    std::memcpy(ta.end_pf, p->thomas_end_pf, sizeof(ta.end_pf));
    if (p->dtype == TDS_F64) {
        ta.rec = r64;
        ta.fc = r64 + 4 * n;
        ta.z = cyc ? r64 + 6 * n : nullptr;
        return cyc ? launch_form<double, true, false>(ta, in, out, st) : launch_form<double, false, false>(ta, in, out, st);
    }
    const float *r = reinterpret_cast<const float *>(b + off32);
    ta.rec = r;
    ta.fc = r + 4 * n;
    ta.z = cyc ? r + 6 * n : nullptr;
    if (cyc) return launch_form<float, true, false>(ta, in, out, st);
    // closed lines need at least 2 x 4 rows for the FP64 end rows (the planner's minimum line)
    if (ta.op.e64 && n >= 2 * (size_t)kEdgeRows) return launch_form<float, false, true>(ta, in, out, st);
    return launch_form<float, false, false>(ta, in, out, st);
}

} // namespace tds
