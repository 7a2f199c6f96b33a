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
// rows at each end run both passes in FP64 -- right-hand sides from the exact FP32 inputs with
// the taps as written, forward steps with the FP64 records, forward values kept in registers for
// the backward steps -- and only their final values are rounded to FP32.
#include "tds_device.cuh"

namespace tds {
namespace {

struct ThomasArgs {
    DevOp op;
    const void *rec;   // [n] {f t0 (FP32 symmetric taps: f tapsum), f t1, f t2, f a}
    const void *fc;    // [n] {f, c'}
    const void *z;     // [n] z = A'^{-1} u (cyclic lines), else null
    const double *rec64, *fc64;   // the FP64 records (the FP64 end rows of FP32 sweeps)
    double ratio, inv_den;
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

// E64: FP32 sweep of a closed line with the four rows at each end in FP64 (see the header).
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
    // a closure row in FP64: the taps as written on the (exact) inputs, then the FP64 records
    auto edge_row64 = [&](int j, double d) {
        const int e = (j < kEdgeRows) ? j : kEdgeRows + j - (n - kEdgeRows);
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int o = 0; o < kTaps; o += 2) {
            s0 = ::fma(op.edge[e][o], (double)w[o], s0);
            if (o + 1 < kTaps) s1 = ::fma(op.edge[e][o + 1], (double)w[o + 1], s1);
        }
        return ::fma(-__ldg(ta.rec64 + 4 * j + 3), d, __ldg(ta.fc64 + 2 * j) * (s0 + s1));
    };
    const int e = CYC ? 0 : kEdgeRows;
    T d = T(0);
    double dh[E64 ? kEdgeRows : 1], dt[E64 ? kEdgeRows : 1];   // FP64 forward values of the end rows
    if constexpr (E64) {
        double x = 0.0;
#pragma unroll
        for (int j = 0; j < kEdgeRows; ++j) {
            x = edge_row64(j, x);
            dh[j] = x;
            slide(j);
        }
        d = T(x);
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
        // the last rows: forward in FP64 from d_{n-5}, then their backward steps in FP64
        double x = (n > 2 * kEdgeRows) ? (double)d : dh[kEdgeRows - 1];
#pragma unroll
        for (int t = 0; t < kEdgeRows; ++t) {
            x = edge_row64(n - kEdgeRows + t, x);
            dt[t] = x;
            slide(n - kEdgeRows + t);
        }
        dst[(size_t)(n - 1) * kSZ] = T(x);
#pragma unroll
        for (int t = kEdgeRows - 2; t >= 0; --t) {
            const int j = n - kEdgeRows + t;
            x = ::fma(-__ldg(ta.fc64 + 2 * j + 1), x, dt[t]);
            dst[(size_t)j * kSZ] = T(x);
        }
        // interior rows in FP32, in place
        y = T(x);
#pragma unroll 4
        for (int j = n - kEdgeRows - 1; j >= kEdgeRows; --j) {
            y = fma(-__ldg(&fc[j].y), y, dst[(size_t)j * kSZ]);
            dst[(size_t)j * kSZ] = y;
        }
        // the first rows in FP64 from their forward values in registers
        x = (n > 2 * kEdgeRows) ? (double)y : x;
#pragma unroll
        for (int j = kEdgeRows - 1; j >= 0; --j) {
            x = ::fma(-__ldg(ta.fc64 + 2 * j + 1), x, dh[j]);
            dst[(size_t)j * kSZ] = T(x);
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
    ta.rec64 = r64;
    ta.fc64 = r64 + 4 * n;
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
