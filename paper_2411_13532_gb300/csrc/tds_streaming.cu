// tds_streaming.cu -- the three-kernel DistD2 pipeline through global memory (Sec. 4.2), for
// lines no resident CTA can hold and segments cannot split (or P x 8 > 512): decoupling
// (Algorithm 5) writes the intermediate to `out` and the chunk ends to the workspace, the
// reduced chunk-end system is solved one thread per line in FP64, and the substitution
// (Algorithm 6) finishes `out` in place.  This is the paper's own phase order (backward pass
// then substitution); the resident kernels fuse them.  One lane per line, one warp per
// (group, chunk), so every row access is one coalesced 128/256-byte transaction.
#include "tds_device.cuh"

namespace tds {
namespace {

// ------------------------------------------------------------------------------------------
// STREAMING pipeline.  Workspace: ends[G][P][2][32] (double), then for the adjoint the
// decoupled values of the first and last 3 rows of every chunk, halo[G][P][6][32] (T).
// ------------------------------------------------------------------------------------------
constexpr int kStreamWarps = 4;

template <typename T, bool ADJ>
__global__ void __launch_bounds__(kStreamWarps * 32) k_decouple(const __grid_constant__ DevOp op, const T *__restrict__ in,
                                                                T *__restrict__ out,
                                                                double *__restrict__ ends,
                                                                T *__restrict__ halo) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kStreamWarps + (threadIdx.x >> 5);
    if (gw >= (long long)op.ngroups * op.P) return;
    const int g = (int)(gw / op.P), k = (int)(gw % op.P);
    const int n = op.n, m = op.m, cls = chunk_class(op, k), J0 = k * m;
    const T *src = in + (size_t)g * n * kSZ + lane;
    T *row = out + (size_t)g * n * kSZ + (size_t)J0 * kSZ + lane;
    T dprev = T(0);
    // FP32 sweeps of closed lines take the four rows at each end of the line in FP64: the
    // closure makes the chunk ends ill-conditioned (an error at row 1 reaches row 0 multiplied
    // by about 100 for the second derivative); h64 keeps the first chunk's forward values of
    // rows 0..3, xl the last chunk's d_{m-1}
    const bool e64 = sizeof(T) == 4 && op.e64;
    const bool head = e64 && k == 0, tail = e64 && k == op.P - 1;
    double h64[4] = {0.0, 0.0, 0.0, 0.0}, d64 = 0.0;
    auto step64 = [&](int j, double s) {
        d64 = rowc<double>(op, kF, cls, j) * (s - rowc<double>(op, kR, cls, j) * d64);
        if (j < 4) h64[j] = d64;
        dprev = T(d64);
        row[(size_t)j * kSZ] = dprev;
    };
    const int ja = head ? 4 : 0, jz = tail ? m - 4 : m;
    if (!ADJ) {
        T win[kTaps];
#pragma unroll
        for (int i = 0; i < kTaps; ++i) {
            const int r = line_row(op, J0 - 3 + i);
            win[i] = (r >= 0) ? __ldg(src + (size_t)r * kSZ) : T(0);
        }
        auto slide = [&](int j) {
#pragma unroll
            for (int i = 0; i < kTaps - 1; ++i) win[i] = win[i + 1];
            const int r = line_row(op, J0 + j + 4);
            win[kTaps - 1] = (r >= 0) ? __ldg(src + (size_t)r * kSZ) : T(0);
        };
        auto rows64 = [&](int jb) {
            for (int j = jb; j < jb + 4; ++j) {
                const int J = J0 + j, e = (J < kEdgeRows) ? J : kEdgeRows + J - (n - kEdgeRows);
                double s = 0.0;
#pragma unroll
                for (int o = 0; o < kTaps; ++o) s = ::fma(op.edge[e][o], (double)win[o], s);
                step64(j, s);
                slide(j);
            }
        };
        if (head) rows64(0);
#pragma unroll 4
        for (int j = ja; j < jz; ++j) {
            const T s = stencil<T>(op, J0 + j, win);
            const T d = rowc<T>(op, kF, cls, j) * (s - rowc<T>(op, kR, cls, j) * dprev);
            row[(size_t)j * kSZ] = d;
            dprev = d;
            slide(j);
        }
        if (tail) {
            d64 = (double)dprev;
            rows64(m - 4);
        }
    } else {
        const T *gsrc = src + (size_t)J0 * kSZ;
        if (head)
            for (int j = 0; j < 4; ++j) step64(j, (double)__ldg(gsrc + (size_t)j * kSZ));
#pragma unroll 4
        for (int j = ja; j < jz; ++j) {
            const T d = rowc<T>(op, kF, cls, j) * (__ldg(gsrc + (size_t)j * kSZ) - rowc<T>(op, kR, cls, j) * dprev);
            row[(size_t)j * kSZ] = d;
            dprev = d;
        }
        if (tail) {
            d64 = (double)dprev;
            for (int j = m - 4; j < m; ++j) step64(j, (double)__ldg(gsrc + (size_t)j * kSZ));
        }
    }
    const double xl = d64;
    const int jlo = head ? 4 : 1;
    T dnext = row[(size_t)(m - 2) * kSZ];
#pragma unroll 4
    for (int j = m - 3; j >= jlo; --j) {
        const T d = row[(size_t)j * kSZ] - rowc<T>(op, kW, cls, j) * dnext;
        row[(size_t)j * kSZ] = d;
        dnext = d;
    }
    double *e = ends + ((size_t)gw * 2) * kSZ + lane;
    if (head) {
        // rows min(3, m-3)..1 of the backward pass and row 0 in FP64
        double dn = (m - 2 >= 4) ? (double)dnext : h64[m - 2];
        for (int j = (m - 3 < 3 ? m - 3 : 3); j >= 1; --j) {
            dn = h64[j] - rowc<double>(op, kW, cls, j) * dn;
            row[(size_t)j * kSZ] = T(dn);
        }
        const double d0 = __ldg(op.n1 + cls) * (h64[0] - rowc<double>(op, kW, cls, 0) * dn);
        row[0] = T(d0);
        e[0] = d0;
    } else {
        const T d0 = T(__ldg(op.n1 + cls)) * (row[0] - rowc<T>(op, kW, cls, 0) * dnext);
        row[0] = d0;
        e[0] = double(d0);
    }
    e[kSZ] = tail ? xl : double(row[(size_t)(m - 1) * kSZ]);
    if (ADJ) {
        T *hl = halo + (size_t)gw * 6 * kSZ + lane;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            hl[(size_t)i * kSZ] = row[(size_t)i * kSZ];
            hl[(size_t)(3 + i) * kSZ] = row[(size_t)(m - 3 + i) * kSZ];
        }
    }
}

__global__ void k_reduced(const __grid_constant__ DevOp op, double *__restrict__ ends) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= op.nlines) return;
    const long long g = l / kSZ;
    const int s = (int)(l % kSZ);
    // ends[g][k][e][s]: unknown i = 2k + e sits at stride 32
    reduced_solve(op, ends + (size_t)g * op.P * 2 * kSZ + s, kSZ);
}

template <typename T>
__global__ void __launch_bounds__(kStreamWarps * 32) k_substitute(const __grid_constant__ DevOp op, T *__restrict__ out,
                                                                  const double *__restrict__ ends) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kStreamWarps + (threadIdx.x >> 5);
    if (gw >= (long long)op.ngroups * op.P) return;
    const int g = (int)(gw / op.P), k = (int)(gw % op.P);
    const int m = op.m, cls = chunk_class(op, k);
    const T F = T(ends[((size_t)gw * 2) * kSZ + lane]);
    const T L = T(ends[((size_t)gw * 2 + 1) * kSZ + lane]);
    T *row = out + (size_t)g * op.n * kSZ + (size_t)k * m * kSZ + lane;
    row[0] = F;
#pragma unroll 4
    for (int j = 1; j < m - 1; ++j)
        row[(size_t)j * kSZ] = row[(size_t)j * kSZ] - rowc<T>(op, kSA, cls, j) * F - rowc<T>(op, kSC, cls, j) * L;
    row[(size_t)(m - 1) * kSZ] = L;
}

// Adjoint: substitution fused with the B^T taps.  y at any row is recomputed on the fly from
// the decoupled value (own rows from `out`, neighbour rows from the halo workspace) and the
// owning chunk's F, L; x = B^T y overwrites this chunk's rows of `out` behind the window.
template <typename T>
__device__ __forceinline__ T adj_y(const DevOp &op, int g, int J0, int J, const T *own,
                                   const double *ends, const T *halo) {
    const int r = line_row(op, J);
    if (r < 0) return T(0);
    const int m = op.m, kk = r / m, jj = r - kk * m;
    const size_t gk = (size_t)g * op.P + kk;
    const int lane = threadIdx.x & 31;
    const T F = T(ends[(gk * 2) * kSZ + lane]), L = T(ends[(gk * 2 + 1) * kSZ + lane]);
    if (jj == 0) return F;
    if (jj == m - 1) return L;
    T d;
    // rows of this warp's own chunk range are read from `out` (not yet overwritten, they are
    // ahead of the window); every other row -- including a wrapped row of the same chunk when
    // P = 1 -- comes from the halo copy, because `out` there may already hold x
    if (J >= J0 && J < J0 + m) d = own[(size_t)(J - J0) * kSZ];
    else d = halo[(gk * 6 + (jj < 3 ? jj : 3 + jj - (m - 3))) * kSZ + lane];
    const int cls = chunk_class(op, kk);
    return d - rowc<T>(op, kSA, cls, jj) * F - rowc<T>(op, kSC, cls, jj) * L;
}

template <typename T>
__global__ void __launch_bounds__(kStreamWarps * 32) k_subst_bt(const __grid_constant__ DevOp op, T *__restrict__ out,
                                                                const double *__restrict__ ends,
                                                                const T *__restrict__ halo) {
    const int lane = threadIdx.x & 31;
    const long long gw = (long long)blockIdx.x * kStreamWarps + (threadIdx.x >> 5);
    if (gw >= (long long)op.ngroups * op.P) return;
    const int g = (int)(gw / op.P), k = (int)(gw % op.P);
    const int m = op.m, J0 = k * m;
    T *own = out + (size_t)g * op.n * kSZ + (size_t)J0 * kSZ + lane;
    T win[kTaps];
#pragma unroll
    for (int i = 0; i < kTaps; ++i) win[i] = adj_y<T>(op, g, J0, J0 - 3 + i, own, ends, halo);
    // the window never needs the next chunk's row 3: the halo holds only rows 0..2 and m-3..m-1
    // of each chunk, so the shift after the last row is skipped rather than loaded
#pragma unroll 2
    for (int j = 0; j < m; ++j) {
        const T x = stencil<T>(op, J0 + j, win);
        if (j + 1 < m) {
#pragma unroll
            for (int i = 0; i < kTaps - 1; ++i) win[i] = win[i + 1];
            win[kTaps - 1] = adj_y<T>(op, g, J0, J0 + j + 4, own, ends, halo);
        }
        own[(size_t)j * kSZ] = x;
    }
}

__global__ void k_reduced_lines(const __grid_constant__ DevOp op, const double *__restrict__ rhs, double *__restrict__ x) {
    const long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= op.nlines) return;
    const int R = 2 * op.P;
    double *xl = x + (size_t)l * R;
    for (int i = 0; i < R; ++i) xl[i] = rhs[(size_t)l * R + i];
    reduced_solve(op, xl, 1);
}

// MODE: 0 stencil right-hand side; 1 identity right-hand side then B^T (adjoint on closed
// lines); 2 identity right-hand side only (the solve alone).
template <typename T, int MODE>
tds_status launch_streaming_t(const DevOp &op, const void *in, void *out, void *ws, cudaStream_t st) {
    double *ends = static_cast<double *>(ws);
    T *halo = reinterpret_cast<T *>(ends + (size_t)op.nlines * op.P * 2);
    const long long warps = (long long)op.ngroups * op.P;
    const unsigned blocks = (unsigned)((warps + kStreamWarps - 1) / kStreamWarps);
    k_decouple<T, MODE != 0><<<blocks, kStreamWarps * 32, 0, st>>>(op, static_cast<const T *>(in),
                                                                   static_cast<T *>(out), ends, halo);
    k_reduced<<<(unsigned)((op.nlines + 127) / 128), 128, 0, st>>>(op, ends);
    if (MODE != 1) k_substitute<T><<<blocks, kStreamWarps * 32, 0, st>>>(op, static_cast<T *>(out), ends);
    else k_subst_bt<T><<<blocks, kStreamWarps * 32, 0, st>>>(op, static_cast<T *>(out), ends, halo);
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

} // namespace

size_t streaming_ws_bytes(const tds_plan *p) {
    const size_t es = (p->dtype == TDS_F64) ? 8 : 4;
    const size_t units = (size_t)p->nlines * p->P;
    return (units * 2 * 8 + units * 6 * es + 255) & ~(size_t)255;
}

tds_status launch_streaming(const tds_plan *p, int which, const void *in, void *out, void *ws,
                            cudaStream_t st) {
    const DevOp &op = p->op[which];
    if (p->dtype == TDS_F64)
        return op.adjoint == 2 ? launch_streaming_t<double, 2>(op, in, out, ws, st)
             : op.adjoint == 1 ? launch_streaming_t<double, 1>(op, in, out, ws, st)
                               : launch_streaming_t<double, 0>(op, in, out, ws, st);
    return op.adjoint == 2 ? launch_streaming_t<float, 2>(op, in, out, ws, st)
         : op.adjoint == 1 ? launch_streaming_t<float, 1>(op, in, out, ws, st)
                           : launch_streaming_t<float, 0>(op, in, out, ws, st);
}

tds_status launch_reduced_only(const tds_plan *p, const double *rhs, double *x, cudaStream_t st) {
    const DevOp &op = p->op[0];
    k_reduced_lines<<<(unsigned)((op.nlines + 127) / 128), 128, 0, st>>>(op, rhs, x);
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

} // namespace tds
