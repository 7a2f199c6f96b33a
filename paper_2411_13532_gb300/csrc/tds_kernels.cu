// tds_kernels.cu -- sm_103a kernels of the DistD2 derivative pipeline (Sec. 4.2).
//
// Thread mapping (Sec. 4.2, last paragraphs): one lane per line, the 32 lines of a group in
// one warp, so every access to a row of the interleaved layout is one coalesced 128/256-byte
// transaction.  A line is cut into P chunks (the paper's ranks); each chunk runs
//   decoupling   (Algorithm 5): stencil right-hand side fused into the modified-Thomas
//                forward pass, then the backward pass;
//   reduced      (communication phase): the 2P chunk-end unknowns of a line, FP64;
//   substitution (Algorithm 6).
//
// Two pipelines:
//   RESIDENT  -- one CTA per group of 32 lines, one warp per chunk.  The group's n x 32 tile
//                is brought into shared memory with TMA bulk copies (one mbarrier per chunk),
//                swept in place, the reduced system is solved by warp 0 from shared memory,
//                and the substituted rows are written straight to global memory: the field is
//                read once and written once.
//   STREAMING -- three kernels through global memory (decouple writes the intermediate to
//                `out` and the chunk ends to the workspace; reduced; substitute in place), for
//                lines whose group does not fit in one CTA's shared memory.
// The adjoint B^T A^{-T} runs the same sweeps on A^T with the identity right-hand side and
// applies the B^T taps after the substitution.
#include <cstdint>

#include "tds_internal.h"

namespace tds {

// Device-side status word: a bounded wait that gives up records TDS_ERR_TIMEOUT here.
__device__ int g_device_status = 0;

namespace {

constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s bound on any wait
constexpr long long kWaitIters = 1ll << 30;

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// TMA bulk copy global -> shared, completion signalled on `bar` (bytes % 16 == 0, both
// addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`: false if it did not complete within kWaitNs.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (long long it = 0; it < kWaitIters; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void record_timeout() { atomicExch(&g_device_status, (int)TDS_ERR_TIMEOUT); }

template <typename T>
__device__ __forceinline__ T rowc(const DevOp &op, int arr, int cls, int j) {
    if constexpr (sizeof(T) == 8)
        return __ldg(op.row64 + ((size_t)arr * op.ncls + cls) * op.m + j);
    else
        return __ldg(op.row32 + ((size_t)arr * op.ncls + cls) * op.m + j);
}

__device__ __forceinline__ int chunk_class(const DevOp &op, int k) {
    return (k == 0) ? op.cls_first : (k == op.P - 1 ? op.cls_last : op.cls_mid);
}

// Stencil of global row J from the window w[i] = v[J - 3 + i] (Eq. cfds and its closures,
// or the transposed taps for the adjoint).
template <typename T>
__device__ __forceinline__ T stencil(const DevOp &op, int J, const T (&w)[kTaps]) {
    if (!op.periodic && (J < kEdgeRows || J >= op.n - kEdgeRows)) {
        const int e = (J < kEdgeRows) ? J : kEdgeRows + J - (op.n - kEdgeRows);
        T s = T(0);
#pragma unroll
        for (int o = 0; o < kTaps; ++o) s += T(op.edge[e][o]) * w[o];
        return s;
    }
    const T t1 = T(op.tap[4]), t2 = T(op.tap[5]);
    if (op.symmetric > 0) return T(op.tap[3]) * w[3] + t1 * (w[4] + w[2]) + t2 * (w[5] + w[1]);
    return t1 * (w[4] - w[2]) + t2 * (w[5] - w[1]);
}

template <typename T>
__device__ __forceinline__ T pick3(int i, T a0, T a1, T a2) {
    return (i == 0) ? a0 : (i == 1 ? a1 : a2);
}

// Row index of the line with cyclic wrap; -1 when outside a closed line.
__device__ __forceinline__ int line_row(const DevOp &op, int J) {
    if (J >= 0 && J < op.n) return J;
    if (!op.periodic) return -1;
    return (J < 0) ? J + op.n : J - op.n;
}

// Reduced chunk-end system of one line, in place in x[i * stride] (i = 0..2P-1), FP64:
// Thomas with the precomputed factorisation, Sherman-Morrison correction if cyclic.
__device__ void reduced_solve(const DevOp &op, double *x, int stride) {
    const int R = 2 * op.P;
    const double *sub = op.red + (size_t)kRedSub * R, *wf = op.red + (size_t)kRedWf * R;
    const double *cp = op.red + (size_t)kRedCp * R, *q = op.red + (size_t)kRedQ * R;
    double y = __ldg(wf) * x[0];
    x[0] = y;
    for (int i = 1; i < R; ++i) {
        y = __ldg(wf + i) * (x[(size_t)i * stride] - __ldg(sub + i) * y);
        x[(size_t)i * stride] = y;
    }
    for (int i = R - 2; i >= 0; --i) {
        y = x[(size_t)i * stride] - __ldg(cp + i) * y;
        x[(size_t)i * stride] = y;
    }
    if (op.red_cyclic) {
        const double beta = (x[0] + op.red_vlast * x[(size_t)(R - 1) * stride]) * op.red_den_inv;
        for (int i = 0; i < R; ++i) x[(size_t)i * stride] -= beta * __ldg(q + i);
    }
}

// ------------------------------------------------------------------------------------------
// RESIDENT pipeline: one CTA per group, warp k = chunk k.
// Shared memory: tile[n][32] (T) | ends[2P][32] (double) | bars[P] (mbarrier).
// ------------------------------------------------------------------------------------------
template <typename T, bool ADJ>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident(const __grid_constant__ DevOp op, const T *__restrict__ in,
                                                   T *__restrict__ out) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int n = op.n, m = op.m, P = op.P;
    const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
    const size_t gofs = (size_t)blockIdx.x * n * kSZ;
    T *tile = reinterpret_cast<T *>(smem);
    double *ends = reinterpret_cast<double *>(smem + (((size_t)n * kSZ * sizeof(T) + 15) & ~(size_t)15));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * kSZ);
    const uint32_t chunk_bytes = (uint32_t)((size_t)m * kSZ * sizeof(T));

    if (threadIdx.x == 0) {
        failed = 0;
        for (int c = 0; c < P; ++c) mbar_init(&bars[c], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < P; ++c) {
            mbar_expect_tx(&bars[c], chunk_bytes);
            bulk_g2s(tile + (size_t)c * m * kSZ, in + gofs + (size_t)c * m * kSZ, chunk_bytes, &bars[c]);
        }
    }
    // this warp's chunk and, for the stencil halo, its neighbours
    bool ok = mbar_wait(&bars[k], 0);
    if (!ADJ) {
        if (k > 0 || op.periodic) ok = mbar_wait(&bars[(k - 1 + P) % P], 0) && ok;
        if (k < P - 1 || op.periodic) ok = mbar_wait(&bars[(k + 1) % P], 0) && ok;
    }
    if (!ok && lane == 0) atomicExch(&failed, 1);

    const int cls = chunk_class(op, k);
    const int J0 = k * m;
    T win[kTaps];
    T halo_after[3];
    if (!ADJ) {
        // halo rows of u before anyone overwrites them
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int rb = line_row(op, J0 - 3 + i);
            win[i] = (ok && rb >= 0) ? tile[(size_t)rb * kSZ + lane] : T(0);
            const int ra = line_row(op, J0 + m + i);
            halo_after[i] = (ok && ra >= 0) ? tile[(size_t)ra * kSZ + lane] : T(0);
        }
    }
    __syncthreads();
    if (failed) {
        // let every bulk copy land before the CTA's shared memory is released
        if (threadIdx.x < P) mbar_wait(&bars[threadIdx.x], 0);
        if (threadIdx.x == 0) record_timeout();
        return;
    }

    // ---- decoupling (Algorithm 5): forward pass with the fused right-hand side ----
    T *row = tile + (size_t)J0 * kSZ + lane;
    T dprev = T(0);
    if (!ADJ) {
#pragma unroll
        for (int i = 3; i < kTaps; ++i) win[i] = row[(size_t)(i - 3) * kSZ];
#pragma unroll 4
        for (int j = 0; j < m; ++j) {
            const T s = stencil<T>(op, J0 + j, win);
            const T d = rowc<T>(op, kF, cls, j) * (s - rowc<T>(op, kR, cls, j) * dprev);
            row[(size_t)j * kSZ] = d;
            dprev = d;
#pragma unroll
            for (int i = 0; i < kTaps - 1; ++i) win[i] = win[i + 1];
            const int jn = j + 4;
            win[kTaps - 1] = (jn < m) ? row[(size_t)jn * kSZ]
                                      : pick3<T>(jn - m, halo_after[0], halo_after[1], halo_after[2]);
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < m; ++j) {
            const T d = rowc<T>(op, kF, cls, j) * (row[(size_t)j * kSZ] - rowc<T>(op, kR, cls, j) * dprev);
            row[(size_t)j * kSZ] = d;
            dprev = d;
        }
    }
    // backward pass j = m-3 .. 1, then row 0 eliminates row 1
    T dnext = row[(size_t)(m - 2) * kSZ];
#pragma unroll 4
    for (int j = m - 3; j >= 1; --j) {
        const T d = row[(size_t)j * kSZ] - rowc<T>(op, kW, cls, j) * dnext;
        row[(size_t)j * kSZ] = d;
        dnext = d;
    }
    const T d0 = T(__ldg(op.n1 + cls)) * (row[0] - rowc<T>(op, kW, cls, 0) * dnext);
    row[0] = d0;
    ends[(size_t)(2 * k) * kSZ + lane] = double(d0);
    ends[(size_t)(2 * k + 1) * kSZ + lane] = double(row[(size_t)(m - 1) * kSZ]);
    __syncthreads();

    // ---- reduced chunk-end system, FP64, one lane per line ----
    if (k == 0) reduced_solve(op, ends + lane, kSZ);
    __syncthreads();

    // ---- substitution (Algorithm 6) ----
    const double F64 = ends[(size_t)(2 * k) * kSZ + lane];
    const double L64 = ends[(size_t)(2 * k + 1) * kSZ + lane];
    const T F = T(F64), L = T(L64);
    T *orow = out + gofs + (size_t)J0 * kSZ + lane;
    if (!ADJ) {
        orow[0] = F;
#pragma unroll 4
        for (int j = 1; j < m - 1; ++j)
            orow[(size_t)j * kSZ] = row[(size_t)j * kSZ] - rowc<T>(op, kSA, cls, j) * F - rowc<T>(op, kSC, cls, j) * L;
        orow[(size_t)(m - 1) * kSZ] = L;
        return;
    }
    // adjoint: y in place, then x = B^T y with a rolling window over this chunk
    row[0] = F;
#pragma unroll 4
    for (int j = 1; j < m - 1; ++j)
        row[(size_t)j * kSZ] = row[(size_t)j * kSZ] - rowc<T>(op, kSA, cls, j) * F - rowc<T>(op, kSC, cls, j) * L;
    row[(size_t)(m - 1) * kSZ] = L;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kTaps; ++i) {
        const int r = line_row(op, J0 - 3 + i);
        win[i] = (r >= 0) ? tile[(size_t)r * kSZ + lane] : T(0);
    }
#pragma unroll 4
    for (int j = 0; j < m; ++j) {
        orow[(size_t)j * kSZ] = stencil<T>(op, J0 + j, win);
#pragma unroll
        for (int i = 0; i < kTaps - 1; ++i) win[i] = win[i + 1];
        const int r = line_row(op, J0 + j + 4);
        win[kTaps - 1] = (r >= 0) ? tile[(size_t)r * kSZ + lane] : T(0);
    }
}

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
    if (!ADJ) {
        T win[kTaps];
#pragma unroll
        for (int i = 0; i < kTaps; ++i) {
            const int r = line_row(op, J0 - 3 + i);
            win[i] = (r >= 0) ? __ldg(src + (size_t)r * kSZ) : T(0);
        }
#pragma unroll 4
        for (int j = 0; j < m; ++j) {
            const T s = stencil<T>(op, J0 + j, win);
            const T d = rowc<T>(op, kF, cls, j) * (s - rowc<T>(op, kR, cls, j) * dprev);
            row[(size_t)j * kSZ] = d;
            dprev = d;
#pragma unroll
            for (int i = 0; i < kTaps - 1; ++i) win[i] = win[i + 1];
            const int r = line_row(op, J0 + j + 4);
            win[kTaps - 1] = (r >= 0) ? __ldg(src + (size_t)r * kSZ) : T(0);
        }
    } else {
        const T *gsrc = src + (size_t)J0 * kSZ;
#pragma unroll 4
        for (int j = 0; j < m; ++j) {
            const T d = rowc<T>(op, kF, cls, j) * (__ldg(gsrc + (size_t)j * kSZ) - rowc<T>(op, kR, cls, j) * dprev);
            row[(size_t)j * kSZ] = d;
            dprev = d;
        }
    }
    T dnext = row[(size_t)(m - 2) * kSZ];
#pragma unroll 4
    for (int j = m - 3; j >= 1; --j) {
        const T d = row[(size_t)j * kSZ] - rowc<T>(op, kW, cls, j) * dnext;
        row[(size_t)j * kSZ] = d;
        dnext = d;
    }
    const T d0 = T(__ldg(op.n1 + cls)) * (row[0] - rowc<T>(op, kW, cls, 0) * dnext);
    row[0] = d0;
    double *e = ends + ((size_t)gw * 2) * kSZ + lane;
    e[0] = double(d0);
    e[kSZ] = double(row[(size_t)(m - 1) * kSZ]);
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
#pragma unroll 2
    for (int j = 0; j < m; ++j) {
        const T x = stencil<T>(op, J0 + j, win);
#pragma unroll
        for (int i = 0; i < kTaps - 1; ++i) win[i] = win[i + 1];
        win[kTaps - 1] = adj_y<T>(op, g, J0, J0 + j + 4, own, ends, halo);
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

template <typename T, bool ADJ>
tds_status launch_resident_t(const DevOp &op, const void *in, void *out, int smem, cudaStream_t st) {
    auto kern = k_resident<T, ADJ>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    kern<<<op.ngroups, op.P * 32, smem, st>>>(op, static_cast<const T *>(in), static_cast<T *>(out));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

template <typename T, bool ADJ>
tds_status launch_streaming_t(const DevOp &op, const void *in, void *out, void *ws, cudaStream_t st) {
    double *ends = static_cast<double *>(ws);
    T *halo = reinterpret_cast<T *>(ends + (size_t)op.nlines * op.P * 2);
    const long long warps = (long long)op.ngroups * op.P;
    const unsigned blocks = (unsigned)((warps + kStreamWarps - 1) / kStreamWarps);
    k_decouple<T, ADJ><<<blocks, kStreamWarps * 32, 0, st>>>(op, static_cast<const T *>(in),
                                                            static_cast<T *>(out), ends, halo);
    k_reduced<<<(unsigned)((op.nlines + 127) / 128), 128, 0, st>>>(op, ends);
    if (!ADJ) k_substitute<T><<<blocks, kStreamWarps * 32, 0, st>>>(op, static_cast<T *>(out), ends);
    else k_subst_bt<T><<<blocks, kStreamWarps * 32, 0, st>>>(op, static_cast<T *>(out), ends, halo);
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

} // namespace

size_t resident_smem_bytes(int n, int P, tds_dtype dtype) {
    const size_t es = (dtype == TDS_F64) ? 8 : 4;
    return (((size_t)n * kSZ * es + 15) & ~(size_t)15) + (size_t)2 * P * kSZ * 8 + (size_t)P * 8;
}

tds_status launch_resident(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    const DevOp &op = p->op[which];
    if (p->dtype == TDS_F64)
        return which ? launch_resident_t<double, true>(op, in, out, p->resident_smem, st)
                     : launch_resident_t<double, false>(op, in, out, p->resident_smem, st);
    return which ? launch_resident_t<float, true>(op, in, out, p->resident_smem, st)
                 : launch_resident_t<float, false>(op, in, out, p->resident_smem, st);
}

size_t streaming_ws_bytes(const tds_plan *p) {
    const size_t es = (p->dtype == TDS_F64) ? 8 : 4;
    const size_t units = (size_t)p->nlines * p->P;
    return (units * 2 * 8 + units * 6 * es + 255) & ~(size_t)255;
}

tds_status launch_streaming(const tds_plan *p, int which, const void *in, void *out, void *ws,
                            cudaStream_t st) {
    const DevOp &op = p->op[which];
    if (p->dtype == TDS_F64)
        return which ? launch_streaming_t<double, true>(op, in, out, ws, st)
                     : launch_streaming_t<double, false>(op, in, out, ws, st);
    return which ? launch_streaming_t<float, true>(op, in, out, ws, st)
                 : launch_streaming_t<float, false>(op, in, out, ws, st);
}

tds_status launch_reduced_only(const tds_plan *p, const double *rhs, double *x, cudaStream_t st) {
    const DevOp &op = p->op[0];
    k_reduced_lines<<<(unsigned)((op.nlines + 127) / 128), 128, 0, st>>>(op, rhs, x);
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

tds_status read_device_status() {
    int v = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return TDS_ERR_CUDA;
    if (cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int)) != cudaSuccess) return TDS_ERR_CUDA;
    if (cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int)) != cudaSuccess) return TDS_ERR_CUDA;
    return (tds_status)v;
}

} // namespace tds
