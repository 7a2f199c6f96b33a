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

// TMA bulk copy shared -> global (bytes % 16 == 0, 16-byte aligned), tracked by bulk groups.
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
                 ::"l"(dst), "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Wait until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
// RESIDENT pipeline: one CTA holds a whole group of 32 lines.  Chunk k is swept by 32/V
// threads; each thread carries V adjacent lines (one 16-byte vector of a row for FP32 V=4),
// which gives V independent recurrences per thread and spreads the per-row work (plan
// coefficients, addressing, loop control) over V points.
// ------------------------------------------------------------------------------------------
template <typename T, int V>
struct Pack {
    T v[V];
};

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ldv(const T *p) {
    Pack<T, V> r;
    if constexpr (V == 1) {
        r.v[0] = *p;
    } else if constexpr (sizeof(T) * V == 16 && sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
    } else if constexpr (sizeof(T) * V == 16 && sizeof(T) == 8) {
        const double2 x = *reinterpret_cast<const double2 *>(p);
        r.v[0] = x.x; r.v[1] = x.y;
    } else {
        const float2 x = *reinterpret_cast<const float2 *>(p);
        r.v[0] = x.x; r.v[1] = x.y;
    }
    return r;
}

template <typename T, int V>
__device__ __forceinline__ void stv(T *p, const Pack<T, V> &r) {
    if constexpr (V == 1) {
        *p = r.v[0];
    } else if constexpr (sizeof(T) * V == 16 && sizeof(T) == 4) {
        *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else if constexpr (sizeof(T) * V == 16 && sizeof(T) == 8) {
        *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
    } else {
        *reinterpret_cast<float2 *>(p) = make_float2(r.v[0], r.v[1]);
    }
}

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> zero_pack() {
    Pack<T, V> r;
#pragma unroll
    for (int i = 0; i < V; ++i) r.v[i] = T(0);
    return r;
}

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> pick3v(int i, const Pack<T, V> &a0, const Pack<T, V> &a1,
                                             const Pack<T, V> &a2) {
    return (i == 0) ? a0 : (i == 1 ? a1 : a2);
}

// Whether the resident kernels store a finished tile with one TMA bulk copy (FP32, where the
// sweep is HBM-bound) or each thread stores its rows directly (FP64, where the sweep is bound by
// the FP64 pipe and the direct stores overlap it).
template <typename T>
constexpr bool kBulkStore = (sizeof(T) == 4);

// Plan row records of the resident sweep (see DevOp::fwd64 / bwd64).
template <typename T>
struct FwdRec {
    T f, r, pi;
};

template <typename T>
__device__ __forceinline__ FwdRec<T> ld_fwd(const DevOp &op, int cls, int j) {
    const size_t i = (size_t)cls * op.m + j;
    if constexpr (sizeof(T) == 4) {
        const float4 x = __ldg(reinterpret_cast<const float4 *>(op.fwd32) + i);
        return {x.x, x.y, x.z};
    } else {
        const double2 x = __ldg(reinterpret_cast<const double2 *>(op.fwd64) + 2 * i);
        return {x.x, x.y, __ldg(op.fwd64 + 4 * i + 2)};
    }
}

template <typename T>
__device__ __forceinline__ void ld_bwd(const DevOp &op, int cls, int j, T &sa, T &sc) {
    const size_t i = (size_t)cls * op.m + j;
    if constexpr (sizeof(T) == 4) {
        const float2 x = __ldg(reinterpret_cast<const float2 *>(op.bwd32) + i);
        sa = x.x; sc = x.y;
    } else {
        const double2 x = __ldg(reinterpret_cast<const double2 *>(op.bwd64) + i);
        sa = x.x; sc = x.y;
    }
}

// Interior stencil (offsets -2..2) of V lines from the window w[i] = v[J - 2 + i].
template <typename T, int V, bool SYM>
__device__ __forceinline__ void istencil(T t0, T t1, T t2, const Pack<T, V> (&w)[5], T (&s)[V]) {
#pragma unroll
    for (int i = 0; i < V; ++i) {
        if (SYM) s[i] = t0 * w[2].v[i] + t1 * (w[3].v[i] + w[1].v[i]) + t2 * (w[4].v[i] + w[0].v[i]);
        else s[i] = t1 * (w[3].v[i] - w[1].v[i]) + t2 * (w[4].v[i] - w[0].v[i]);
    }
}

// Closure-row stencil (offsets -3..3, closed lines only) from w[i] = v[J - 3 + i]; e indexes
// the plan's edge rows (0..3 = rows 0..3, 4..7 = rows n-4..n-1).
template <typename T, int V>
__device__ __forceinline__ void estencil(const DevOp &op, int e, const Pack<T, V> (&w)[kTaps], T (&s)[V]) {
#pragma unroll
    for (int i = 0; i < V; ++i) s[i] = T(0);
#pragma unroll
    for (int o = 0; o < kTaps; ++o) {
        const T c = T(op.edge[e][o]);
#pragma unroll
        for (int i = 0; i < V; ++i) s[i] += c * w[o].v[i];
    }
}

template <typename T, int V>
__device__ __forceinline__ Pack<T, V> ld_row(const DevOp &op, const T *tile, int J, int c) {
    const int r = line_row(op, J);
    return (r >= 0) ? ldv<T, V>(tile + (size_t)r * kSZ + c) : zero_pack<T, V>();
}

// Before the sweep (and before the CTA barrier that lets any thread overwrite the tile): the
// stencil halo of this chunk (2 rows before, 2 after) into registers, and on closed lines the
// first and last 7 rows of the line into the scratch rows xs[0..6], xs[7..13] (the closure
// rows reach 3 points in, and the sweep overwrites the tile in place).
template <typename T, int V>
__device__ __forceinline__ void read_halo(const DevOp &op, const T *tile, T *xs, int k, int c,
                                          Pack<T, V> (&hb)[2], Pack<T, V> (&ha)[2]) {
    const int J0 = k * op.m;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        hb[i] = ld_row<T, V>(op, tile, J0 - 2 + i, c);
        ha[i] = ld_row<T, V>(op, tile, J0 + op.m + i, c);
    }
    if (!op.periodic) {
        if (k == 0)
            for (int i = 0; i < kTaps; ++i) stv<T, V>(xs + (size_t)i * kSZ + c, ld_row<T, V>(op, tile, i, c));
        if (k == op.P - 1)
            for (int i = 0; i < kTaps; ++i)
                stv<T, V>(xs + (size_t)(kTaps + i) * kSZ + c, ld_row<T, V>(op, tile, op.n - kTaps + i, c));
    }
}

// Forward pass over rows [jb, je) of the chunk with the interior stencil: d_j = f_j (s_j -
// r_j d_{j-1}), S += pi_j d_j, d_j written over the tile row.  w[0..3] holds v[j-2..j+1] on
// entry; v[j+2] comes from the tile while inside the chunk, then from the halo after it.
template <typename T, int V, bool SYM>
__device__ __forceinline__ void fwd_interior(const DevOp &op, int cls, T *row, int jb, int je,
                                             Pack<T, V> (&w)[5], const Pack<T, V> (&ha)[2],
                                             Pack<T, V> &dprev, Pack<T, V> &S) {
    const int m = op.m;
    const T t0 = T(op.tap[3]), t1 = T(op.tap[4]), t2 = T(op.tap[5]);
    const int jm = (je < m - 2) ? je : m - 2;
    if (jb < jm) {
        // one row ahead: the next tile row and plan record are in flight during this row
        Pack<T, V> wn = ldv<T, V>(row + (size_t)(jb + 2) * kSZ);
        FwdRec<T> qn = ld_fwd<T>(op, cls, jb);
#pragma unroll 4
        for (int j = jb; j < jm; ++j) {
            w[4] = wn;
            const FwdRec<T> q = qn;
            const int jn = (j + 1 < jm) ? j + 1 : j;
            wn = ldv<T, V>(row + (size_t)(jn + 2) * kSZ);
            qn = ld_fwd<T>(op, cls, jn);
            T sv[V];
            istencil<T, V, SYM>(t0, t1, t2, w, sv);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                dprev.v[i] = q.f * (sv[i] - q.r * dprev.v[i]);
                S.v[i] = fma(q.pi, dprev.v[i], S.v[i]);
            }
            stv<T, V>(row + (size_t)j * kSZ, dprev);
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
        }
    }
    for (int j = (jb > m - 2 ? jb : m - 2); j < je; ++j) {
        w[4] = (j + 2 - m == 0) ? ha[0] : ha[1];
        T sv[V];
        istencil<T, V, SYM>(t0, t1, t2, w, sv);
        const FwdRec<T> q = ld_fwd<T>(op, cls, j);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            dprev.v[i] = q.f * (sv[i] - q.r * dprev.v[i]);
            S.v[i] = fma(q.pi, dprev.v[i], S.v[i]);
        }
        stv<T, V>(row + (size_t)j * kSZ, dprev);
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
    }
}

// Closure rows of the forward pass: local rows j0..j0+3 whose 7-point windows are the scratch
// rows x[t + o] (t = 0..3, o = 0..6) with x[i] = v[Jx + i]; entries outside the line are zero.
template <typename T, int V>
__device__ __forceinline__ void fwd_edge(const DevOp &op, int cls, T *row, int j0, int e0,
                                         const T *xs, int c, int xlo, int xhi,
                                         Pack<T, V> &dprev, Pack<T, V> &S) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        Pack<T, V> w7[kTaps];
#pragma unroll
        for (int o = 0; o < kTaps; ++o) {
            const int x = t + o + xlo;   // scratch index, valid in [0, xhi)
            w7[o] = (x >= 0 && x < xhi) ? ldv<T, V>(xs + (size_t)x * kSZ + c) : zero_pack<T, V>();
        }
        T sv[V];
        estencil<T, V>(op, e0 + t, w7, sv);
        const int j = j0 + t;
        const FwdRec<T> q = ld_fwd<T>(op, cls, j);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            dprev.v[i] = q.f * (sv[i] - q.r * dprev.v[i]);
            S.v[i] = fma(q.pi, dprev.v[i], S.v[i]);
        }
        stv<T, V>(row + (size_t)j * kSZ, dprev);
    }
}

// In-place x = B^T y over rows [jb, je) of this chunk with the interior taps: w[0..3] holds
// y[j-2..j+1] on entry; y[j+2] comes from the tile while inside the chunk (rows ahead of the
// window are not yet overwritten), then from the halo after it.
template <typename T, int V, bool SYM>
__device__ __forceinline__ void bt_interior_inplace(const DevOp &op, T *row, int jb, int je,
                                                    Pack<T, V> (&w)[5], const Pack<T, V> (&ha)[2]) {
    const int m = op.m;
    const T t0 = T(op.tap[3]), t1 = T(op.tap[4]), t2 = T(op.tap[5]);
    const int jm = (je < m - 2) ? je : m - 2;
#pragma unroll 4
    for (int j = jb; j < jm; ++j) {
        w[4] = ldv<T, V>(row + (size_t)(j + 2) * kSZ);
        T sv[V];
        istencil<T, V, SYM>(t0, t1, t2, w, sv);
        Pack<T, V> x;
#pragma unroll
        for (int i = 0; i < V; ++i) x.v[i] = sv[i];
        stv<T, V>(row + (size_t)j * kSZ, x);
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
    }
    for (int j = (jb > m - 2 ? jb : m - 2); j < je; ++j) {
        w[4] = (j + 2 - m == 0) ? ha[0] : ha[1];
        T sv[V];
        istencil<T, V, SYM>(t0, t1, t2, w, sv);
        Pack<T, V> x;
#pragma unroll
        for (int i = 0; i < V; ++i) x.v[i] = sv[i];
        stv<T, V>(row + (size_t)j * kSZ, x);
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
    }
}

// In-place closure rows of the B^T pass: local rows j0..j0+3 with 7-point windows from the
// scratch rows (x[i] = y[Jx + i], entries outside the line zero).
template <typename T, int V>
__device__ __forceinline__ void bt_edge_inplace(const DevOp &op, T *row, int j0, int e0, const T *xs,
                                                int c, int xlo, int xhi) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        Pack<T, V> w7[kTaps];
#pragma unroll
        for (int o = 0; o < kTaps; ++o) {
            const int x = t + o + xlo;
            w7[o] = (x >= 0 && x < xhi) ? ldv<T, V>(xs + (size_t)x * kSZ + c) : zero_pack<T, V>();
        }
        T sv[V];
        estencil<T, V>(op, e0 + t, w7, sv);
        Pack<T, V> x;
#pragma unroll
        for (int i = 0; i < V; ++i) x.v[i] = sv[i];
        stv<T, V>(row + (size_t)(j0 + t) * kSZ, x);
    }
}

// One group, called by every thread of the CTA after the tile has landed and every thread has
// run read_halo.  The DistD2 phases of Sec. 4.2 with the backward pass fused into the
// substitution:
//   forward  : fused stencil + forward elimination (Algorithm 5), accumulating the back-swept
//              row 1 as S = sum_j pi_j d_j, so that row 0 is decoupled (d0~ = N1 (d_0 - w_0 S))
//              without a separate backward pass;
//   reduced  : the chunk-end system in FP64 (decoupled 2x2 boundaries or the full 2P system);
//   back-substitution: u_{m-1} = L, u_j = d_j - s^a_j F - s^c_j u_{j+1}, u_0 = F -- the
//              backward pass and Algorithm 6 in one reverse sweep over the forward rows.
// Results go to `og` (forward operator) or back into the tile for the B^T pass (adjoint).
template <typename T, int V, bool ADJ>
__device__ __forceinline__ void group_sweep(const DevOp &op, T *tile, T *xs, double *ends, T *og,
                                            int k, int c, const Pack<T, V> (&hb)[2],
                                            const Pack<T, V> (&ha)[2]) {
    const int m = op.m, P = op.P, n = op.n;
    const int cls = chunk_class(op, k);
    const int J0 = k * m;
    const bool first_edge = !op.periodic && k == 0;
    const bool last_edge = !op.periodic && k == P - 1;
    T *row = tile + (size_t)J0 * kSZ + c;
    Pack<T, V> dprev = zero_pack<T, V>(), S = zero_pack<T, V>();

    // ---- forward pass ----
    if (!ADJ) {
        const int jb = first_edge ? 4 : 0, je = last_edge ? m - 4 : m;
        if (first_edge) fwd_edge<T, V>(op, cls, row, 0, 0, xs, c, -3, kTaps, dprev, S);
        Pack<T, V> w[5];
        if (first_edge) {
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = ldv<T, V>(xs + (size_t)(2 + i) * kSZ + c);
        } else {
            w[0] = hb[0]; w[1] = hb[1];
            w[2] = ldv<T, V>(row); w[3] = ldv<T, V>(row + kSZ);
        }
        if (op.symmetric > 0) fwd_interior<T, V, true>(op, cls, row, jb, je, w, ha, dprev, S);
        else fwd_interior<T, V, false>(op, cls, row, jb, je, w, ha, dprev, S);
        // last 4 rows of a closed line: scratch rows 7..13 hold v[n-7..n-1]; row n-4+t has
        // window v[n-7+t .. n-1+t]
        if (last_edge) fwd_edge<T, V>(op, cls, row, m - 4, kEdgeRows, xs + (size_t)kTaps * kSZ, c, 0, kTaps, dprev, S);
    } else {
#pragma unroll 4
        for (int j = 0; j < m; ++j) {
            const Pack<T, V> g = ldv<T, V>(row + (size_t)j * kSZ);
            const FwdRec<T> q = ld_fwd<T>(op, cls, j);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                dprev.v[i] = q.f * (g.v[i] - q.r * dprev.v[i]);
                S.v[i] = fma(q.pi, dprev.v[i], S.v[i]);
            }
            stv<T, V>(row + (size_t)j * kSZ, dprev);
        }
    }
    {
        // row 0 eliminates the back-swept row 1: d0~ = N1 (d_0 - w_0 S); chunk ends to `ends`
        const Pack<T, V> d0 = ldv<T, V>(row);
        T sa0, w0;
        ld_bwd<T>(op, cls, 0, sa0, w0);
        const T n1 = T(__ldg(op.n1 + cls));
#pragma unroll
        for (int i = 0; i < V; ++i) {
            ends[(size_t)(2 * k) * kSZ + c + i] = double(n1 * (d0.v[i] - w0 * S.v[i]));
            ends[(size_t)(2 * k + 1) * kSZ + c + i] = double(dprev.v[i]);
        }
    }
    __syncthreads();

    // ---- reduced chunk-end system, FP64 ----
    if (op.red_decoupled) {
        // boundary k joins L_{k-1} (ends slot 2k-1) and F_k (slot 2k): every thread solves its
        // own lines' boundary; each slot is read and written by exactly one thread
        const int R = 2 * P, prev = (k == 0) ? P - 1 : k - 1;
        const double a = __ldg(op.red + (size_t)kRedBa * R + k);
        const double cc = __ldg(op.red + (size_t)kRedBc * R + k);
        const double inv = __ldg(op.red + (size_t)kRedBinv * R + k);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            double *ef = ends + (size_t)(2 * k) * kSZ + c + i;
            double *el = ends + (size_t)(2 * prev + 1) * kSZ + c + i;
            const double dl = *el;
            const double Fk = (*ef - a * dl) * inv;
            *ef = Fk;
            *el = dl - cc * Fk;
        }
    } else {
        for (int l = threadIdx.x; l < kSZ; l += blockDim.x) reduced_solve(op, ends + l, kSZ);
    }
    __syncthreads();

    // ---- back-substitution: u_{m-1} = L, u_j = d_j - s^a_j F - s^c_j u_{j+1}, u_0 = F ----
    Pack<T, V> F, u;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        F.v[i] = T(ends[(size_t)(2 * k) * kSZ + c + i]);
        u.v[i] = T(ends[(size_t)(2 * k + 1) * kSZ + c + i]);
    }
    T *orow = og + (size_t)J0 * kSZ + c;
    // the result stays in the tile: the kernel stores the whole tile with one TMA bulk copy
    // (forward operator), or the B^T pass reads it (adjoint)
    T *dst = row;
    stv<T, V>(dst + (size_t)(m - 1) * kSZ, u);
#pragma unroll 4
    for (int j = m - 2; j >= 1; --j) {
        const Pack<T, V> d = ldv<T, V>(row + (size_t)j * kSZ);
        T sa, sc;
        ld_bwd<T>(op, cls, j, sa, sc);
#pragma unroll
        for (int i = 0; i < V; ++i) u.v[i] = (d.v[i] - sa * F.v[i]) - sc * u.v[i];
        stv<T, V>(dst + (size_t)j * kSZ, u);
    }
    stv<T, V>(dst, F);
    if (ADJ) {
        // ---- adjoint: x = B^T y, in place, with the same halo scheme as the forward stencil ----
        __syncthreads();
        Pack<T, V> yb[2], ya[2];
        read_halo<T, V>(op, tile, xs, k, c, yb, ya);
        __syncthreads();
        const int jb = first_edge ? 4 : 0, je = last_edge ? m - 4 : m;
        if (first_edge) bt_edge_inplace<T, V>(op, row, 0, 0, xs, c, -3, kTaps);
        Pack<T, V> w[5];
        if (first_edge) {
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = ldv<T, V>(xs + (size_t)(2 + i) * kSZ + c);
        } else {
            w[0] = yb[0]; w[1] = yb[1];
            w[2] = ldv<T, V>(row); w[3] = ldv<T, V>(row + kSZ);
        }
        if (op.symmetric > 0) bt_interior_inplace<T, V, true>(op, row, jb, je, w, ya);
        else bt_interior_inplace<T, V, false>(op, row, jb, je, w, ya);
        if (last_edge) bt_edge_inplace<T, V>(op, row, m - 4, kEdgeRows, xs + (size_t)kTaps * kSZ, c, 0, kTaps);
    }
    // the result is in the tile: make this thread's writes visible to the kernel's bulk store,
    // or store the rows directly
    if (kBulkStore<T>) {
        fence_async_smem();
    } else {
#pragma unroll 4
        for (int j = 0; j < m; ++j) stv<T, V>(orow + (size_t)j * kSZ, ldv<T, V>(row + (size_t)j * kSZ));
    }
    (void)n;
}

// Shared-memory layout of the resident kernels (per tile buffer, then once per CTA):
//   tiles[nbuf][n][32] (T) | xs[14][32] (T, closure rows) | ends[2P][32] (double) | bars
__host__ __device__ inline size_t tile_bytes_of(int n, size_t es) { return (size_t)n * kSZ * es; }
__host__ __device__ inline size_t xs_bytes_of(size_t es) { return ((size_t)2 * kTaps * kSZ * es + 15) & ~(size_t)15; }

// One CTA per group, P * 32/V threads.  The tile arrives as one TMA bulk copy per chunk; a
// thread starts as soon as its own chunk and its neighbours' have landed.
template <typename T, int V, bool ADJ>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident(const __grid_constant__ DevOp op,
                                                                 const T *__restrict__ in,
                                                                 T *__restrict__ out) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int n = op.n, m = op.m, P = op.P;
    constexpr int tpc = kSZ / V;
    const int k = threadIdx.x / tpc, c = (threadIdx.x % tpc) * V;
    const size_t gofs = (size_t)blockIdx.x * n * kSZ;
    T *tile = reinterpret_cast<T *>(smem);
    T *xs = reinterpret_cast<T *>(smem + tile_bytes_of(n, sizeof(T)));
    double *ends = reinterpret_cast<double *>(smem + tile_bytes_of(n, sizeof(T)) + xs_bytes_of(sizeof(T)));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * kSZ);
    const uint32_t chunk_bytes = (uint32_t)((size_t)m * kSZ * sizeof(T));

    if (threadIdx.x == 0) {
        failed = 0;
        for (int q = 0; q < P; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < P; ++q) {
            mbar_expect_tx(&bars[q], chunk_bytes);
            bulk_g2s(tile + (size_t)q * m * kSZ, in + gofs + (size_t)q * m * kSZ, chunk_bytes, &bars[q]);
        }
    }
    bool ok = mbar_wait(&bars[k], 0);
    if (!ADJ) {
        if (k > 0 || op.periodic) ok = mbar_wait(&bars[(k - 1 + P) % P], 0) && ok;
        if (k < P - 1 || op.periodic) ok = mbar_wait(&bars[(k + 1) % P], 0) && ok;
        // the closure rows of a closed line may reach into the second / second-to-last chunk
        if (!op.periodic && (k == 0 || k == P - 1))
            for (int q = 0; q < P; ++q) ok = mbar_wait(&bars[q], 0) && ok;
    }
    if (!ok) atomicExch(&failed, 1);
    Pack<T, V> hb[2], ha[2];
    if (!ADJ && ok) read_halo<T, V>(op, tile, xs, k, c, hb, ha);
    __syncthreads();
    if (failed) {
        // let every bulk copy land before the CTA's shared memory is released
        for (int q = threadIdx.x; q < P; q += blockDim.x) mbar_wait(&bars[q], 0);
        if (threadIdx.x == 0) record_timeout();
        return;
    }
    group_sweep<T, V, ADJ>(op, tile, xs, ends, out + gofs, k, c, hb, ha);
    if (kBulkStore<T>) {
        __syncthreads();
        if (threadIdx.x == 0) {
            bulk_s2g(out + gofs, tile, (uint32_t)tile_bytes_of(n, sizeof(T)));
            bulk_commit();
            bulk_wait_read();   // shared memory must stay valid until the copy has read it
        }
    }
}

// Persistent variant: each CTA walks groups blockIdx.x, +gridDim.x, ... through `nbuf` tile
// buffers; the TMA bulk copy of a group is issued `nbuf` groups ahead, so HBM reads stay in
// flight while the threads sweep.
template <typename T, int V, bool ADJ>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident_pipe(const __grid_constant__ DevOp op,
                                                                      const T *__restrict__ in,
                                                                      T *__restrict__ out, int nbuf) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int n = op.n, P = op.P, G = op.ngroups;
    constexpr int tpc = kSZ / V;
    const int k = threadIdx.x / tpc, c = (threadIdx.x % tpc) * V;
    const size_t tile_elems = (size_t)n * kSZ;
    const uint32_t tile_bytes = (uint32_t)tile_bytes_of(n, sizeof(T));
    T *tiles = reinterpret_cast<T *>(smem);
    T *xs = reinterpret_cast<T *>(smem + (size_t)nbuf * tile_bytes);
    double *ends = reinterpret_cast<double *>(smem + (size_t)nbuf * tile_bytes + xs_bytes_of(sizeof(T)));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * kSZ);

    if (threadIdx.x == 0) {
        failed = 0;
        for (int b = 0; b < nbuf; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) {
            const long long g = blockIdx.x + (long long)b * gridDim.x;
            if (g >= G) break;
            mbar_expect_tx(&bars[b], tile_bytes);
            bulk_g2s(tiles + (size_t)b * tile_elems, in + (size_t)g * tile_elems, tile_bytes, &bars[b]);
        }
    }
    for (int it = 0;; ++it) {
        const long long g = blockIdx.x + (long long)it * gridDim.x;
        if (g >= G) break;
        const int b = it % nbuf;
        T *tile = tiles + (size_t)b * tile_elems;
        const bool ok = mbar_wait(&bars[b], (uint32_t)((it / nbuf) & 1));
        if (!ok) atomicExch(&failed, 1);
        Pack<T, V> hb[2], ha[2];
        if (!ADJ && ok) read_halo<T, V>(op, tile, xs, k, c, hb, ha);
        __syncthreads();
        if (failed) {
            // drain every bulk copy still in flight into this CTA's buffers, then give up
            for (int d = threadIdx.x; d < nbuf; d += blockDim.x)
                if (blockIdx.x + (long long)(it + d) * gridDim.x < G)
                    mbar_wait(&bars[(it + d) % nbuf], (uint32_t)(((it + d) / nbuf) & 1));
            if (threadIdx.x == 0) record_timeout();
            return;
        }
        group_sweep<T, V, ADJ>(op, tile, xs, ends, out + (size_t)g * tile_elems, k, c, hb, ha);
        __syncthreads();   // every thread is done with this tile, the scratch rows and `ends`
        if (threadIdx.x == 0) {
            if (kBulkStore<T>) {
                bulk_s2g(out + (size_t)g * tile_elems, tile, tile_bytes);
                bulk_commit();
            }
            const long long gn = g + (long long)nbuf * gridDim.x;
            if (gn < G) {
                // the buffer is refilled only after the store has read it, and generic-proxy
                // accesses are ordered before the async refill
                if (kBulkStore<T>) bulk_wait_read();
                fence_async_smem();
                mbar_expect_tx(&bars[b], tile_bytes);
                bulk_g2s(tile, in + (size_t)gn * tile_elems, tile_bytes, &bars[b]);
            }
        }
    }
    if (kBulkStore<T> && threadIdx.x == 0) bulk_wait_read();
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

template <typename T, int V, bool ADJ>
tds_status launch_resident_t(const DevOp &op, const void *in, void *out, int smem, cudaStream_t st) {
    auto kern = k_resident<T, V, ADJ>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    kern<<<op.ngroups, op.P * (kSZ / V), smem, st>>>(op, static_cast<const T *>(in), static_cast<T *>(out));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

template <typename T, int V, bool ADJ>
tds_status launch_pipe_t(const DevOp &op, const void *in, void *out, int nbuf, int smem, int grid,
                         cudaStream_t st) {
    auto kern = k_resident_pipe<T, V, ADJ>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    kern<<<grid, op.P * (kSZ / V), smem, st>>>(op, static_cast<const T *>(in), static_cast<T *>(out), nbuf);
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
    return tile_bytes_of(n, es) + xs_bytes_of(es) + (size_t)2 * P * kSZ * 8 + (size_t)P * 8;
}

size_t pipe_smem_bytes(int n, int P, tds_dtype dtype, int nbuf) {
    const size_t es = (dtype == TDS_F64) ? 8 : 4;
    return (size_t)nbuf * tile_bytes_of(n, es) + xs_bytes_of(es) + (size_t)2 * P * kSZ * 8 + (size_t)nbuf * 8;
}

// Lines per thread in the resident kernels (tds_plan::lanes): 1, 2 or 4 for FP32, 1 or 2 for
// FP64.  More lanes spread the per-row work (plan coefficients, addressing, loop control) over
// more points and give each thread independent recurrences; fewer lanes give more threads.
template <typename T, int V>
tds_status launch_pipelined_v(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    const DevOp &op = p->op[which];
    const int smem = (int)pipe_smem_bytes(p->n, p->P, p->dtype, p->pipe_nbuf);
    const int grid = op.ngroups < p->pipe_grid ? op.ngroups : p->pipe_grid;
    return which ? launch_pipe_t<T, V, true>(op, in, out, p->pipe_nbuf, smem, grid, st)
                 : launch_pipe_t<T, V, false>(op, in, out, p->pipe_nbuf, smem, grid, st);
}

template <typename T, int V>
tds_status launch_resident_v(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    const DevOp &op = p->op[which];
    return which ? launch_resident_t<T, V, true>(op, in, out, p->resident_smem, st)
                 : launch_resident_t<T, V, false>(op, in, out, p->resident_smem, st);
}

tds_status launch_pipelined(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    if (p->dtype == TDS_F64)
        return p->lanes == 2 ? launch_pipelined_v<double, 2>(p, which, in, out, st)
                             : launch_pipelined_v<double, 1>(p, which, in, out, st);
    return p->lanes == 4 ? launch_pipelined_v<float, 4>(p, which, in, out, st)
         : p->lanes == 2 ? launch_pipelined_v<float, 2>(p, which, in, out, st)
                         : launch_pipelined_v<float, 1>(p, which, in, out, st);
}

tds_status launch_resident(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    if (p->dtype == TDS_F64)
        return p->lanes == 2 ? launch_resident_v<double, 2>(p, which, in, out, st)
                             : launch_resident_v<double, 1>(p, which, in, out, st);
    return p->lanes == 4 ? launch_resident_v<float, 4>(p, which, in, out, st)
         : p->lanes == 2 ? launch_resident_v<float, 2>(p, which, in, out, st)
                         : launch_resident_v<float, 1>(p, which, in, out, st);
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
