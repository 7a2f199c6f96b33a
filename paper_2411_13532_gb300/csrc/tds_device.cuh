// tds_device.cuh -- device helpers shared by the resident and streaming kernels of libtds:
// TMA bulk copies and mbarriers (inline PTX, bounded waits), plan accessors, the stencil of one
// row, the reduced chunk-end solve, and small per-thread row vectors.
#pragma once

#include <cstdint>

#include <cuda.h>

#include "tds_internal.h"

namespace tds {
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

// 2-D TMA tensor copy global -> shared of one box of `tmap` at element coordinates (x, y),
// completion signalled on `bar`.  The destination is 128-byte aligned; x * element size is a
// multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 2-D TMA tensor copy shared -> global of one box at (x, y) (x, y >= 0), tracked by bulk groups.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tmap, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                 ::"l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(src))
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

// Bounded wait for phase `parity` of `bar`: false if it did not complete within `limit_ns`.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          unsigned long long limit_ns = kWaitNs) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (long long it = 0; it < kWaitIters; ++it) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return false;
}

template <typename T>
__device__ __forceinline__ T rowc(const DevOp &op, int arr, int cls, int j) {
    if constexpr (sizeof(T) == 8)
        return __ldg(op.row64 + ((size_t)arr * op.ncls + cls) * op.m + j);
    else
        return __ldg(op.row32 + ((size_t)arr * op.ncls + cls) * op.m + j);
}

__device__ __forceinline__ int chunk_class(const DevOp &op, int k) {
    if (op.cls_each) return k;
    return (k == 0) ? op.cls_first : (k == op.P - 1 ? op.cls_last : op.cls_mid);
}

// Index of a chunk class's per-class scalars (cut-off rows, constant-record runs).
__device__ __forceinline__ int scal_cls(const DevOp &op, int cls) { return op.cls_each ? 0 : cls; }

// Stencil of global row J from the window w[i] = v[J - 3 + i] (Eq. cfds and its closures,
// or the transposed taps for the adjoint).
template <typename T>
__device__ __forceinline__ T stencil(const DevOp &op, int J, const T (&w)[kTaps]) {
    if (!op.periodic && (J < kEdgeRows || J >= op.n - kEdgeRows)) {
        const int e = (J < kEdgeRows) ? J : kEdgeRows + J - (op.n - kEdgeRows);
        // the row's form (DevOp::edge_form; FP64: the taps as written), as in the resident sweep
        const int form = (sizeof(T) == 8) ? 0 : op.edge_form[e];
        T s = T(0);
        // FP32: the plan's float copies of the taps (a conversion would issue on the FP64 pipe)
        if (form == 2) {
            T a[kTaps - 1];
#pragma unroll
            for (int o = 0; o < kTaps - 1; ++o) a[o] = w[o + 1] - w[o];
#pragma unroll
            for (int k = 1; k <= 5; ++k)
                s += (sizeof(T) == 4 ? T(op.edge_dd32[e][k - 1]) : T(op.edge_dd[e][k - 1])) * (a[k] - a[k - 1]);
        } else {
#pragma unroll
            for (int o = 0; o < kTaps; ++o)
                s += (sizeof(T) == 4 ? T(op.edge_pf[e][o][0]) : T(op.edge[e][o])) * (form == 1 ? w[o] - w[3] : w[o]);
        }
        return s;
    }
    // uniform interior rows: taps at offsets 0, +1, +2 and the form of op.symmetric
    const T t0 = sizeof(T) == 4 ? T(op.tap32[3]) : T(op.tap[3]);
    const T t1 = sizeof(T) == 4 ? T(op.tap32[4]) : T(op.tap[4]);
    const T t2 = sizeof(T) == 4 ? T(op.tap32[5]) : T(op.tap[5]);
    switch (op.symmetric) {
    case 1:
    case 4:   // symmetric (filter, second derivative); FP32: second differences and the tap sum
        if constexpr (sizeof(T) == 4)
            return T(op.tapsum32) * w[3] + t1 * ((w[4] - w[3]) - (w[3] - w[2])) + t2 * ((w[5] - w[3]) - (w[3] - w[1]));
        else
            return t0 * w[3] + t1 * (w[4] + w[2]) + t2 * (w[5] + w[1]);
    case 2: return t1 * (w[3] + w[4]) + t2 * (w[2] + w[5]);              // nodes -> mid-points
    case 3: return t0 * (w[2] + w[3]) + t1 * (w[1] + w[4]);              // mid-points -> nodes
    default: return t1 * (w[4] - w[2]) + t2 * (w[5] - w[1]);             // antisymmetric
    }
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
__device__ __forceinline__ void reduced_solve(const DevOp &op, double *x, int stride) {
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

} // namespace
} // namespace tds
