// tds_resident.cuh -- the resident DistD2 kernels (Sec. 4.2): one CTA holds W lines of a group of
// 32 (W = 32, 16 or 8; all P chunks) in shared memory, so the field is read once and written
// once.
//
// Per CTA: TMA copies bring the n x W tile into shared memory (one mbarrier per chunk, bounded
// waits; W = 32 one bulk copy per chunk, W < 32 2-D tensor boxes); chunk k is swept by W/V
// threads, each carrying V adjacent lines; then
//   forward  : stencil right-hand side fused into the modified-Thomas forward elimination
//              (Algorithm 5), in place, accumulating the back-swept row 1 as S = sum pi_j d_j
//              so that row 0 is decoupled without a separate backward pass; rows whose folded
//              coefficients have converged take them from registers; the uniform interior
//              stencil has one of five forms (antisymmetric, symmetric, second differences,
//              and the two half-point forms of the mid-point interpolation and its transpose);
//              FP32 sweeps of closed lines take the closure rows' steps in FP64 (Ends64);
//   reduced  : the chunk-end system in FP64 (communication phase; decoupled 2x2 boundary
//              systems when the couplings they ignore are below 2^-64, else the full system);
//   back-substitution: u_{m-1} = L, u_j = d_j - s^a_j F - s^c_j u_{j+1}, u_0 = F -- the
//              backward pass and Algorithm 6 in one reverse sweep;
//   modes    : 0 the stencil right-hand side (derivatives; adjoints on periodic lines, whose
//              operator has the forward form); 1 the closed-line adjoint, the same on A^T with
//              the identity right-hand side, then x = B^T y in place; 2 the solve alone
//              (identity right-hand side, the back-substitution written as the output);
//   output   : FP32 tiles leave with TMA stores; FP64 tiles with per-thread stores.
// Also here: the persistent pipelined variant, the fused pass over several operators of one
// input, the fused term group of the transport equation (three sweeps and their combination),
// and the SEGMENTED kernels for lines no CTA can hold.
//
// The sweep is written once over storage/arithmetic traits (FP32, FP64, split FP64).  The kernel
// templates live here; each arithmetic family is instantiated in a translation unit of its own
// (tds_fam_*.cu, compiled in parallel), and tds_resident.cu dispatches between them.
#pragma once

#include <cstdlib>
#include <cstring>
#include <type_traits>

#include <cudaTypedefs.h>

#include "tds_device.cuh"
#include "tds_df.cuh"

namespace tds {

namespace {

// Device-side status word of this translation unit's kernels: a bounded wait that gives up
// records TDS_ERR_TIMEOUT here (read_device_status collects every unit's word).
__device__ int g_device_status = 0;

__device__ __forceinline__ void record_timeout() { atomicExch(&g_device_status, (int)TDS_ERR_TIMEOUT); }

// a * b + c
__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return ::fma(a, b, c); }

// ------------------------------------------------------------------------------------------
// Storage / arithmetic traits of the sweep.
//   S: element type in HBM and in the tile; A: arithmetic type of the sweep.
//   in  : a raw input row (u, or g for the adjoint) -> A
//   mid : an intermediate value (d_j, y_j) kept in the tile slot of its row
//   out : a final value into the tile slot, as S
// ------------------------------------------------------------------------------------------
template <typename T, int W_ = kSZ, bool E64_ = false>
struct TrNative {
    using S = T;
    using A = T;
    static constexpr int W = W_;   // lines per CTA: the row stride of the tile in shared memory
    static constexpr bool kE64 = E64_;   // FP32 closed lines: closure rows in FP64 (Ends64)
    static constexpr bool kDF = false;   // float-pair recurrences (TrSplit)
    static __device__ __forceinline__ A from_d(double x) { return A(x); }
    static __device__ __forceinline__ double to_d(A x) { return double(x); }
    template <int V>
    static __device__ __forceinline__ Pack<A, V> ld_in(const DevOp &, const S *p, int &) { return ldv<T, V>(p); }
    template <int V>
    static __device__ __forceinline__ Pack<A, V> ld_mid(const S *p) { return ldv<T, V>(p); }
    template <int V>
    static __device__ __forceinline__ void st_mid(S *p, const Pack<A, V> &v) { stv<T, V>(p, v); }
    template <int V>
    static __device__ __forceinline__ void st_out(const DevOp &, S *p, const Pack<A, V> &v) { stv<T, V>(p, v); }
    // FP32: the plan's float copies (the FP64 -> FP32 conversion issues on the FP64 pipe)
    static __device__ __forceinline__ A tap(const DevOp &op, int i) {
        if constexpr (sizeof(T) == 4) return op.tap32[i];
        else return op.tap[i];
    }
    static __device__ __forceinline__ A tapsum(const DevOp &op) {
        if constexpr (sizeof(T) == 4) return op.tapsum32;
        else return op.tapsum;
    }
    static __device__ __forceinline__ A edge(const DevOp &op, int e, int o) {
        if constexpr (sizeof(T) == 4) return op.edge_pf[e][o][0];
        else return op.edge[e][o];
    }
    static __device__ __forceinline__ A edge_dd(const DevOp &op, int e, int k) {
        if constexpr (sizeof(T) == 4) return op.edge_dd32[e][k];
        else return op.edge_dd[e][k];
    }
    static __device__ __forceinline__ void fwd(const DevOp &op, int cls, int j, A &f, A &r, A &pi) {
        const size_t i = (size_t)cls * op.m + j;
        if constexpr (sizeof(T) == 4) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(op.fwd32) + i);
            f = x.x; r = x.y; pi = x.z;
        } else {
            const double2 x = __ldg(reinterpret_cast<const double2 *>(op.fwd64) + 2 * i);
            f = x.x; r = x.y; pi = __ldg(op.fwd64 + 4 * i + 2);
        }
    }
    static __device__ __forceinline__ void bwd(const DevOp &op, int cls, int j, A &sa, A &sc) {
        const size_t i = (size_t)cls * op.m + j;
        if constexpr (sizeof(T) == 4) {
            const float2 x = __ldg(reinterpret_cast<const float2 *>(op.bwd32) + i);
            sa = x.x; sc = x.y;
        } else {
            const double2 x = __ldg(reinterpret_cast<const double2 *>(op.bwd64) + i);
            sa = x.x; sc = x.y;
        }
    }
    // folded interior record {c0, c1, c2, g} and the weight pi_j
    static __device__ __forceinline__ void ifw(const DevOp &op, int cls, int j, A &c0, A &c1, A &c2, A &g) {
        const size_t i = (size_t)cls * op.m + j;
        if constexpr (sizeof(T) == 4) {
            const float4 x = __ldg(reinterpret_cast<const float4 *>(op.ifw32) + i);
            c0 = x.x; c1 = x.y; c2 = x.z; g = x.w;
        } else {
            const double2 a = __ldg(reinterpret_cast<const double2 *>(op.ifw64) + 2 * i);
            const double2 b = __ldg(reinterpret_cast<const double2 *>(op.ifw64) + 2 * i + 1);
            c0 = a.x; c1 = a.y; c2 = b.x; g = b.y;
        }
    }
    static __device__ __forceinline__ A pi(const DevOp &op, int cls, int j) {
        const size_t i = (size_t)cls * op.m + j;
        if constexpr (sizeof(T) == 4) return __ldg(op.fwd32 + 4 * i + 2);
        else return __ldg(op.fwd64 + 4 * i + 2);
    }
    static __device__ __forceinline__ int jpi(const DevOp &op, int cls) {
        cls = scal_cls(op, cls);
        return sizeof(T) == 4 ? op.jpi32[cls] : op.jpi64[cls];
    }
    static __device__ __forceinline__ int jsa(const DevOp &op, int cls) {
        cls = scal_cls(op, cls);
        return sizeof(T) == 4 ? op.jsa32[cls] : op.jsa64[cls];
    }
    // the run of rows [lo, hi) with the constant forward record, and that record
    static __device__ __forceinline__ void kf_run(const DevOp &op, int cls, int &lo, int &hi) {
        cls = scal_cls(op, cls);
        lo = sizeof(T) == 4 ? op.kfl32[cls] : op.kfl64[cls];
        hi = sizeof(T) == 4 ? op.kfh32[cls] : op.kfh64[cls];
    }
    static __device__ __forceinline__ void kf(const DevOp &op, int cls, A &c0, A &c1, A &c2, A &g) {
        cls = scal_cls(op, cls);
        if constexpr (sizeof(T) == 4) {
            c0 = op.kf32[cls][0]; c1 = op.kf32[cls][1]; c2 = op.kf32[cls][2]; g = op.kf32[cls][3];
        } else {
            c0 = op.kf64[cls][0]; c1 = op.kf64[cls][1]; c2 = op.kf64[cls][2]; g = op.kf64[cls][3];
        }
    }
    // the run of rows [lo, hi) with the constant back-substitution coupling s^c, and that value
    static __device__ __forceinline__ void kb_run(const DevOp &op, int cls, int &lo, int &hi) {
        cls = scal_cls(op, cls);
        lo = sizeof(T) == 4 ? op.kbl32[cls] : op.kbl64[cls];
        hi = sizeof(T) == 4 ? op.kbh32[cls] : op.kbh64[cls];
    }
    static __device__ __forceinline__ A kb(const DevOp &op, int cls) {
        cls = scal_cls(op, cls);
        if constexpr (sizeof(T) == 4) return op.kb32[cls];
        else return op.kb64[cls];
    }
};

// Split-precision FP64 sweeps: FP64 storage in HBM and in the tile, recurrences as float pairs
// on the FP32 pipes (tds_df.cuh).  Input rows travel as the FP64 value's bits (ld_in: the stencil
// takes its differences in FP64 before splitting them, so that on smooth data nothing cancels in
// the pairs); intermediate values sit in their row's slot as a pair; results leave as FP64.
// Forward-form operators only (the stencil right-hand side), one line per thread.
template <int W_ = kSZ>
struct TrSplit {
    using S = double;
    using A = DF;
    static constexpr int W = W_;
    static constexpr bool kE64 = true;   // closed lines with a high end gain: closure rows in FP64 (Ends64)
    static constexpr bool kDF = true;
    // by integer operations (tds_df.cuh): the chunk-end values cross to and from the FP64 reduced
    // system without FP64-pipe conversions
    static __device__ __forceinline__ A from_d(double x) { return df_split(x); }
    static __device__ __forceinline__ double to_d(A x) { return df_join(x); }
    template <int V>
    static __device__ __forceinline__ Pack<A, V> ld_in(const DevOp &, const S *p, int &) {
        Pack<A, V> r;
#pragma unroll
        for (int i = 0; i < V; ++i) r.v[i] = df_raw(p[i]);
        return r;
    }
    template <int V>
    static __device__ __forceinline__ Pack<A, V> ld_mid(const S *p) {
        Pack<A, V> r;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float2 x = *reinterpret_cast<const float2 *>(p + i);
            r.v[i] = df_make(x.x, x.y);
        }
        return r;
    }
    template <int V>
    static __device__ __forceinline__ void st_mid(S *p, const Pack<A, V> &v) {
#pragma unroll
        for (int i = 0; i < V; ++i) *reinterpret_cast<float2 *>(p + i) = make_float2(v.v[i].h, v.v[i].l);
    }
    template <int V>
    static __device__ __forceinline__ void st_out(const DevOp &, S *p, const Pack<A, V> &v) {
#pragma unroll
        for (int i = 0; i < V; ++i) p[i] = df_join(v.v[i]);
    }
    static __device__ __forceinline__ A tap(const DevOp &op, int i) { return DF(op.tap[i]); }
    static __device__ __forceinline__ A tapsum(const DevOp &op) { return DF(op.tapsum); }
    static __device__ __forceinline__ A edge(const DevOp &op, int e, int o) { return DF(op.edge[e][o]); }
    static __device__ __forceinline__ A edge_dd(const DevOp &op, int e, int k) { return DF(op.edge_dd[e][k]); }
    static __device__ __forceinline__ void fwd(const DevOp &op, int cls, int j, A &f, A &r, A &pi) {
        const float4 *q = reinterpret_cast<const float4 *>(op.fwdd) + 2 * ((size_t)cls * op.m + j);
        const float4 a = __ldg(q);
        const float2 b = __ldg(reinterpret_cast<const float2 *>(q + 1));
        f = df_make(a.x, a.y); r = df_make(a.z, a.w); pi = df_make(b.x, b.y);
    }
    static __device__ __forceinline__ void bwd(const DevOp &op, int cls, int j, A &sa, A &sc) {
        const float4 a = __ldg(reinterpret_cast<const float4 *>(op.bwdd) + (size_t)cls * op.m + j);
        sa = df_make(a.x, a.y); sc = df_make(a.z, a.w);
    }
    static __device__ __forceinline__ void ifw(const DevOp &op, int cls, int j, A &c0, A &c1, A &c2, A &g) {
        const float4 *q = reinterpret_cast<const float4 *>(op.ifwd) + 2 * ((size_t)cls * op.m + j);
        const float4 a = __ldg(q), b = __ldg(q + 1);
        c0 = df_make(a.x, a.y); c1 = df_make(a.z, a.w); c2 = df_make(b.x, b.y); g = df_make(b.z, b.w);
    }
    static __device__ __forceinline__ A pi(const DevOp &op, int cls, int j) {
        const float2 b = __ldg(reinterpret_cast<const float2 *>(op.fwdd) + 4 * ((size_t)cls * op.m + j) + 2);
        return df_make(b.x, b.y);
    }
    static __device__ __forceinline__ int jpi(const DevOp &op, int cls) { return op.jpid[scal_cls(op, cls)]; }
    static __device__ __forceinline__ int jsa(const DevOp &op, int cls) { return op.jsad[scal_cls(op, cls)]; }
    static __device__ __forceinline__ void kf_run(const DevOp &op, int cls, int &lo, int &hi) {
        cls = scal_cls(op, cls);
        lo = op.kfl64[cls];
        hi = op.kfh64[cls];
    }
    static __device__ __forceinline__ void kf(const DevOp &op, int cls, A &c0, A &c1, A &c2, A &g) {
        const float *k = op.kfd[scal_cls(op, cls)];
        c0 = df_make(k[0], k[1]); c1 = df_make(k[2], k[3]); c2 = df_make(k[4], k[5]); g = df_make(k[6], k[7]);
    }
    static __device__ __forceinline__ void kb_run(const DevOp &op, int cls, int &lo, int &hi) {
        cls = scal_cls(op, cls);
        lo = op.kbl64[cls];
        hi = op.kbh64[cls];
    }
    static __device__ __forceinline__ A kb(const DevOp &op, int cls) {
        const float *k = op.kbd[scal_cls(op, cls)];
        return df_make(k[0], k[1]);
    }
};

using TrF32 = TrNative<float>;
using TrF64 = TrNative<double>;
template <int W> using TrF32w = TrNative<float, W>;
template <int W> using TrF64w = TrNative<double, W>;
using TrF32c = TrNative<float, kSZ, true>;
template <int W> using TrF32cw = TrNative<float, W, true>;

// Whether a finished tile leaves with one TMA bulk store (FP32: the sweep is HBM-bound) or
// with per-thread stores that overlap the sweep (FP64 storage).
template <typename Tr>
constexpr bool kBulkStore = (sizeof(typename Tr::S) == 4);

template <typename Tr, int V>
__device__ __forceinline__ Pack<typename Tr::A, V> zero_a() {
    Pack<typename Tr::A, V> r;
#pragma unroll
    for (int i = 0; i < V; ++i) r.v[i] = Tr::from_d(0.0);
    return r;
}

// Row bounds that cut a sweep into loops (the pi and s^a cut-offs, the constant-record runs)
// belong to the chunk's class.  A warp that holds chunks of several classes (CTAs of 8 or 16
// lines on closed lines: the first and last chunks share warps with interior ones) would run
// every loop to the latest lane's bound, one class's segment after another; the warp takes
// common bounds instead: the latest cut-off (rows past a lane's own cut-off add terms below its
// threshold) and the common part of the constant runs (a lane's per-row records equal its
// class constant there).  Any subset of lanes gives valid bounds, so the mask is the converged
// lanes'.
__device__ __forceinline__ int warp_max_i(int x) { return __reduce_max_sync(__activemask(), x); }
__device__ __forceinline__ int warp_min_i(int x) { return __reduce_min_sync(__activemask(), x); }

template <typename Tr>
__device__ __forceinline__ int warp_jpi(const DevOp &op, int cls) { return warp_max_i(Tr::jpi(op, cls)); }
template <typename Tr>
__device__ __forceinline__ int warp_jsa(const DevOp &op, int cls) { return warp_max_i(Tr::jsa(op, cls)); }
template <typename Tr>
__device__ __forceinline__ void warp_kf_run(const DevOp &op, int cls, int &lo, int &hi) {
    Tr::kf_run(op, cls, lo, hi);
    lo = warp_max_i(lo);
    hi = warp_min_i(hi);
    if (hi < lo) hi = lo;
}
template <typename Tr>
__device__ __forceinline__ void warp_kb_run(const DevOp &op, int cls, int &lo, int &hi) {
    Tr::kb_run(op, cls, lo, hi);
    lo = warp_max_i(lo);
    hi = warp_min_i(hi);
    if (hi < lo) hi = lo;
}

// Forms of the uniform interior stencil (taps t0, t1, t2 at offsets 0, +1, +2 of the row):
//   kAnti: t1 (v[j+1] - v[j-1]) + t2 (v[j+2] - v[j-2])              (first derivative)
//   kSym : t0 v[j] + t1 (v[j+1] + v[j-1]) + t2 (v[j+2] + v[j-2])     (second derivative, filter: FP64)
//   kHalfFwd: t1 (v[j] + v[j+1]) + t2 (v[j-1] + v[j+2])              (nodes -> mid-points)
//   kHalfBwd: t0 (v[j-1] + v[j]) + t1 (v[j-2] + v[j+1])              (its transpose)
//   kSymD: s v[j] + t1 ((v[j+1] - v[j]) - (v[j] - v[j-1])) + t2 ((v[j+2] - v[j]) - (v[j] - v[j-2]))
//          with s = t0 + 2 t1 + 2 t2: the same symmetric taps, for FP32 sweeps -- on smooth data
//          the differences of nearby values are exact, where the kSym sum of a second
//          derivative (s = 0) loses about 6 bits to cancellation
// (the plan's op.symmetric: -1; 1 and 4 (kSym in FP64 sweeps, kSymD in FP32 sweeps); 2; 3).
constexpr int kAnti = 0, kSym = 1, kHalfFwd = 2, kHalfBwd = 3, kSymD = 4;

template <typename A, int FORM>
__device__ __forceinline__ A interior_rhs(A t0, A t1, A t2, A w0, A w1, A w2, A w3, A w4) {
    if (FORM == kSym) return mad(t0, w2, mad(t1, w3 + w1, t2 * (w4 + w0)));
    if (FORM == kSymD) return mad(t0, w2, mad(t1, (w3 - w2) - (w2 - w1), t2 * ((w4 - w2) - (w2 - w0))));
    if (FORM == kHalfFwd) return mad(t1, w2 + w3, t2 * (w1 + w4));
    if (FORM == kHalfBwd) return mad(t0, w1 + w2, t1 * (w0 + w3));
    return mad(t1, w3 - w1, t2 * (w4 - w0));
}

// Interior stencil (offsets -2..2) of V lines from the window w[i] = v[J - 2 + i].
template <typename A, int V, int FORM>
__device__ __forceinline__ void istencil(A t0, A t1, A t2, const Pack<A, V> (&w)[5], A (&s)[V]) {
#pragma unroll
    for (int i = 0; i < V; ++i)
        s[i] = interior_rhs<A, FORM>(t0, t1, t2, w[0].v[i], w[1].v[i], w[2].v[i], w[3].v[i], w[4].v[i]);
}

// Closure-row stencil (offsets -3..3, closed lines) from w[i] = v[J - 3 + i]; e indexes the
// plan's edge rows (0..3 = rows 0..3, 4..7 = rows n-4..n-1).
template <typename Tr, int V>
__device__ __forceinline__ void estencil(const DevOp &op, int e, const Pack<typename Tr::A, V> (&w)[kTaps],
                                         typename Tr::A (&s)[V]) {
    using A = typename Tr::A;
    // FP64 sweeps take the taps as written: their cancellation stays far below the FP64 bar, and
    // the direct form has the fewest FP64 operations (closure rows run on few lanes of a warp)
    const int form = (sizeof(A) == 8) ? 0 : op.edge_form[e];
#pragma unroll
    for (int i = 0; i < V; ++i) s[i] = Tr::from_d(0.0);
    if (form == 2) {          // sum_k d_k (a_k - a_{k-1}), a_k = v[J+k-2] - v[J+k-3]
#pragma unroll
        for (int i = 0; i < V; ++i) {
            A a[kTaps - 1];
#pragma unroll
            for (int o = 0; o < kTaps - 1; ++o) a[o] = w[o + 1].v[i] - w[o].v[i];
#pragma unroll
            for (int k = 1; k <= 5; ++k) s[i] = mad(Tr::edge_dd(op, e, k - 1), a[k] - a[k - 1], s[i]);
        }
    } else {                  // form 1: sum_o c_o (v[J+o] - v[J]); form 0: sum_o c_o v[J+o]
#pragma unroll
        for (int o = 0; o < kTaps; ++o) {
            const A c = Tr::edge(op, e, o);
#pragma unroll
            for (int i = 0; i < V; ++i)
                s[i] = mad(c, form == 1 ? w[o].v[i] - w[3].v[i] : w[o].v[i], s[i]);
        }
    }
}

// The rows of the W lines a CTA holds: line rows [r0, r1) are in `tile` (row r at (r - r0)*W);
// other rows of the same lines are read from HBM at `gin` (read-only input, row stride 32).
template <typename S>
struct TileView {
    S *tile;
    int r0, r1;
    const S *gin;
};

// Row J of the line (cyclic wrap; zero outside a closed line) as an input or mid value.
template <typename Tr, int V, bool MID>
__device__ __forceinline__ Pack<typename Tr::A, V> ld_row(const DevOp &op, const TileView<typename Tr::S> &tv,
                                                          int J, int c, int &unsafe) {
    const int r = line_row(op, J);
    if (r < 0) return zero_a<Tr, V>();
    const typename Tr::S *p = (r >= tv.r0 && r < tv.r1) ? tv.tile + (size_t)(r - tv.r0) * Tr::W + c
                                                        : tv.gin + (size_t)r * kSZ + c;
    return MID ? Tr::template ld_mid<V>(p) : Tr::template ld_in<V>(op, p, unsafe);
}

// Captured before the CTA barrier that lets any thread overwrite the tile: the stencil halo of
// chunk K (2 rows before, 2 after) in registers and, on closed lines, the first and last 7
// rows of the line in the scratch rows xs[0..6], xs[7..13] (closure rows reach 3 points in and
// the sweep works in place), copied as they are: raw inputs for the forward stencil, mid values
// (MID) for the adjoint B^T pass.
template <typename Tr, int V, bool MID>
__device__ __forceinline__ void read_halo(const DevOp &op, const TileView<typename Tr::S> &tv,
                                          typename Tr::S *xs, int K, int c, Pack<typename Tr::A, V> (&hb)[2],
                                          Pack<typename Tr::A, V> (&ha)[2], int &unsafe) {
    using S = typename Tr::S;
    const int J0 = K * op.m;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        hb[i] = ld_row<Tr, V, MID>(op, tv, J0 - 2 + i, c, unsafe);
        ha[i] = ld_row<Tr, V, MID>(op, tv, J0 + op.m + i, c, unsafe);
    }
    if (!op.periodic) {
        auto copy_row = [&](int src, int dst) {
            const S *p = (src >= tv.r0 && src < tv.r1) ? tv.tile + (size_t)(src - tv.r0) * Tr::W + c
                                                       : tv.gin + (size_t)src * kSZ + c;
            if (!MID) (void)Tr::template ld_in<V>(op, p, unsafe);   // range check of the input
            stv<S, V>(xs + (size_t)dst * Tr::W + c, ldv<S, V>(p));
        };
        if (K == 0)
            for (int i = 0; i < kTaps; ++i) copy_row(i, i);
        if (K == op.P - 1)
            for (int i = 0; i < kTaps; ++i) copy_row(op.n - kTaps + i, kTaps + i);
    }
}

// One row of the forward pass: d_j = f_j (s_j - r_j d_{j-1}), S += pi_j d_j, d_j -> tile.
template <typename Tr, int V>
__device__ __forceinline__ void fwd_row(const DevOp &op, int cls, int j, typename Tr::S *row,
                                        const typename Tr::A (&sv)[V], Pack<typename Tr::A, V> &dprev,
                                        Pack<typename Tr::A, V> &S) {
    typename Tr::A f, r, pi;
    Tr::fwd(op, cls, j, f, r, pi);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        dprev.v[i] = f * (sv[i] - r * dprev.v[i]);
        S.v[i] = mad(pi, dprev.v[i], S.v[i]);
    }
    Tr::template st_mid<V>(row + (size_t)j * Tr::W, dprev);
}

// FP32 sweeps of closed lines: a closure can make the chunk ends ill-conditioned -- an error in
// the right-hand side or the forward value of row 1 (n-2) reaches the solution at row 0 (n-1)
// multiplied by about 100 for the second derivative (f''_0 + 11 f''_1 = ...).  Where the planner
// finds such a gain (DevOp::e64; the kernels are the TrNative<float, W, true> instantiations),
// the FP32 sweeps take the four closure rows at each end of the line in FP64: their right-hand sides from
// the (exact) FP32 inputs, their forward steps with the FP64 records, and the quantities the
// reduced system receives from them -- x0 = d_0 - w_0 sum_{j<4} pi_j d_j of the first chunk,
// row 0's value before the rest of S joins it, and the last forward value xl when it belongs to
// an FP64 row.  The stored d_j of those rows are rounded to FP32 as usual (the back-substitution
// does not amplify them).  FP64 sweeps carry none of it (first = last = false).
template <int V>
struct Ends64 {
    double x0[V], xl[V];
    bool first;   // x0 holds the first chunk's row-0 term
    bool last;    // xl holds d_{m-1}
};

// One closure row of an FP32 sweep in FP64: d = f (s - r d), Sx += pi d, d -> tile as FP32.
template <typename Tr, int V>
__device__ __forceinline__ void fwd_row64(const DevOp &op, int cls, int j, typename Tr::S *row,
                                          const double (&sv)[V], double (&d)[V], double (&Sx)[V]) {
    const size_t i = (size_t)cls * op.m + j;
    const double2 fr = __ldg(reinterpret_cast<const double2 *>(op.fwd64) + 2 * i);
    const double pi = __ldg(op.fwd64 + 4 * i + 2);
    Pack<typename Tr::A, V> x;
#pragma unroll
    for (int q = 0; q < V; ++q) {
        d[q] = fr.x * (sv[q] - fr.y * d[q]);
        Sx[q] = ::fma(pi, d[q], Sx[q]);
        x.v[q] = static_cast<typename Tr::A>(d[q]);
    }
    Tr::template st_mid<V>(row + (size_t)j * Tr::W, x);
}

// After FP64 rows [j0, j0 + 4) of a chunk (head: the line's first rows, d0 = d_0 of each line):
// hand the state back to the FP32 sweep and keep what the chunk ends need.
template <typename Tr, int V>
__device__ __forceinline__ void close_rows64(const DevOp &op, int cls, int j0, bool head, const double (&d)[V],
                                             const double (&Sx)[V], const double (&d0)[V],
                                             Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S,
                                             Ends64<V> &ex) {
    if (head) {
        const double w0 = __ldg(op.bwd64 + 2 * (size_t)cls * op.m + 1);   // c_0 / b_0
#pragma unroll
        for (int q = 0; q < V; ++q) ex.x0[q] = ::fma(-w0, Sx[q], d0[q]);
        ex.first = true;
    } else {
#pragma unroll
        for (int q = 0; q < V; ++q) S.v[q] += static_cast<typename Tr::A>(Sx[q]);
    }
    if (j0 + 4 == op.m) {
#pragma unroll
        for (int q = 0; q < V; ++q) ex.xl[q] = d[q];
        ex.last = true;
    }
#pragma unroll
    for (int q = 0; q < V; ++q) dprev.v[q] = static_cast<typename Tr::A>(d[q]);
}

// FP32 sweeps of closed lines with e64 take the closure rows in float-pair arithmetic (about 48
// bits) on the FP32 pipes: the FP64 pipe issues at 1/64 of the FP32 rate on GB300, and in FP64
// these rows put some 70 dependent FP64 warp instructions on the first and last chunks' critical
// path; pairs leave their rounding, magnified about 100 times by the closure, far below the FP32
// bar.  The FP32 inputs are exact in a pair; the quantities handed to the FP64 reduced system
// are joined to FP64 by integer operations (df_join).

// sum_o c_o x_o over the taps of closure row e, c_o as float pairs (DevOp::edge_pf)
__device__ __forceinline__ DF edge_dot_pf(const DevOp &op, int e, const float (&x)[kTaps]) {
    float sh = 0.0f, se = 0.0f;
#pragma unroll
    for (int o = 0; o < kTaps; ++o) {
        const float ch = op.edge_pf[e][o][0], cl = op.edge_pf[e][o][1];
        const float p = __fmul_rn(ch, x[o]);
        float err = __fmaf_rn(ch, x[o], -p);
        err = __fmaf_rn(cl, x[o], err);
        const DF t = df_two(sh, p);
        sh = t.h;
        se = __fadd_rn(se, __fadd_rn(t.l, err));
    }
    return df_two(sh, se);
}

// One closure row in pairs: d = f (s - r d), Sx += pi d (the pair records), d -> tile as FP32.
template <typename Tr, int V>
__device__ __forceinline__ void fwd_row_pf(const DevOp &op, int cls, int j, typename Tr::S *row,
                                           const DF (&sv)[V], DF (&d)[V], DF (&Sx)[V]) {
    const float4 *q = reinterpret_cast<const float4 *>(op.fwdd) + 2 * ((size_t)cls * op.m + j);
    const float4 a = __ldg(q);
    const float2 b = __ldg(reinterpret_cast<const float2 *>(q + 1));
    const DF f = df_make(a.x, a.y), r = df_make(a.z, a.w), pi = df_make(b.x, b.y);
    Pack<typename Tr::A, V> x;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        d[i] = f * (sv[i] - r * d[i]);
        Sx[i] = mad(pi, d[i], Sx[i]);
        x.v[i] = __fadd_rn(d[i].h, d[i].l);
    }
    Tr::template st_mid<V>(row + (size_t)j * Tr::W, x);
}

// After pair rows [j0, j0 + 4) of a chunk: as close_rows64.
template <typename Tr, int V>
__device__ __forceinline__ void close_rows_pf(const DevOp &op, int cls, int j0, bool head, const DF (&d)[V],
                                              const DF (&Sx)[V], const DF (&d0)[V],
                                              Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S,
                                              Ends64<V> &ex) {
    if (head) {
        const float4 b = __ldg(reinterpret_cast<const float4 *>(op.bwdd) + (size_t)cls * op.m);
        const DF w0 = df_make(b.z, b.w);   // c_0 / b_0
#pragma unroll
        for (int i = 0; i < V; ++i) ex.x0[i] = df_join(d0[i] - w0 * Sx[i]);
        ex.first = true;
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) S.v[i] += __fadd_rn(Sx[i].h, Sx[i].l);
    }
    if (j0 + 4 == op.m) {
#pragma unroll
        for (int i = 0; i < V; ++i) ex.xl[i] = df_join(d[i]);
        ex.last = true;
    }
#pragma unroll
    for (int i = 0; i < V; ++i) dprev.v[i] = __fadd_rn(d[i].h, d[i].l);
}

// Interior row of the forward pass with f folded into the coefficients:
// d_j = (the FORM's stencil with taps c0, c1, c2) - g d_{j-1}, one FMA on the recurrence;
// ACC: S += pi_j d_j (rows past the plan's cut-off skip it).
template <typename Tr, int V, int FORM, bool ACC>
__device__ __forceinline__ void fwd_irow_c(const DevOp &op, int cls, int j, typename Tr::S *row,
                                           const Pack<typename Tr::A, V> (&w)[5],
                                           Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S,
                                           typename Tr::A c0, typename Tr::A c1, typename Tr::A c2,
                                           typename Tr::A g) {
    using A = typename Tr::A;
    A p = A(0);
    if (ACC) p = Tr::pi(op, cls, j);
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const A base = interior_rhs<A, FORM>(c0, c1, c2, w[0].v[i], w[1].v[i], w[2].v[i], w[3].v[i], w[4].v[i]);
        dprev.v[i] = mad(-g, dprev.v[i], base);
        if (ACC) S.v[i] = mad(p, dprev.v[i], S.v[i]);
    }
    Tr::template st_mid<V>(row + (size_t)j * Tr::W, dprev);
}

// The same with the row's own record from the plan.
template <typename Tr, int V, int FORM, bool ACC>
__device__ __forceinline__ void fwd_irow(const DevOp &op, int cls, int j, typename Tr::S *row,
                                         const Pack<typename Tr::A, V> (&w)[5],
                                         Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S) {
    typename Tr::A c0, c1, c2, g;
    Tr::ifw(op, cls, j, c0, c1, c2, g);
    fwd_irow_c<Tr, V, FORM, ACC>(op, cls, j, row, w, dprev, S, c0, c1, c2, g);
}

// Interior forward rows [jb, je) reading v[j+2] from the tile (inside the chunk); CONST: every
// row has the class's constant record (k0..kg), else each row loads its own.
template <typename Tr, int V, int FORM, bool ACC, bool CONST>
__device__ __forceinline__ void fwd_irows(const DevOp &op, int cls, typename Tr::S *row, int jb, int je,
                                          Pack<typename Tr::A, V> (&w)[5], Pack<typename Tr::A, V> &dprev,
                                          Pack<typename Tr::A, V> &S, int &unsafe,
                                          typename Tr::A k0 = typename Tr::A(0), typename Tr::A k1 = typename Tr::A(0),
                                          typename Tr::A k2 = typename Tr::A(0), typename Tr::A kg = typename Tr::A(0)) {
#pragma unroll 4
    for (int j = jb; j < je; ++j) {
        w[4] = Tr::template ld_in<V>(op, row + (size_t)(j + 2) * Tr::W, unsafe);
        if (CONST) fwd_irow_c<Tr, V, FORM, ACC>(op, cls, j, row, w, dprev, S, k0, k1, k2, kg);
        else fwd_irow<Tr, V, FORM, ACC>(op, cls, j, row, w, dprev, S);
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
    }
}

// Forward rows [jb, je): the part inside the class's constant-record run [lo, hi) with the
// record in registers, the rest with per-row records.
template <typename Tr, int V, int FORM, bool ACC>
__device__ __forceinline__ void fwd_span(const DevOp &op, int cls, typename Tr::S *row, int jb, int je,
                                         Pack<typename Tr::A, V> (&w)[5], Pack<typename Tr::A, V> &dprev,
                                         Pack<typename Tr::A, V> &S, int &unsafe) {
    int lo, hi;
    warp_kf_run<Tr>(op, cls, lo, hi);
    const int a = (lo < jb) ? jb : (lo > je ? je : lo);
    const int b = (hi < a) ? a : (hi > je ? je : hi);
    typename Tr::A k0, k1, k2, kg;
    Tr::kf(op, cls, k0, k1, k2, kg);
    fwd_irows<Tr, V, FORM, ACC, false>(op, cls, row, jb, a, w, dprev, S, unsafe);
    fwd_irows<Tr, V, FORM, ACC, true>(op, cls, row, a, b, w, dprev, S, unsafe, k0, k1, k2, kg);
    fwd_irows<Tr, V, FORM, ACC, false>(op, cls, row, b, je, w, dprev, S, unsafe);
}

// Split-precision forward rows [jb, je) of a chunk (TrSplit, one line per thread): the stencil's
// differences of the FP64 inputs taken in FP64 and split into float pairs (on smooth data the
// differences are exact and small, so the pairs lose nothing to cancellation), then the folded
// taps, the recurrence d_j = (stencil) - g d_{j-1} and S += pi_j d_j in float-pair arithmetic.
//   antisymmetric taps: c1 (v[j+1] - v[j-1]) + c2 (v[j+2] - v[j-2]), with b_j = v[j+1] - v[j-1]
//       split once per row and v[j+2] - v[j-2] = b_{j+1} + b_{j-1};
//   symmetric taps: c0 v[j] + c1 e_j + c2 (e_{j+1} + e_{j-1}), e_j = (v[j+1] - v[j]) - (v[j] -
//       v[j-1]): the first difference v[j+2] - v[j+1] taken in FP64 and split once per row, e
//       formed in pairs (c0 = f tapsum: zero for a second derivative);
//   half-point taps (the mid-point interpolation and its transpose), with a_j = v[j] + v[j+1]
//       summed in FP64 and split once per row: nodes -> mid-points c1 a_j + c2 (v[j-1] + v[j+2])
//       and mid-points -> nodes c0 a_{j-1} + c1 (v[j-2] + v[j+1]), the outer sums formed in pairs
//       as a_{j+1} + a_{j-1} - a_j and a_j + a_{j-2} - a_{j-1}.
// w[0..3] carry v[jb-2 .. jb+1] as FP64 bits; v[j+2] comes from the tile ahead of the sweep, then
// from the halo `ha` (the next chunk's first two rows).
template <typename Tr, int FORM>
__device__ __forceinline__ void sweep_interior_df(const DevOp &op, int cls, double *row, int jb, int je,
                                                  const Pack<DF, 1> (&w)[5], const Pack<DF, 1> (&ha)[2],
                                                  Pack<DF, 1> &dprev, Pack<DF, 1> &S) {
    static_assert(FORM == kAnti || FORM == kSym || FORM == kHalfFwd || FORM == kHalfBwd,
                  "split sweeps evaluate the antisymmetric, symmetric and half-point forms");
    const int m = op.m;
    const int jm = (je < m - 2) ? je : m - 2;
    const double v0 = df_unraw(w[0].v[0]), v1 = df_unraw(w[1].v[0]);
    double v2 = df_unraw(w[2].v[0]), v3 = df_unraw(w[3].v[0]);
    DF p, c;   // antisymmetric: b_{j-1}, b_j; symmetric: e_{j-1}, e_j; nodes -> mid-points:
               // a_{j-1}, a_j; mid-points -> nodes: a_{j-2}, a_{j-1}
    DF A2;     // symmetric: v[j+1] - v[j], split
    if (FORM == kAnti) {
        p = df_split(v2 - v0);
        c = df_split(v3 - v1);
    } else if (FORM == kHalfFwd) {
        p = df_split(v1 + v2);
        c = df_split(v2 + v3);
    } else if (FORM == kHalfBwd) {
        p = df_split(v0 + v1);
        c = df_split(v1 + v2);
    } else {
        const double a0 = v1 - v0, a1 = v2 - v1, a2 = v3 - v2;
        p = df_split(a1 - a0);
        c = df_split(a2 - a1);
        A2 = df_split(a2);
    }
    const bool c0 = (FORM == kSym) && op.tapsum != 0.0;
    DF d = dprev.v[0], Sa = S.v[0];
    int lo, hi;
    warp_kf_run<Tr>(op, cls, lo, hi);
    DF k0, k1, k2, kg;
    Tr::kf(op, cls, k0, k1, k2, kg);
    const int jp = warp_jpi<Tr>(op, cls);
    auto step = [&](int j, double v4, bool acc, bool cst) {
        DF q0 = k0, q1 = k1, q2 = k2, qg = kg;
        if (!cst) Tr::ifw(op, cls, j, q0, q1, q2, qg);
        DF nx;
        if (FORM == kAnti) {
            nx = df_split(v4 - v2);
        } else if (FORM == kHalfFwd) {
            nx = df_split(v3 + v4);   // a_{j+1}
        } else if (FORM == kHalfBwd) {
            nx = df_split(v2 + v3);   // a_j
        } else {
            // e_{j+1} = a_{j+1} - a_j with the first differences split (one FP64 operation per row;
            // measured 10 % faster for the second derivative than taking e in FP64 too)
            const DF A3 = df_split(v4 - v3);
            nx = A3 - A2;
            A2 = A3;
        }
        DF dn;
        if (FORM == kHalfFwd) dn = dot3(q1, c, q2, (nx + p) - c, -qg, d);
        else if (FORM == kHalfBwd) dn = dot3(q0, c, q1, (nx + p) - c, -qg, d);
        else dn = dot3(q1, c, q2, nx + p, -qg, d);
        if (c0) dn = mad(q0, df_split(v2), dn);
        d = dn;
        if (acc) Sa = mad(Tr::pi(op, cls, j), d, Sa);
        *reinterpret_cast<float2 *>(row + (size_t)j * Tr::W) = make_float2(d.h, d.l);
        p = c;
        c = nx;
        v2 = v3;
        v3 = v4;
    };
    auto run = [&](int a, int b, bool acc, bool cst) {
#pragma unroll 4
        for (int j = a; j < b; ++j) step(j, row[(size_t)(j + 2) * Tr::W], acc, cst);
    };
    auto span = [&](int a, int b, bool acc) {
        const int x = (lo < a) ? a : (lo > b ? b : lo);
        const int y = (hi < x) ? x : (hi > b ? b : hi);
        run(a, x, acc, false);
        run(x, y, acc, true);
        run(y, b, acc, false);
    };
    const int j1 = (jp < jb) ? jb : (jp > jm ? jm : jp);
    span(jb, j1, true);
    span(j1, jm, false);
    for (int j = (jb > m - 2 ? jb : m - 2); j < je; ++j) step(j, df_unraw(ha[j + 2 - m].v[0]), j < jp, false);
    dprev.v[0] = d;
    S.v[0] = Sa;
}

// Interior rows [jb, je) of a stencil sweep over this chunk, in place: w[0..3] holds
// v[j-2..j+1] on entry; v[j+2] is read from the tile while inside the chunk (rows ahead of the
// window are not yet overwritten), then from the halo `ha`.  FWD: forward elimination rows
// (input values); else B^T rows (mid values, result written as output).
template <typename Tr, int V, int FORM, bool FWD>
__device__ __forceinline__ void sweep_interior(const DevOp &op, int cls, typename Tr::S *row, int jb, int je,
                                               Pack<typename Tr::A, V> (&w)[5],
                                               const Pack<typename Tr::A, V> (&ha)[2],
                                               Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S,
                                               int &unsafe) {
    using A = typename Tr::A;
    if constexpr (Tr::kDF && FWD && (FORM == kAnti || FORM == kSym || FORM == kHalfFwd || FORM == kHalfBwd)) {
        sweep_interior_df<Tr, FORM>(op, cls, row, jb, je, w, ha, dprev, S);
        return;
    }
    const int m = op.m;
    const A t0 = (FORM == kSymD) ? Tr::tapsum(op) : Tr::tap(op, 3), t1 = Tr::tap(op, 4), t2 = Tr::tap(op, 5);
    const int jm = (je < m - 2) ? je : m - 2;
    const int jp = FWD ? warp_jpi<Tr>(op, cls) : 0;
    if (FWD) {
        // rows before the pi cut-off accumulate S, the rest do not
        const int j1 = (jp < jb) ? jb : (jp > jm ? jm : jp);
        fwd_span<Tr, V, FORM, true>(op, cls, row, jb, j1, w, dprev, S, unsafe);
        fwd_span<Tr, V, FORM, false>(op, cls, row, j1, jm, w, dprev, S, unsafe);
    } else {
#pragma unroll 4
        for (int j = jb; j < jm; ++j) {
            w[4] = Tr::template ld_mid<V>(row + (size_t)(j + 2) * Tr::W);
            A sv[V];
            istencil<A, V, FORM>(t0, t1, t2, w, sv);
            Pack<A, V> x;
#pragma unroll
            for (int i = 0; i < V; ++i) x.v[i] = sv[i];
            Tr::template st_out<V>(op, row + (size_t)j * Tr::W, x);
#pragma unroll
            for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
        }
    }
    for (int j = (jb > m - 2 ? jb : m - 2); j < je; ++j) {
        w[4] = (j + 2 - m == 0) ? ha[0] : ha[1];
        if (FWD) {
            // FP64 sweeps skip S on these rows past the pi cut-off too (measured: the FP32
            // sweeps run faster with the uniform row)
            if (sizeof(A) == 4 || j < jp) fwd_irow<Tr, V, FORM, true>(op, cls, j, row, w, dprev, S);
            else fwd_irow<Tr, V, FORM, false>(op, cls, j, row, w, dprev, S);
        } else {
            A sv[V];
            istencil<A, V, FORM>(t0, t1, t2, w, sv);
            Pack<A, V> x;
#pragma unroll
            for (int i = 0; i < V; ++i) x.v[i] = sv[i];
            Tr::template st_out<V>(op, row + (size_t)j * Tr::W, x);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = w[i + 1];
    }
}

// Closure rows j0..j0+3 of a stencil sweep: 7-point windows from the scratch rows
// (x[i] = v[Jx + i] at scratch index i - xlo, entries outside [0, xhi) zero).  head: the line's
// first rows.  The forward rows of an FP32 sweep run in FP64 (Ends64).
template <typename Tr, int V, bool FWD>
__device__ __forceinline__ void sweep_edge(const DevOp &op, int cls, typename Tr::S *row, int j0, int e0,
                                           const typename Tr::S *xs, int c, int xlo, int xhi, bool head,
                                           Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S,
                                           Ends64<V> &ex) {
    using A = typename Tr::A;
    bool done = false;
    if constexpr (FWD && Tr::kDF) {
        // split-precision sweeps: the closure rows' right-hand sides in FP64 from the FP64
        // inputs (the taps as written); where the closure magnifies end errors (DevOp::e64) their
        // forward steps in FP64 too (Ends64, as for FP32 sweeps), else in float pairs
        double xw[kTaps + 3][V];
#pragma unroll
        for (int o = 0; o < kTaps + 3; ++o) {
            const int x = o + xlo;
#pragma unroll
            for (int q = 0; q < V; ++q) xw[o][q] = (x >= 0 && x < xhi) ? xs[(size_t)x * Tr::W + c + q] : 0.0;
        }
        double d[V], Sx[V], d0[V];
#pragma unroll
        for (int q = 0; q < V; ++q) { d[q] = head ? 0.0 : static_cast<double>(dprev.v[q]); Sx[q] = 0.0; d0[q] = 0.0; }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const double *cf = op.edge[e0 + t];
            double sd[V];
            A sv[V];
#pragma unroll
            for (int q = 0; q < V; ++q) {
                double s0 = cf[0] * xw[t][q], s1 = cf[1] * xw[t + 1][q];
#pragma unroll
                for (int o = 2; o < kTaps; o += 2) {
                    s0 = ::fma(cf[o], xw[t + o][q], s0);
                    if (o + 1 < kTaps) s1 = ::fma(cf[o + 1], xw[t + o + 1][q], s1);
                }
                sd[q] = s0 + s1;
                sv[q] = df_split(sd[q]);
            }
            if (op.e64) {
                fwd_row64<Tr, V>(op, cls, j0 + t, row, sd, d, Sx);
                if (t == 0) {
#pragma unroll
                    for (int q = 0; q < V; ++q) d0[q] = d[q];
                }
            } else {
                fwd_row<Tr, V>(op, cls, j0 + t, row, sv, dprev, S);
            }
        }
        if (op.e64) close_rows64<Tr, V>(op, cls, j0, head, d, Sx, d0, dprev, S, ex);
        done = true;
    }
    if constexpr (FWD && Tr::kE64 && !Tr::kDF) {
        if (op.e64) {
            // the ten input rows the four windows cover, then the four rows in pairs
            float xw[kTaps + 3][V];
#pragma unroll
            for (int o = 0; o < kTaps + 3; ++o) {
                const int x = o + xlo;
                int dummy = 0;
                const Pack<A, V> v = (x >= 0 && x < xhi) ? Tr::template ld_in<V>(op, xs + (size_t)x * Tr::W + c, dummy)
                                                         : zero_a<Tr, V>();
#pragma unroll
                for (int q = 0; q < V; ++q) xw[o][q] = (float)v.v[q];
            }
            DF d[V], Sx[V], d0[V];
#pragma unroll
            for (int q = 0; q < V; ++q) {
                d[q] = df_make(head ? 0.0f : (float)dprev.v[q], 0.0f);
                Sx[q] = df_make(0.0f, 0.0f);
                d0[q] = Sx[q];
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                DF sv[V];
#pragma unroll
                for (int q = 0; q < V; ++q) {
                    float xv[kTaps];
#pragma unroll
                    for (int o = 0; o < kTaps; ++o) xv[o] = xw[t + o][q];
                    sv[q] = edge_dot_pf(op, e0 + t, xv);
                }
                fwd_row_pf<Tr, V>(op, cls, j0 + t, row, sv, d, Sx);
                if (t == 0) {
#pragma unroll
                    for (int q = 0; q < V; ++q) d0[q] = d[q];
                }
            }
            close_rows_pf<Tr, V>(op, cls, j0, head, d, Sx, d0, dprev, S, ex);
            done = true;
        }
    }
    if (!done) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            A sv[V];
            {
                Pack<A, V> w7[kTaps];
#pragma unroll
                for (int o = 0; o < kTaps; ++o) {
                    const int x = t + o + xlo;
                    int dummy = 0;
                    w7[o] = (x >= 0 && x < xhi)
                                ? (FWD ? Tr::template ld_in<V>(op, xs + (size_t)x * Tr::W + c, dummy)
                                       : Tr::template ld_mid<V>(xs + (size_t)x * Tr::W + c))
                                : zero_a<Tr, V>();
                }
                estencil<Tr, V>(op, e0 + t, w7, sv);
            }
            if (FWD) {
                fwd_row<Tr, V>(op, cls, j0 + t, row, sv, dprev, S);
            } else {
                Pack<A, V> x;
#pragma unroll
                for (int i = 0; i < V; ++i) x.v[i] = sv[i];
                Tr::template st_out<V>(op, row + (size_t)(j0 + t) * Tr::W, x);
            }
        }
    }
}

// A full stencil sweep over this chunk (closure rows peeled on closed lines).
template <typename Tr, int V, bool FWD>
__device__ __forceinline__ void stencil_sweep(const DevOp &op, int k, int cls, typename Tr::S *row,
                                              const typename Tr::S *xs, int c,
                                              const Pack<typename Tr::A, V> (&hb)[2],
                                              const Pack<typename Tr::A, V> (&ha)[2],
                                              Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &S,
                                              Ends64<V> &ex, int &unsafe) {
    const int m = op.m;
    const bool first_edge = !op.periodic && k == 0;
    const bool last_edge = !op.periodic && k == op.P - 1;
    const int jb = first_edge ? 4 : 0, je = last_edge ? m - 4 : m;
    if (first_edge) sweep_edge<Tr, V, FWD>(op, cls, row, 0, 0, xs, c, -3, kTaps, true, dprev, S, ex);
    Pack<typename Tr::A, V> w[5];
    if (first_edge) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            w[i] = FWD ? Tr::template ld_in<V>(op, xs + (size_t)(2 + i) * Tr::W + c, unsafe)
                       : Tr::template ld_mid<V>(xs + (size_t)(2 + i) * Tr::W + c);
    } else {
        w[0] = hb[0];
        w[1] = hb[1];
        w[2] = FWD ? Tr::template ld_in<V>(op, row, unsafe) : Tr::template ld_mid<V>(row);
        w[3] = FWD ? Tr::template ld_in<V>(op, row + Tr::W, unsafe) : Tr::template ld_mid<V>(row + Tr::W);
    }
    if (op.symmetric == 1 || op.symmetric == 4) {
        if constexpr (sizeof(typename Tr::A) == 8)
            sweep_interior<Tr, V, kSym, FWD>(op, cls, row, jb, je, w, ha, dprev, S, unsafe);
        else
            sweep_interior<Tr, V, kSymD, FWD>(op, cls, row, jb, je, w, ha, dprev, S, unsafe);
    } else if (op.symmetric < 0) {
        sweep_interior<Tr, V, kAnti, FWD>(op, cls, row, jb, je, w, ha, dprev, S, unsafe);
    } else if constexpr (V == 1) {
        // the half-point forms belong to the mid-point interpolation and its transpose, one line
        // per thread (the planner fixes it): the forward sweep, and on closed lines the B^T pass
        // of the transpose
        if (op.symmetric == 2) sweep_interior<Tr, V, kHalfFwd, FWD>(op, cls, row, jb, je, w, ha, dprev, S, unsafe);
        else sweep_interior<Tr, V, kHalfBwd, FWD>(op, cls, row, jb, je, w, ha, dprev, S, unsafe);
    }
    // the last 4 rows of a closed line: scratch rows 7..13 hold v[n-7..n-1]
    if (last_edge)
        sweep_edge<Tr, V, FWD>(op, cls, row, m - 4, kEdgeRows, xs + (size_t)kTaps * Tr::W, c, 0, kTaps, false,
                               dprev, S, ex);
}

// Forward pass of chunk K (rows at `row` in the tile): the fused stencil (forward operator) or
// the identity right-hand side (adjoint) with the forward elimination, accumulating S.
template <typename Tr, int V, bool ADJ>
__device__ __forceinline__ void forward_phase(const DevOp &op, typename Tr::S *row, const typename Tr::S *xs,
                                              int K, int cls, int c, const Pack<typename Tr::A, V> (&hb)[2],
                                              const Pack<typename Tr::A, V> (&ha)[2],
                                              Pack<typename Tr::A, V> &dprev, Pack<typename Tr::A, V> &Ssum,
                                              Ends64<V> &ex, int &unsafe) {
    using A = typename Tr::A;
    const int m = op.m;
    ex.first = ex.last = false;
    if constexpr (!ADJ) {
        stencil_sweep<Tr, V, true>(op, K, cls, row, xs, c, hb, ha, dprev, Ssum, ex, unsafe);
    } else {
        // identity right-hand side: d_j = f_j g_j - (f_j r_j) d_{j-1}
        int lo, hi;
        warp_kf_run<Tr>(op, cls, lo, hi);
        const int jp0 = warp_jpi<Tr>(op, cls);
        A k0, k1, k2, kg;
        Tr::kf(op, cls, k0, k1, k2, kg);
        auto arow = [&](int j, bool acc, bool cst) {
            A c0 = k0, c1, c2, gg = kg;
            if (!cst) Tr::ifw(op, cls, j, c0, c1, c2, gg);
            const Pack<A, V> g = Tr::template ld_in<V>(op, row + (size_t)j * Tr::W, unsafe);
            const A p = acc ? Tr::pi(op, cls, j) : A(0);
#pragma unroll
            for (int i = 0; i < V; ++i) {
                dprev.v[i] = mad(-gg, dprev.v[i], c0 * g.v[i]);
                if (acc) Ssum.v[i] = mad(p, dprev.v[i], Ssum.v[i]);
            }
            Tr::template st_mid<V>(row + (size_t)j * Tr::W, dprev);
        };
        // rows [a, b): per-row records outside the constant run, the register record inside it
        auto span = [&](int a, int b, bool acc) {
            const int x = (lo < a) ? a : (lo > b ? b : lo);
            const int y = (hi < x) ? x : (hi > b ? b : hi);
#pragma unroll 4
            for (int j = a; j < x; ++j) arow(j, acc, false);
#pragma unroll 4
            for (int j = x; j < y; ++j) arow(j, acc, true);
#pragma unroll 4
            for (int j = y; j < b; ++j) arow(j, acc, false);
        };
        // FP32 sweeps of closed lines: the four rows at each end of the line in float pairs
        // (Ends64; the FP32 right-hand side is exact in a pair)
        auto rows64 = [&](int j0, bool head) {
            DF d[V], Sx[V], d0[V];
#pragma unroll
            for (int i = 0; i < V; ++i) {
                d[i] = df_make(head ? 0.0f : (float)dprev.v[i], 0.0f);
                Sx[i] = df_make(0.0f, 0.0f);
                d0[i] = Sx[i];
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const Pack<A, V> g = Tr::template ld_in<V>(op, row + (size_t)(j0 + t) * Tr::W, unsafe);
                DF sv[V];
#pragma unroll
                for (int i = 0; i < V; ++i) sv[i] = df_make((float)g.v[i], 0.0f);
                fwd_row_pf<Tr, V>(op, cls, j0 + t, row, sv, d, Sx);
                if (t == 0) {
#pragma unroll
                    for (int i = 0; i < V; ++i) d0[i] = d[i];
                }
            }
            close_rows_pf<Tr, V>(op, cls, j0, head, d, Sx, d0, dprev, Ssum, ex);
        };
        const bool e64 = Tr::kE64 && op.e64;
        const bool head = e64 && K == 0, tail = e64 && K == op.P - 1;
        const int ja = head ? 4 : 0, jz = tail ? m - 4 : m;
        if (head) rows64(0, true);
        const int jp = (jp0 < ja) ? ja : (jp0 > jz ? jz : jp0);
        span(ja, jp, true);
        span(jp, jz, false);
        if (tail) rows64(m - 4, false);
    }
}

// Chunk ends after the forward pass: row 0 eliminates the back-swept row 1,
// e0 = N1 (d_0 - w_0 S); e1 = d_{m-1}.
// With FP64 closure rows (Ends64): e0 = N1 (x0 - w_0 S_rest), e1 = xl, in FP64.
template <typename Tr, int V>
__device__ __forceinline__ void chunk_ends(const DevOp &op, const typename Tr::S *row, int cls,
                                           const Pack<typename Tr::A, V> &dprev,
                                           const Pack<typename Tr::A, V> &Ssum, const Ends64<V> &ex,
                                           double (&e0)[V], double (&e1)[V]) {
    using A = typename Tr::A;
    const Pack<A, V> d0 = Tr::template ld_mid<V>(row);
    A sa0, w0;
    Tr::bwd(op, cls, 0, sa0, w0);
    const A n1 = Tr::from_d(__ldg(op.n1 + cls));
#pragma unroll
    for (int i = 0; i < V; ++i) {
        e0[i] = Tr::to_d(n1 * (d0.v[i] - w0 * Ssum.v[i]));
        e1[i] = Tr::to_d(dprev.v[i]);
    }
    if constexpr (Tr::kE64) {
        if (ex.first) {
            const double n1d = __ldg(op.n1 + cls), w0d = __ldg(op.bwd64 + 2 * (size_t)cls * op.m + 1);
#pragma unroll
            for (int i = 0; i < V; ++i) e0[i] = n1d * ::fma(-w0d, (double)Ssum.v[i], ex.x0[i]);
        }
        if (ex.last) {
#pragma unroll
            for (int i = 0; i < V; ++i) e1[i] = ex.xl[i];
        }
    }
}

// Back-substitution of one chunk from its reduced unknowns F (first row) and L (last row):
// u_{m-1} = L, u_j = d_j - s^a_j F - s^c_j u_{j+1}, u_0 = F.  MID: results stay mid values
// (adjoint y for the B^T pass), else they are written as outputs.
// Rows j = hi-1 down to lo (1 <= lo, hi <= m-1) of the back-substitution: u carries u_{hi} in
// and u_lo out, and each row reaches `put(j, u_j)` in descending order.  Rows at or past the s^a
// cut-off: u_j = d_j - s^c_j u_{j+1}, inside the class's constant run [lo, hi) of s^c from a
// register; rows before it also subtract s^a_j F.  U: unroll factor of the row loops.
template <typename Tr, int V, int U, typename Put>
__device__ __forceinline__ void backsub_range(const DevOp &op, typename Tr::S *row, int cls,
                                              const Pack<typename Tr::A, V> &F, Pack<typename Tr::A, V> &u,
                                              int lo, int hi, Put &&put) {
    using A = typename Tr::A;
    if (lo >= hi) return;
    const int m = op.m;
    const int js0 = warp_jsa<Tr>(op, cls), js = js0 > 1 ? js0 : 1;
    int rl, rh;
    warp_kb_run<Tr>(op, cls, rl, rh);
    const int kh = (rh < js) ? js : (rh > m - 1 ? m - 1 : rh);
    const int kl = (rl < js) ? js : (rl > kh ? kh : rl);
    auto clip = [&](int x) { return x < lo ? lo : (x > hi ? hi : x); };
    const int b1 = clip(kh), b2 = clip(kl), b3 = clip(js);
    auto step = [&](int j, A sc) {
        const Pack<A, V> d = Tr::template ld_mid<V>(row + (size_t)j * Tr::W);
#pragma unroll
        for (int i = 0; i < V; ++i) u.v[i] = mad(-sc, u.v[i], d.v[i]);
        put(j, u);
    };
#pragma unroll U
    for (int j = hi - 1; j >= b1; --j) {
        A sa, sc;
        Tr::bwd(op, cls, j, sa, sc);
        step(j, sc);
    }
    const A kc = Tr::kb(op, cls);
#pragma unroll U
    for (int j = b1 - 1; j >= b2; --j) step(j, kc);
#pragma unroll U
    for (int j = b2 - 1; j >= b3; --j) {
        A sa, sc;
        Tr::bwd(op, cls, j, sa, sc);
        step(j, sc);
    }
#pragma unroll U
    for (int j = b3 - 1; j >= lo; --j) {
        const Pack<A, V> d = Tr::template ld_mid<V>(row + (size_t)j * Tr::W);
        A sa, sc;
        Tr::bwd(op, cls, j, sa, sc);
#pragma unroll
        for (int i = 0; i < V; ++i) u.v[i] = mad(-sc, u.v[i], mad(-sa, F.v[i], d.v[i]));
        put(j, u);
    }
}

// The whole chunk: u_{m-1} = L, rows m-2..1, u_0 = F.
template <typename Tr, int V, typename Put>
__device__ __forceinline__ void backsub_rows(const DevOp &op, typename Tr::S *row, int cls,
                                             const Pack<typename Tr::A, V> &F, Pack<typename Tr::A, V> u,
                                             Put &&put) {
    put(op.m - 1, u);
    backsub_range<Tr, V, 8>(op, row, cls, F, u, 1, op.m - 1, put);
    put(0, F);
}

template <typename Tr, int V, bool MID>
__device__ __forceinline__ void backsub_phase(const DevOp &op, typename Tr::S *row, int cls,
                                              const Pack<typename Tr::A, V> &F, Pack<typename Tr::A, V> u) {
    using A = typename Tr::A;
    backsub_rows<Tr, V>(op, row, cls, F, u, [&](int j, const Pack<A, V> &v) {
        if (MID) Tr::template st_mid<V>(row + (size_t)j * Tr::W, v);
        else Tr::template st_out<V>(op, row + (size_t)j * Tr::W, v);
    });
}

// The closed-line adjoint's x = B^T y folded into the back-substitution (chunks of m >= 16 rows):
// as y_j leaves the recurrence, the interior B^T row j+2 -- whose window y_j..y_{j+4} the thread
// now holds in registers -- is formed and written in place.  What the fold cannot finish waits
// for one barrier: rows 0, 1 and m-2, m-1 of a chunk need two y values of the neighbouring chunk
// (their slots keep y until then), and the four closure rows at each end of the line take their
// 7-point windows from the scratch rows, which the first and last chunks fill with y_0..y_6 and
// y_{n-7}..y_{n-1} on the way.  A second barrier separates those reads from the writes.
template <typename Tr, int V, int FORM>
__device__ __forceinline__ void adjoint_fold(const DevOp &op, typename Tr::S *row, typename Tr::S *xs, int k,
                                             int cls, int c, const Pack<typename Tr::A, V> &F,
                                             const Pack<typename Tr::A, V> &L, Pack<typename Tr::A, V> &dprev,
                                             Pack<typename Tr::A, V> &Ssum, Ends64<V> &ex) {
    using A = typename Tr::A;
    const int m = op.m, P = op.P;
    const A t0 = (FORM == kSymD) ? Tr::tapsum(op) : Tr::tap(op, 3), t1 = Tr::tap(op, 4), t2 = Tr::tap(op, 5);
    auto emit = [&](int r, const Pack<A, V> (&v)[5]) {
        A sv[V];
        istencil<A, V, FORM>(t0, t1, t2, v, sv);
        Pack<A, V> x;
#pragma unroll
        for (int i = 0; i < V; ++i) x.v[i] = sv[i];
        Tr::template st_out<V>(op, row + (size_t)r * Tr::W, x);
    };
    Pack<A, V> w[5], yt[4];   // w[i] = y_{j+i} after row j; yt[i] = y_{m-1-i}
#pragma unroll
    for (int i = 0; i < 5; ++i) w[i] = zero_a<Tr, V>();
#pragma unroll
    for (int i = 0; i < 4; ++i) yt[i] = zero_a<Tr, V>();
    // generic back-substitution row (any j in 1..m-2; the row's own s^c record, s^a F before the
    // cut-off): the straight-line blocks at both ends of the chunk
    const int js0 = warp_jsa<Tr>(op, cls), js = js0 > 1 ? js0 : 1;
    Pack<A, V> u = L;
    auto gstep = [&](int j) {
        const Pack<A, V> d = Tr::template ld_mid<V>(row + (size_t)j * Tr::W);
        A sa, sc;
        Tr::bwd(op, cls, j, sa, sc);
#pragma unroll
        for (int i = 0; i < V; ++i) u.v[i] = (j < js) ? mad(-sc, u.v[i], mad(-sa, F.v[i], d.v[i])) : mad(-sc, u.v[i], d.v[i]);
    };
    auto push = [&](const Pack<A, V> &y) {
#pragma unroll
        for (int i = 4; i > 0; --i) w[i] = w[i - 1];
        w[0] = y;
    };
    // rows m-1 .. m-8: y_{m-1..m-4} kept in registers, y_{m-2}, y_{m-1} in their slots for the next
    // chunk, the last chunk's y_{m-7..m-1} in the scratch rows; B^T rows m-3 .. m-6 where interior
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int j = m - 1 - t;
        if (t > 0) gstep(j);
        push(u);
        if (t < 4) yt[t] = u;
        if (t < 2) Tr::template st_mid<V>(row + (size_t)j * Tr::W, u);
        if (t < kTaps && k == P - 1) Tr::template st_mid<V>(xs + (size_t)(2 * kTaps - 1 - t) * Tr::W + c, u);
        if (t >= 6 || (t >= 4 && k < P - 1)) emit(j + 2, w);
    }
    // rows m-9 .. 7: the window and B^T row j+2
    backsub_range<Tr, V, 8>(op, row, cls, F, u, kTaps, m - 8, [&](int j, const Pack<A, V> &y) {
        push(y);
        emit(j + 2, w);
    });
    // rows 6 .. 0: y_0, y_1 in their slots for the previous chunk, the first chunk's y_0..y_6 in the
    // scratch rows; B^T rows 8 .. 2 where interior
#pragma unroll
    for (int t = 0; t < kTaps; ++t) {
        const int j = kTaps - 1 - t;
        if (j > 0) gstep(j);
        else u = F;
        push(u);
        if (j <= 1) Tr::template st_mid<V>(row + (size_t)j * Tr::W, u);
        if (k == 0) Tr::template st_mid<V>(xs + (size_t)j * Tr::W + c, u);
        if (j >= 2 || k > 0) emit(j + 2, w);
    }
    __syncthreads();
    Pack<A, V> yl[2], yr[2];
    if (k > 0) {
        yl[0] = Tr::template ld_mid<V>(row - (size_t)2 * Tr::W);
        yl[1] = Tr::template ld_mid<V>(row - (size_t)Tr::W);
    }
    if (k < P - 1) {
        yr[0] = Tr::template ld_mid<V>(row + (size_t)m * Tr::W);
        yr[1] = Tr::template ld_mid<V>(row + (size_t)(m + 1) * Tr::W);
    }
    __syncthreads();
    if (k > 0) {
        const Pack<A, V> v0[5] = {yl[0], yl[1], w[0], w[1], w[2]};
        emit(0, v0);
        const Pack<A, V> v1[5] = {yl[1], w[0], w[1], w[2], w[3]};
        emit(1, v1);
    }
    if (k < P - 1) {
        const Pack<A, V> v0[5] = {yt[3], yt[2], yt[1], yt[0], yr[0]};
        emit(m - 2, v0);
        const Pack<A, V> v1[5] = {yt[2], yt[1], yt[0], yr[0], yr[1]};
        emit(m - 1, v1);
    }
    if (k == 0) sweep_edge<Tr, V, false>(op, cls, row, 0, 0, xs, c, -3, kTaps, true, dprev, Ssum, ex);
    if (k == P - 1)
        sweep_edge<Tr, V, false>(op, cls, row, m - kEdgeRows, kEdgeRows, xs + (size_t)kTaps * Tr::W, c, 0, kTaps,
                                 false, dprev, Ssum, ex);
}

// One group, whole line in the tile.  Called by every thread of the CTA after the tile has
// landed and every thread has run read_halo; leaves the result in the tile (as S).  Contains
// __syncthreads().
template <typename Tr, int V, int MODE>
__device__ __forceinline__ void group_sweep(const DevOp &op, typename Tr::S *tile, typename Tr::S *xs,
                                            double *ends, int k, int c,
                                            const Pack<typename Tr::A, V> (&hb)[2],
                                            const Pack<typename Tr::A, V> (&ha)[2], int &unsafe) {
    using A = typename Tr::A;
    using S = typename Tr::S;
    const int m = op.m, P = op.P;
    const int cls = chunk_class(op, k);
    S *row = tile + (size_t)k * m * Tr::W + c;
    Pack<A, V> dprev = zero_a<Tr, V>(), Ssum = zero_a<Tr, V>();
    Ends64<V> ex;

    forward_phase<Tr, V, MODE != 0>(op, row, xs, k, cls, c, hb, ha, dprev, Ssum, ex, unsafe);
    {
        double e0[V], e1[V];
        chunk_ends<Tr, V>(op, row, cls, dprev, Ssum, ex, e0, e1);
#pragma unroll
        for (int i = 0; i < V; ++i) {
            ends[(size_t)(2 * k) * Tr::W + c + i] = e0[i];
            ends[(size_t)(2 * k + 1) * Tr::W + c + i] = e1[i];
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
            double *ef = ends + (size_t)(2 * k) * Tr::W + c + i;
            double *el = ends + (size_t)(2 * prev + 1) * Tr::W + c + i;
            const double dl = *el;
            const double Fk = (*ef - a * dl) * inv;
            *ef = Fk;
            *el = dl - cc * Fk;
        }
    } else {
        for (int l = threadIdx.x; l < Tr::W; l += blockDim.x) reduced_solve(op, ends + l, Tr::W);
    }
    __syncthreads();

    Pack<A, V> F, L;
#pragma unroll
    for (int i = 0; i < V; ++i) {
        F.v[i] = Tr::from_d(ends[(size_t)(2 * k) * Tr::W + c + i]);
        L.v[i] = Tr::from_d(ends[(size_t)(2 * k + 1) * Tr::W + c + i]);
    }
    if (MODE == 1 && op.bt_fold) {
        // closed lines only (periodic adjoints have the forward form)
        if (op.symmetric == 1 || op.symmetric == 4) {
            if constexpr (sizeof(A) == 8) adjoint_fold<Tr, V, kSym>(op, row, xs, k, cls, c, F, L, dprev, Ssum, ex);
            else adjoint_fold<Tr, V, kSymD>(op, row, xs, k, cls, c, F, L, dprev, Ssum, ex);
        } else if (op.symmetric < 0) {
            adjoint_fold<Tr, V, kAnti>(op, row, xs, k, cls, c, F, L, dprev, Ssum, ex);
        } else if constexpr (V == 1) {
            if (op.symmetric == 2) adjoint_fold<Tr, V, kHalfFwd>(op, row, xs, k, cls, c, F, L, dprev, Ssum, ex);
            else adjoint_fold<Tr, V, kHalfBwd>(op, row, xs, k, cls, c, F, L, dprev, Ssum, ex);
        }
        return;
    }
    backsub_phase<Tr, V, MODE == 1>(op, row, cls, F, L);
    if (MODE == 1) {
        // ---- adjoint: x = B^T y, in place, with the same halo scheme as the forward stencil ----
        __syncthreads();
        Pack<A, V> yb[2], ya[2];
        const TileView<S> tv{tile, 0, op.n, nullptr};
        read_halo<Tr, V, true>(op, tv, xs, k, c, yb, ya, unsafe);
        __syncthreads();
        stencil_sweep<Tr, V, false>(op, k, cls, row, xs, c, yb, ya, dprev, Ssum, ex, unsafe);
    }
}

// Shared-memory layout of the resident kernels (W lines per CTA):
//   tiles[nbuf][n][W] (S) | xs[14][W] (S, closure rows) | ends[2P][W] (double) | bars
__host__ __device__ inline size_t tile_bytes_of(int n, size_t es, int w = kSZ) { return (size_t)n * w * es; }
__host__ __device__ inline size_t xs_bytes_of(size_t es, int w = kSZ) {
    return ((size_t)2 * kTaps * w * es + 15) & ~(size_t)15;
}

// A CTA that holds W < 32 lines of a group moves its rows with 2-D TMA tensor copies: the field
// is seen as a [rows][32] array (rows = n x groups, row stride 32 elements) and one box is
// box_rows rows of W elements (box_rows divides the chunk length m, at most 256).
struct TileMaps {
    CUtensorMap in, out;
    int box_rows;
};

// FP32 whole-group CTAs: each chunk's rows leave as soon as its own threads have finished them
// -- one bulk copy per chunk (contiguous in the tile and in HBM), issued by the chunk's first
// thread once its warp's writes are fenced -- rather than one copy of the whole tile after a CTA
// barrier, so that the early chunks' stores overlap the slowest chunk's last rows.  Called by
// every thread of the CTA once it has written the last of its chunk's rows (no thread writes
// another chunk's rows after that); the issuing thread waits until its copy has read shared
// memory.
template <typename S>
__device__ __forceinline__ void store_chunk(S *og, const S *tile, int m, int k, int c) {
    fence_async_smem();
    __syncwarp();
    if (c == 0) {
        bulk_s2g(og + (size_t)k * m * kSZ, tile + (size_t)k * m * kSZ, (uint32_t)((size_t)m * kSZ * sizeof(S)));
        bulk_commit();
        bulk_wait_read();
    }
}

// The finished tile (in shared memory) to HBM.  og: the first element of this CTA's lines of
// the group; y0: the group's first row in the [rows][32] view; x0: its first line.
template <typename Tr, int V>
__device__ __forceinline__ void store_tile(const DevOp &op, const TileMaps &tm, const typename Tr::S *tile,
                                           typename Tr::S *og, int x0, int y0, int k, int c) {
    using S = typename Tr::S;
    if constexpr (kBulkStore<Tr> && Tr::W == kSZ) {
        store_chunk<S>(og, tile, op.m, k, c);
    } else if (kBulkStore<Tr>) {
        fence_async_smem();   // this thread's tile writes are visible to the bulk store
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int r = 0; r < op.n; r += tm.box_rows)
                tma_store_2d(&tm.out, x0, y0 + r, tile + (size_t)r * Tr::W);
            bulk_commit();
            bulk_wait_read();   // shared memory must stay valid until the copy has read it
        }
    } else {
        const size_t ot = (size_t)k * op.m * Tr::W + c, ob = (size_t)k * op.m * kSZ + c;
#pragma unroll 4
        for (int j = 0; j < op.m; ++j)
            stv<S, V>(og + ob + (size_t)j * kSZ, ldv<S, V>(tile + ot + (size_t)j * Tr::W));
    }
}

// One CTA per W lines of a group (32/W CTAs per group), P * W/V threads.  The tile arrives as
// TMA copies, one mbarrier per chunk (W = 32: one bulk copy of the contiguous chunk; W < 32:
// m / box_rows tensor boxes); a thread starts as soon as its own chunk and its neighbours'
// have landed.
template <typename Tr, int V, int MODE>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident(const __grid_constant__ DevOp op,
                                                                 const __grid_constant__ TileMaps tm,
                                                                 const typename Tr::S *__restrict__ in,
                                                                 typename Tr::S *__restrict__ out) {
    using S = typename Tr::S;
    constexpr int W = Tr::W;
    constexpr int tpc = W / V;
    constexpr int parts = kSZ / W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int n = op.n, m = op.m, P = op.P;
    const int k = threadIdx.x / tpc, c = (threadIdx.x % tpc) * V;
    const long long g = blockIdx.x / parts;
    const int x0 = (int)(blockIdx.x % parts) * W;
    const int y0 = (int)(g * n);                                // < 2^31, checked by the host
    const size_t gofs = (size_t)g * n * kSZ + x0;
    S *tile = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + tile_bytes_of(n, sizeof(S), W));
    double *ends = reinterpret_cast<double *>(smem + tile_bytes_of(n, sizeof(S), W) + xs_bytes_of(sizeof(S), W));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * W);
    const uint32_t chunk_bytes = (uint32_t)((size_t)m * W * sizeof(S));
    if constexpr (W < kSZ) {
        // tensor boxes land on 128-byte boundaries of the tile; never issue a misaligned one
        // (the same address for every thread: the whole CTA returns)
        if ((smem_u32(tile) & 127u) != 0) {
            if (threadIdx.x == 0) atomicExch(&g_device_status, (int)TDS_ERR_CUDA);
            return;
        }
    }

    if (threadIdx.x == 0) {
        failed = 0;
        for (int q = 0; q < P; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < P; ++q) {
            mbar_expect_tx(&bars[q], chunk_bytes);
            if constexpr (W == kSZ) {
                bulk_g2s(tile + (size_t)q * m * W, in + gofs + (size_t)q * m * kSZ, chunk_bytes, &bars[q]);
            } else {
                for (int r = q * m; r < (q + 1) * m; r += tm.box_rows)
                    tma_load_2d(tile + (size_t)r * W, &tm.in, x0, y0 + r, &bars[q]);
            }
        }
    }
    bool ok = mbar_wait(&bars[k], 0);
    if (MODE == 0) {
        if (k > 0 || op.periodic) ok = mbar_wait(&bars[(k - 1 + P) % P], 0) && ok;
        if (k < P - 1 || op.periodic) ok = mbar_wait(&bars[(k + 1) % P], 0) && ok;
        // the closure rows of a closed line reach 3 rows in (rows 0..6 and n-7..n-1, copied to
        // the scratch rows by the first and last chunks' threads): with m >= 4 they lie in the
        // chunk and its neighbour, so the first and last chunks start as soon as those two land
    }
    if (!ok) atomicExch(&failed, 1);
    int unsafe = 0;
    Pack<typename Tr::A, V> hb[2], ha[2];
    if (MODE == 0 && ok) read_halo<Tr, V, false>(op, TileView<S>{tile, 0, n, in + gofs}, xs, k, c, hb, ha, unsafe);
    __syncthreads();
    if (failed) {
        // let every copy land before the CTA's shared memory is released
        for (int q = threadIdx.x; q < P; q += blockDim.x) mbar_wait(&bars[q], 0);
        if (threadIdx.x == 0) record_timeout();
        return;
    }
    group_sweep<Tr, V, MODE>(op, tile, xs, ends, k, c, hb, ha, unsafe);
    store_tile<Tr, V>(op, tm, tile, out + gofs, x0, y0, k, c);
}

// Several forward-form operators of one input in one pass (the transport-equation kernels of
// Sec. 5 share one read of the field among several derivative operators): each CTA sweeps its
// W lines once per operator, re-loading the tile for every operator after the first from L2
// (the CTA stored its previous result only microseconds before), so HBM sees one read of the
// input and one write per result.  All operators share the geometry of op[0].
struct MultiArgs {
    DevOp op[kMaxMulti];
    void *out[kMaxMulti];
    int count;
};

struct MultiMaps {
    CUtensorMap in;
    CUtensorMap out[kMaxMulti];
    int box_rows;
};

template <typename Tr>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident_multi(const __grid_constant__ MultiArgs ma,
                                                                       const __grid_constant__ MultiMaps mm,
                                                                       const typename Tr::S *__restrict__ in) {
    using S = typename Tr::S;
    constexpr int W = Tr::W;
    constexpr int parts = kSZ / W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const DevOp &op0 = ma.op[0];
    const int n = op0.n, m = op0.m, P = op0.P;
    const int k = threadIdx.x / W, c = threadIdx.x % W;
    const long long g = blockIdx.x / parts;
    const int x0 = (int)(blockIdx.x % parts) * W;
    const int y0 = (int)(g * n);                                // < 2^31, checked by the host
    const size_t gofs = (size_t)g * n * kSZ + x0;
    S *tile = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + tile_bytes_of(n, sizeof(S), W));
    double *ends = reinterpret_cast<double *>(smem + tile_bytes_of(n, sizeof(S), W) + xs_bytes_of(sizeof(S), W));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * W);
    const uint32_t chunk_bytes = (uint32_t)((size_t)m * W * sizeof(S));
    if constexpr (W < kSZ) {
        if ((smem_u32(tile) & 127u) != 0) {   // see k_resident
            if (threadIdx.x == 0) atomicExch(&g_device_status, (int)TDS_ERR_CUDA);
            return;
        }
    }
    if (threadIdx.x == 0) {
        failed = 0;
        for (int q = 0; q < P; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    for (int o = 0; o < ma.count; ++o) {
        const DevOp &op = ma.op[o];
        const uint32_t par = (uint32_t)(o & 1);
        if (threadIdx.x == 0) {
            for (int q = 0; q < P; ++q) {
                mbar_expect_tx(&bars[q], chunk_bytes);
                if constexpr (W == kSZ) {
                    bulk_g2s(tile + (size_t)q * m * W, in + gofs + (size_t)q * m * kSZ, chunk_bytes, &bars[q]);
                } else {
                    for (int r = q * m; r < (q + 1) * m; r += mm.box_rows)
                        tma_load_2d(tile + (size_t)r * W, &mm.in, x0, y0 + r, &bars[q]);
                }
            }
        }
        bool ok = mbar_wait(&bars[k], par);
        if (k > 0 || op.periodic) ok = mbar_wait(&bars[(k - 1 + P) % P], par) && ok;
        if (k < P - 1 || op.periodic) ok = mbar_wait(&bars[(k + 1) % P], par) && ok;
        if (!ok) atomicExch(&failed, 1);
        int unsafe = 0;
        Pack<typename Tr::A, 1> hb[2], ha[2];
        if (ok) read_halo<Tr, 1, false>(op, TileView<S>{tile, 0, n, in + gofs}, xs, k, c, hb, ha, unsafe);
        __syncthreads();
        if (failed) {
            // let this operator's copies land before the CTA's shared memory is released
            for (int q = threadIdx.x; q < P; q += blockDim.x) mbar_wait(&bars[q], par);
            if (threadIdx.x == 0) record_timeout();
            return;
        }
        group_sweep<Tr, 1, 0>(op, tile, xs, ends, k, c, hb, ha, unsafe);
        S *og = static_cast<S *>(ma.out[o]) + gofs;
        if (kBulkStore<Tr>) {
            fence_async_smem();
            __syncthreads();
            if (threadIdx.x == 0) {
                if constexpr (W == kSZ) {
                    bulk_s2g(og, tile, (uint32_t)tile_bytes_of(n, sizeof(S)));
                } else {
                    for (int r = 0; r < n; r += mm.box_rows)
                        tma_store_2d(&mm.out[o], x0, y0 + r, tile + (size_t)r * W);
                }
                bulk_commit();
                bulk_wait_read();   // the tile is refilled by the next operator's copies
            }
        } else {
            const size_t ot = (size_t)k * m * W + c, ob = (size_t)k * m * kSZ + c;
#pragma unroll 4
            for (int j = 0; j < m; ++j) og[ob + (size_t)j * kSZ] = tile[ot + (size_t)j * W];
        }
        // every thread is done with the tile, the scratch rows and `ends` before the next
        // operator's copies (async proxy) overwrite them
        fence_async_smem();
        __syncthreads();
    }
}

// The same fused pass with one CTA per (unit, operator): the `count` CTAs of a unit (W lines of
// a group) are adjacent in the grid, so they run in the same wave and the first to load the
// input tile brings it from HBM, the others find it in L2; each CTA is the single-operator
// resident kernel (bitwise the same results), and the operators' sweeps run side by side
// instead of one after another.
template <typename Tr>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident_ilv(const __grid_constant__ MultiArgs ma,
                                                                     const __grid_constant__ MultiMaps mm,
                                                                     const typename Tr::S *__restrict__ in) {
    using S = typename Tr::S;
    constexpr int W = Tr::W;
    constexpr int parts = kSZ / W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int o = (int)(blockIdx.x % (unsigned)ma.count);
    const long long unit = blockIdx.x / (unsigned)ma.count;
    const DevOp &op = ma.op[o];
    const int n = op.n, m = op.m, P = op.P;
    const int k = threadIdx.x / W, c = threadIdx.x % W;
    const long long g = unit / parts;
    const int x0 = (int)(unit % parts) * W;
    const int y0 = (int)(g * n);                                // < 2^31, checked by the host
    const size_t gofs = (size_t)g * n * kSZ + x0;
    S *tile = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + tile_bytes_of(n, sizeof(S), W));
    double *ends = reinterpret_cast<double *>(smem + tile_bytes_of(n, sizeof(S), W) + xs_bytes_of(sizeof(S), W));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * W);
    const uint32_t chunk_bytes = (uint32_t)((size_t)m * W * sizeof(S));
    if constexpr (W < kSZ) {
        if ((smem_u32(tile) & 127u) != 0) {   // see k_resident
            if (threadIdx.x == 0) atomicExch(&g_device_status, (int)TDS_ERR_CUDA);
            return;
        }
    }
    if (threadIdx.x == 0) {
        failed = 0;
        for (int q = 0; q < P; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 0; q < P; ++q) {
            mbar_expect_tx(&bars[q], chunk_bytes);
            if constexpr (W == kSZ) {
                bulk_g2s(tile + (size_t)q * m * W, in + gofs + (size_t)q * m * kSZ, chunk_bytes, &bars[q]);
            } else {
                for (int r = q * m; r < (q + 1) * m; r += mm.box_rows)
                    tma_load_2d(tile + (size_t)r * W, &mm.in, x0, y0 + r, &bars[q]);
            }
        }
    }
    bool ok = mbar_wait(&bars[k], 0);
    if (k > 0 || op.periodic) ok = mbar_wait(&bars[(k - 1 + P) % P], 0) && ok;
    if (k < P - 1 || op.periodic) ok = mbar_wait(&bars[(k + 1) % P], 0) && ok;
    if (!ok) atomicExch(&failed, 1);
    int unsafe = 0;
    Pack<typename Tr::A, 1> hb[2], ha[2];
    if (ok) read_halo<Tr, 1, false>(op, TileView<S>{tile, 0, n, in + gofs}, xs, k, c, hb, ha, unsafe);
    __syncthreads();
    if (failed) {
        for (int q = threadIdx.x; q < P; q += blockDim.x) mbar_wait(&bars[q], 0);
        if (threadIdx.x == 0) record_timeout();
        return;
    }
    group_sweep<Tr, 1, 0>(op, tile, xs, ends, k, c, hb, ha, unsafe);
    S *og = static_cast<S *>(ma.out[o]) + gofs;
    if constexpr (kBulkStore<Tr> && W == kSZ) {
        store_chunk<S>(og, tile, m, k, c);
    } else if (kBulkStore<Tr>) {
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int r = 0; r < n; r += mm.box_rows)
                tma_store_2d(&mm.out[o], x0, y0 + r, tile + (size_t)r * W);
            bulk_commit();
            bulk_wait_read();
        }
    } else {
        const size_t ot = (size_t)k * m * W + c, ob = (size_t)k * m * kSZ + c;
#pragma unroll 4
        for (int j = 0; j < m; ++j) og[ob + (size_t)j * kSZ] = tile[ot + (size_t)j * W];
    }
}

// One term group of the skew-symmetric momentum transport right-hand side (Sec. 5, Eq.
// mom-comps), the "abstract kernel" that reads its fields once for three operators:
//   out = -1/2 (u_j * D1 u_i + D1 (u_j u_i)) + nu * D2 u_i
// along the plans' direction j, all fields in that direction's layout (u_i == u_j when i = j).
// Each CTA sweeps its W lines three times (D1 of u_i; D1 of the product, formed in shared memory
// after the tile lands; D2 of u_i), re-loading the tile from L2 between the sweeps, and folds
// the combination into per-thread epilogues whose read-modify-writes of `out` hit L2: HBM sees
// the input fields read once and `out` written once.
struct TransportArgs {
    DevOp op1, op2;   // first and second derivative on one geometry
    double nu;
};

template <typename Tr, int V>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident_transport(const __grid_constant__ TransportArgs ta,
                                                                           const __grid_constant__ MultiMaps mm,
                                                                           const typename Tr::S *__restrict__ ui,
                                                                           const typename Tr::S *__restrict__ uj,
                                                                           typename Tr::S *__restrict__ out) {
    using S = typename Tr::S;
    using A = typename Tr::A;
    constexpr int W = Tr::W;
    constexpr int tpc = W / V;
    constexpr int parts = kSZ / W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int n = ta.op1.n, m = ta.op1.m, P = ta.op1.P;
    const int k = threadIdx.x / tpc, c = (threadIdx.x % tpc) * V;
    const long long g = blockIdx.x / parts;
    const int x0 = (int)(blockIdx.x % parts) * W;
    const int y0 = (int)(g * n);                                // < 2^31, checked by the host
    const size_t gofs = (size_t)g * n * kSZ + x0;
    S *tile = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + tile_bytes_of(n, sizeof(S), W));
    double *ends = reinterpret_cast<double *>(smem + tile_bytes_of(n, sizeof(S), W) + xs_bytes_of(sizeof(S), W));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * W);
    const uint32_t chunk_bytes = (uint32_t)((size_t)m * W * sizeof(S));
    if constexpr (W < kSZ) {
        if ((smem_u32(tile) & 127u) != 0) {   // see k_resident
            if (threadIdx.x == 0) atomicExch(&g_device_status, (int)TDS_ERR_CUDA);
            return;
        }
    }
    if (threadIdx.x == 0) {
        failed = 0;
        for (int q = 0; q < P; ++q) mbar_init(&bars[q], 1);
        fence_mbar_init();
    }
    __syncthreads();
    // this thread's rows: tile row (k m + j) W + c, field element gofs + (k m + j) 32 + c (V lines)
    const size_t ot = (size_t)k * m * W + c, ob = gofs + (size_t)k * m * kSZ + c;
    for (int o = 0; o < 3; ++o) {
        const DevOp &op = (o == 2) ? ta.op2 : ta.op1;
        const uint32_t par = (uint32_t)(o & 1);
        if (threadIdx.x == 0) {
            for (int q = 0; q < P; ++q) {
                mbar_expect_tx(&bars[q], chunk_bytes);
                if constexpr (W == kSZ) {
                    bulk_g2s(tile + (size_t)q * m * W, ui + gofs + (size_t)q * m * kSZ, chunk_bytes, &bars[q]);
                } else {
                    for (int r = q * m; r < (q + 1) * m; r += mm.box_rows)
                        tma_load_2d(tile + (size_t)r * W, &mm.in, x0, y0 + r, &bars[q]);
                }
            }
        }
        // every row of the line enters the sweep (stencil halos and closure rows included), so
        // every chunk has to land; for the product, each thread scales its own rows first
        bool ok = true;
        for (int q = 0; q < P; ++q) ok = mbar_wait(&bars[q], par) && ok;
        if (!ok) atomicExch(&failed, 1);
        // FP64: the per-thread global accesses below go in batches of kB rows, every load of a
        // batch issued before its first use (measured 1.5 % faster); FP32 keeps one row at a
        // time (the batch's registers would cost it a CTA per SM)
        constexpr int kB = 8;
        if (o == 1 && ok) {
            if constexpr (sizeof(S) == 8) {
                for (int j0 = 0; j0 < m; j0 += kB) {
                    const int nb = (m - j0 < kB) ? m - j0 : kB;
                    Pack<S, V> q[kB];
#pragma unroll
                    for (int b = 0; b < kB; ++b)
                        if (b < nb) q[b] = ldv<S, V>(uj + ob + (size_t)(j0 + b) * kSZ);
#pragma unroll
                    for (int b = 0; b < kB; ++b) {
                        if (b < nb) {
                            Pack<S, V> t = ldv<S, V>(tile + ot + (size_t)(j0 + b) * W);
#pragma unroll
                            for (int i = 0; i < V; ++i) t.v[i] = t.v[i] * q[b].v[i];
                            stv<S, V>(tile + ot + (size_t)(j0 + b) * W, t);
                        }
                    }
                }
            } else {
#pragma unroll 4
                for (int j = 0; j < m; ++j) {
                    Pack<S, V> t = ldv<S, V>(tile + ot + (size_t)j * W);
                    const Pack<S, V> q = ldv<S, V>(uj + ob + (size_t)j * kSZ);
#pragma unroll
                    for (int i = 0; i < V; ++i) t.v[i] = t.v[i] * q.v[i];
                    stv<S, V>(tile + ot + (size_t)j * W, t);
                }
            }
        }
        __syncthreads();
        int unsafe = 0;
        Pack<A, V> hb[2], ha[2];
        if (!failed) read_halo<Tr, V, false>(op, TileView<S>{tile, 0, n, nullptr}, xs, k, c, hb, ha, unsafe);
        __syncthreads();
        if (failed) {
            for (int q = threadIdx.x; q < P; q += blockDim.x) mbar_wait(&bars[q], par);
            if (threadIdx.x == 0) record_timeout();
            return;
        }
        group_sweep<Tr, V, 0>(op, tile, xs, ends, k, c, hb, ha, unsafe);
        // epilogue on this thread's rows (the sweep leaves them in the tile): o = 0 writes
        // -1/2 u_j r, the others add their weight times r to what is there (split-precision
        // sweeps leave FP64 results: their epilogue runs in FP64)
        if constexpr (sizeof(S) == 8) {
            using E = std::conditional_t<Tr::kDF, double, A>;
            const E wgt = (o == 2) ? E(ta.nu) : E(-0.5);
            const S *srcb = (o == 0) ? uj : out;
            for (int j0 = 0; j0 < m; j0 += kB) {
                const int nb = (m - j0 < kB) ? m - j0 : kB;
                Pack<S, V> q[kB];
#pragma unroll
                for (int b = 0; b < kB; ++b)
                    if (b < nb) q[b] = ldv<S, V>(srcb + ob + (size_t)(j0 + b) * kSZ);
#pragma unroll
                for (int b = 0; b < kB; ++b) {
                    if (b < nb) {
                        const Pack<S, V> r = ldv<S, V>(tile + ot + (size_t)(j0 + b) * W);
                        Pack<S, V> x;
#pragma unroll
                        for (int i = 0; i < V; ++i)
                            x.v[i] = (o == 0) ? S(wgt * E(q[b].v[i]) * E(r.v[i]))
                                              : S(mad(wgt, E(r.v[i]), E(q[b].v[i])));
                        stv<S, V>(out + ob + (size_t)(j0 + b) * kSZ, x);
                    }
                }
            }
        } else if (o == 0) {
            const A h = A(-0.5);
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const Pack<S, V> r = ldv<S, V>(tile + ot + (size_t)j * W);
                const Pack<S, V> q = ldv<S, V>(uj + ob + (size_t)j * kSZ);
                Pack<S, V> x;
#pragma unroll
                for (int i = 0; i < V; ++i) x.v[i] = S(h * A(q.v[i]) * A(r.v[i]));
                stv<S, V>(out + ob + (size_t)j * kSZ, x);
            }
        } else {
            const A wgt = (o == 1) ? A(-0.5) : A(ta.nu);
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const Pack<S, V> r = ldv<S, V>(tile + ot + (size_t)j * W);
                S *po = out + ob + (size_t)j * kSZ;
                Pack<S, V> x = ldv<S, V>(po);
#pragma unroll
                for (int i = 0; i < V; ++i) x.v[i] = S(mad(wgt, A(r.v[i]), A(x.v[i])));
                stv<S, V>(po, x);
            }
        }
        // every thread is done with the tile, the scratch rows and `ends` before the next
        // sweep's copies (async proxy) overwrite them
        fence_async_smem();
        __syncthreads();
    }
}

// Persistent variant: each CTA walks units (W lines of a group) blockIdx.x, +gridDim.x, ...
// through `nbuf` tile buffers; the TMA copies of a unit are issued `nbuf` units ahead, so HBM
// reads stay in flight while the threads sweep.
template <typename Tr, int V, int MODE>
__global__ void __launch_bounds__(kMaxResidentP * 32) k_resident_pipe(const __grid_constant__ DevOp op,
                                                                      const __grid_constant__ TileMaps tm,
                                                                      const typename Tr::S *__restrict__ in,
                                                                      typename Tr::S *__restrict__ out, int nbuf) {
    using S = typename Tr::S;
    constexpr int W = Tr::W;
    constexpr int tpc = W / V;
    constexpr int parts = kSZ / W;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ int failed;
    const int n = op.n, P = op.P;
    const long long U = (long long)op.ngroups * parts;
    const int k = threadIdx.x / tpc, c = (threadIdx.x % tpc) * V;
    const size_t tile_elems = (size_t)n * W;
    const uint32_t tile_bytes = (uint32_t)tile_bytes_of(n, sizeof(S), W);
    S *tiles = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + (size_t)nbuf * tile_bytes);
    double *ends = reinterpret_cast<double *>(smem + (size_t)nbuf * tile_bytes + xs_bytes_of(sizeof(S), W));
    uint64_t *bars = reinterpret_cast<uint64_t *>(ends + (size_t)2 * P * W);
    if constexpr (W < kSZ) {
        if ((smem_u32(tiles) & 127u) != 0) {   // see k_resident
            if (threadIdx.x == 0) atomicExch(&g_device_status, (int)TDS_ERR_CUDA);
            return;
        }
    }
    // first element of unit u's lines, and its (line, row) coordinates in the [rows][32] view
    auto unit_ofs = [&](long long u) { return (size_t)(u / parts) * n * kSZ + (size_t)(u % parts) * W; };
    auto unit_x0 = [&](long long u) { return (int)(u % parts) * W; };
    auto unit_y0 = [&](long long u) { return (int)((u / parts) * n); };
    auto issue_load = [&](long long u, int b) {
        S *tile = tiles + (size_t)b * tile_elems;
        mbar_expect_tx(&bars[b], tile_bytes);
        if constexpr (W == kSZ) {
            bulk_g2s(tile, in + unit_ofs(u), tile_bytes, &bars[b]);
        } else {
            for (int r = 0; r < n; r += tm.box_rows)
                tma_load_2d(tile + (size_t)r * W, &tm.in, unit_x0(u), unit_y0(u) + r, &bars[b]);
        }
    };

    if (threadIdx.x == 0) {
        failed = 0;
        for (int b = 0; b < nbuf; ++b) mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int b = 0; b < nbuf; ++b) {
            const long long u = blockIdx.x + (long long)b * gridDim.x;
            if (u >= U) break;
            issue_load(u, b);
        }
    }
    for (int it = 0;; ++it) {
        const long long u = blockIdx.x + (long long)it * gridDim.x;
        if (u >= U) break;
        const int b = it % nbuf;
        S *tile = tiles + (size_t)b * tile_elems;
        const bool ok = mbar_wait(&bars[b], (uint32_t)((it / nbuf) & 1));
        if (!ok) atomicExch(&failed, 1);
        int unsafe = 0;
        Pack<typename Tr::A, V> hb[2], ha[2];
        if (MODE == 0 && ok) read_halo<Tr, V, false>(op, TileView<S>{tile, 0, n, in + unit_ofs(u)}, xs, k, c, hb, ha, unsafe);
        __syncthreads();
        if (failed) {
            // drain every copy still in flight into this CTA's buffers, then give up
            for (int d = threadIdx.x; d < nbuf; d += blockDim.x)
                if (blockIdx.x + (long long)(it + d) * gridDim.x < U)
                    mbar_wait(&bars[(it + d) % nbuf], (uint32_t)(((it + d) / nbuf) & 1));
            if (threadIdx.x == 0) record_timeout();
            return;
        }
        group_sweep<Tr, V, MODE>(op, tile, xs, ends, k, c, hb, ha, unsafe);
        S *og = out + unit_ofs(u);
        if (!kBulkStore<Tr>) {
            const size_t ot = (size_t)k * op.m * W + c, ob = (size_t)k * op.m * kSZ + c;
#pragma unroll 4
            for (int j = 0; j < op.m; ++j)
                stv<S, V>(og + ob + (size_t)j * kSZ, ldv<S, V>(tile + ot + (size_t)j * W));
        }
        // this thread's tile accesses are ordered before the async proxy (bulk store, refill)
        fence_async_smem();
        __syncthreads();   // every thread is done with this tile, the scratch rows and `ends`
        if (threadIdx.x == 0) {
            if (kBulkStore<Tr>) {
                if constexpr (W == kSZ) {
                    bulk_s2g(og, tile, tile_bytes);
                } else {
                    for (int r = 0; r < n; r += tm.box_rows)
                        tma_store_2d(&tm.out, unit_x0(u), unit_y0(u) + r, tile + (size_t)r * W);
                }
                bulk_commit();
            }
            const long long un = u + (long long)nbuf * gridDim.x;
            if (un < U) {
                // the buffer is refilled only after the store has read it
                if (kBulkStore<Tr>) bulk_wait_read();
                issue_load(un, b);
            }
        }
    }
    if (kBulkStore<Tr> && threadIdx.x == 0) bulk_wait_read();
}

// ------------------------------------------------------------------------------------------
// SEGMENTED pipeline, for lines whose group does not fit in one CTA.  The line is cut into P'
// segments of sg rows (sg >= 64 and dividing the chunk length, so the segment boundaries
// include the chunk boundaries and, for sg >= 64, every boundary system decouples to rounding);
// `op` describes that partition.  One CTA (one warp, one lane per line) per segment of a group.
//   k_seg_forward : forward pass of the segment (halo rows beyond the segment from HBM),
//                   segment ends -> ws; with STORE_D the forward values d also go to `out`.
//   k_seg_backward: F_K and L_K from the two boundary 2x2 systems of the segment (ends of the
//                   neighbouring segments from ws), the forward values again (recomputed from
//                   the input, or read back from `out`), back-substitution, result to `out`.
// ------------------------------------------------------------------------------------------
template <typename Tr, bool STORE_D>
__global__ void __launch_bounds__(32) k_seg_forward(const __grid_constant__ DevOp op,
                                                    const typename Tr::S *__restrict__ in,
                                                    typename Tr::S *__restrict__ out,
                                                    double *__restrict__ ws) {
    using S = typename Tr::S;
    using A = typename Tr::A;
    static_assert(Tr::W == kSZ, "one warp per segment of a 32-line group");
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = op.n, m = op.m, P = op.P, c = threadIdx.x;
    const long long g = blockIdx.x / P;
    const int K = (int)(blockIdx.x % P);
    const size_t gofs = (size_t)g * n * kSZ;
    S *tile = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + tile_bytes_of(m, sizeof(S)));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + tile_bytes_of(m, sizeof(S)) + xs_bytes_of(sizeof(S)));
    const uint32_t bytes = (uint32_t)tile_bytes_of(m, sizeof(S));
    const int r0 = K * m;
    if (c == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_expect_tx(bar, bytes);
        bulk_g2s(tile, in + gofs + (size_t)r0 * kSZ, bytes, bar);
    }
    __syncwarp();
    if (!mbar_wait(bar, 0)) {
        if (c == 0) record_timeout();
        mbar_wait(bar, 0);
        return;
    }
    int unsafe = 0;
    Pack<A, 1> hb[2], ha[2];
    read_halo<Tr, 1, false>(op, TileView<S>{tile, r0, r0 + m, in + gofs}, xs, K, c, hb, ha, unsafe);
    __syncwarp();
    const int cls = chunk_class(op, K);
    S *row = tile + c;
    Pack<A, 1> dprev = zero_a<Tr, 1>(), Ssum = zero_a<Tr, 1>();
    Ends64<1> ex;
    forward_phase<Tr, 1, false>(op, row, xs, K, cls, c, hb, ha, dprev, Ssum, ex, unsafe);
    double e0[1], e1[1];
    chunk_ends<Tr, 1>(op, row, cls, dprev, Ssum, ex, e0, e1);
    double *e = ws + ((size_t)(g * P + K) * 2) * kSZ + c;
    e[0] = e0[0];
    e[kSZ] = e1[0];
    if (STORE_D) {
        S *o = out + gofs + (size_t)r0 * kSZ + c;
#pragma unroll 4
        for (int j = 0; j < m; ++j) o[(size_t)j * kSZ] = row[(size_t)j * kSZ];
    }
}

// FP32 segments: only their two ends are needed before the boundary systems, and each end
// depends on few rows -- row 0's back-swept value on the rows whose weight pi_j is above the
// plan's cut-off (j < jpi), and d_{m-1} on the last rows of the forward recurrence, whose
// influence decays like the product of its multipliers (the same rate as pi).  So this kernel
// copies in only the segment's first jpi + 3 rows and its last jpi + 11 rows (8 more rows to
// cover the closure rows at a closed line's end, whose multipliers need not contract, and 3 for
// the stencil), starting the tail recurrence from zero: the ends carry an error below 2^-30 of
// max|d| (the FP32 cut-off), and the input is read about 1.2 times in all instead of twice.
// One warp per segment of a group (lane = line); the two row ranges arrive as bulk copies,
// rows outside the segment (stencil halo) are read from HBM.
template <typename Tr>
__device__ __forceinline__ int seg_ends_rows(const DevOp &op, int cls, int &hb1, int &tb0) {
    const int m = op.m, jp = Tr::jpi(op, cls), tail = jp + 8;
    if (jp + tail >= m || jp + 3 >= m - tail - 3) {   // too short to split: the whole segment
        hb1 = m;
        tb0 = m;
        return m;
    }
    hb1 = jp + 3;
    tb0 = m - tail - 3;
    return hb1 + (m - tb0);
}

template <typename Tr>
__global__ void __launch_bounds__(32) k_seg_ends(const __grid_constant__ DevOp op,
                                                 const typename Tr::S *__restrict__ in,
                                                 double *__restrict__ ws) {
    using S = typename Tr::S;
    using A = typename Tr::A;
    static_assert(Tr::W == kSZ, "one warp per segment of a 32-line group");
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = op.n, m = op.m, P = op.P, c = threadIdx.x;
    const long long g = blockIdx.x / P;
    const int K = (int)(blockIdx.x % P);
    const int cls = chunk_class(op, K), J0 = K * m;
    const S *gl = in + (size_t)g * n * kSZ;                       // the group's rows
    const S *seg = gl + (size_t)J0 * kSZ;                          // this segment's rows
    int hb1, tb0;
    const int rows = seg_ends_rows<Tr>(op, cls, hb1, tb0);
    const bool split = hb1 < tb0;
    S *tile = reinterpret_cast<S *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)rows * kSZ * sizeof(S));
    if (c == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_expect_tx(bar, (uint32_t)((size_t)rows * kSZ * sizeof(S)));
        bulk_g2s(tile, seg, (uint32_t)((size_t)hb1 * kSZ * sizeof(S)), bar);
        if (split)
            bulk_g2s(tile + (size_t)hb1 * kSZ, seg + (size_t)tb0 * kSZ,
                     (uint32_t)((size_t)(m - tb0) * kSZ * sizeof(S)), bar);
    }
    __syncwarp();
    if (!mbar_wait(bar, 0)) {
        if (c == 0) record_timeout();
        mbar_wait(bar, 0);
        return;
    }
    // row r of the segment (r may lie outside it: the stencil's halo, from HBM)
    auto val = [&](int r) -> A {
        if (r >= 0 && r < hb1) return A(tile[(size_t)r * kSZ + c]);
        if (r >= tb0 && r < m) return A(tile[(size_t)(hb1 + r - tb0) * kSZ + c]);
        const int R = line_row(op, J0 + r);
        return (R >= 0) ? A(__ldg(gl + (size_t)R * kSZ + c)) : A(0);
    };
    const int jp = Tr::jpi(op, cls);
    auto sweep = [&](int jb, int je, A &dprev, A &Ssum, A &d0) {
        A w[kTaps];
#pragma unroll
        for (int i = 0; i < kTaps; ++i) w[i] = val(jb - 3 + i);
        for (int j = jb; j < je; ++j) {
            const A sv = stencil<A>(op, J0 + j, w);
            const A d = rowc<A>(op, kF, cls, j) * (sv - rowc<A>(op, kR, cls, j) * dprev);
            if (j == 0) d0 = d;
            if (j < jp) Ssum = mad(Tr::pi(op, cls, j), d, Ssum);
            dprev = d;
#pragma unroll
            for (int i = 0; i < kTaps - 1; ++i) w[i] = w[i + 1];
            w[kTaps - 1] = val(j + 4);
        }
    };
    // FP32 sweeps of closed lines: the four rows at each end of the line in FP64 (Ends64)
    const bool e64 = Tr::kE64 && op.e64;
    const bool head = e64 && K == 0, tail = e64 && K == P - 1;
    double x0 = 0.0, xl = 0.0;
    auto rows64 = [&](int jb, double d, double &Sx, double &dfirst) {
        Sx = 0.0;
        for (int t = 0; t < 4; ++t) {
            const int j = jb + t, J = J0 + j;
            const int e = (J < kEdgeRows) ? J : kEdgeRows + J - (n - kEdgeRows);
            double sv = 0.0;
#pragma unroll
            for (int o = 0; o < kTaps; ++o) sv = ::fma(op.edge[e][o], (double)val(j - 3 + o), sv);
            const size_t i = (size_t)cls * m + j;
            d = __ldg(op.fwd64 + 4 * i) * (sv - __ldg(op.fwd64 + 4 * i + 1) * d);
            Sx = ::fma(__ldg(op.fwd64 + 4 * i + 2), d, Sx);
            if (t == 0) dfirst = d;
        }
        return d;
    };
    A dprev = A(0), Ssum = A(0), d0 = A(0);
    const int ja = head ? 4 : 0;
    if (head) {
        double Sx, df;
        const double d3 = rows64(0, 0.0, Sx, df);
        x0 = ::fma(-__ldg(op.bwd64 + 2 * (size_t)cls * m + 1), Sx, df);
        dprev = A(d3);
    }
    if (!split) {
        sweep(ja, tail ? m - 4 : m, dprev, Ssum, d0);
    } else {
        sweep(ja, jp > ja ? jp : ja, dprev, Ssum, d0);
        dprev = A(0);
        sweep(tb0 + 3, tail ? m - 4 : m, dprev, Ssum, d0);
    }
    if (tail) {
        double Sx, df;
        xl = rows64(m - 4, (double)dprev, Sx, df);
        Ssum += A(Sx);
        dprev = A(xl);
    }
    A sa0, w0;
    Tr::bwd(op, cls, 0, sa0, w0);
    const A n1 = Tr::from_d(__ldg(op.n1 + cls));
    double *e = ws + ((size_t)(g * P + K) * 2) * kSZ + c;
    e[0] = head ? __ldg(op.n1 + cls) * ::fma(-__ldg(op.bwd64 + 2 * (size_t)cls * m + 1), (double)Ssum, x0)
                : Tr::to_d(n1 * (d0 - w0 * Ssum));
    e[kSZ] = tail ? xl : Tr::to_d(dprev);
}

template <typename Tr, bool RECOMPUTE>
__global__ void __launch_bounds__(32) k_seg_backward(const __grid_constant__ DevOp op,
                                                     const typename Tr::S *__restrict__ in,
                                                     typename Tr::S *__restrict__ out,
                                                     const double *__restrict__ ws) {
    using S = typename Tr::S;
    using A = typename Tr::A;
    static_assert(Tr::W == kSZ, "one warp per segment of a 32-line group");
    extern __shared__ __align__(128) unsigned char smem[];
    const int n = op.n, m = op.m, P = op.P, c = threadIdx.x;
    const long long g = blockIdx.x / P;
    const int K = (int)(blockIdx.x % P);
    const size_t gofs = (size_t)g * n * kSZ;
    S *tile = reinterpret_cast<S *>(smem);
    S *xs = reinterpret_cast<S *>(smem + tile_bytes_of(m, sizeof(S)));
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + tile_bytes_of(m, sizeof(S)) + xs_bytes_of(sizeof(S)));
    const uint32_t bytes = (uint32_t)tile_bytes_of(m, sizeof(S));
    const int r0 = K * m;
    // the input segment (to recompute the forward pass) or its stored forward values
    const S *src = RECOMPUTE ? in + gofs + (size_t)r0 * kSZ : out + gofs + (size_t)r0 * kSZ;
    if (c == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        mbar_expect_tx(bar, bytes);
        bulk_g2s(tile, src, bytes, bar);
    }
    // the two boundary systems of this segment, FP64
    const int R = 2 * P, prev = (K == 0) ? P - 1 : K - 1, next = (K == P - 1) ? 0 : K + 1;
    const double *eg = ws + (size_t)g * P * 2 * kSZ + c;
    const double e0K = eg[(size_t)(2 * K) * kSZ], e1K = eg[(size_t)(2 * K + 1) * kSZ];
    const double e1p = eg[(size_t)(2 * prev + 1) * kSZ], e0n = eg[(size_t)(2 * next) * kSZ];
    const double F64 = (e0K - __ldg(op.red + (size_t)kRedBa * R + K) * e1p) * __ldg(op.red + (size_t)kRedBinv * R + K);
    const double Fn = (e0n - __ldg(op.red + (size_t)kRedBa * R + next) * e1K) * __ldg(op.red + (size_t)kRedBinv * R + next);
    const double L64 = e1K - __ldg(op.red + (size_t)kRedBc * R + next) * Fn;
    __syncwarp();
    if (!mbar_wait(bar, 0)) {
        if (c == 0) record_timeout();
        mbar_wait(bar, 0);
        return;
    }
    const int cls = chunk_class(op, K);
    S *row = tile + c;
    if (RECOMPUTE) {
        int unsafe = 0;
        Pack<A, 1> hb[2], ha[2];
        read_halo<Tr, 1, false>(op, TileView<S>{tile, r0, r0 + m, in + gofs}, xs, K, c, hb, ha, unsafe);
        __syncwarp();
        Pack<A, 1> dprev = zero_a<Tr, 1>(), Ssum = zero_a<Tr, 1>();
        Ends64<1> ex;
        forward_phase<Tr, 1, false>(op, row, xs, K, cls, c, hb, ha, dprev, Ssum, ex, unsafe);
    }
    Pack<A, 1> F, L;
    F.v[0] = Tr::from_d(F64);
    L.v[0] = Tr::from_d(L64);
    backsub_phase<Tr, 1, false>(op, row, cls, F, L);
    S *o = out + gofs + (size_t)r0 * kSZ;
    if (kBulkStore<Tr>) {
        fence_async_smem();
        __syncwarp();
        if (c == 0) {
            bulk_s2g(o, tile, bytes);
            bulk_commit();
            bulk_wait_read();
        }
    } else {
#pragma unroll 4
        for (int j = 0; j < m; ++j) o[(size_t)j * kSZ + c] = row[(size_t)j * kSZ];
    }
}

template <typename Tr>
tds_status launch_segmented_t(const DevOp &op, const void *in, void *out, void *ws, cudaStream_t st) {
    using S = typename Tr::S;
    constexpr bool kFP64 = sizeof(S) == 8;   // FP64: store d (the sweep is FP64-pipe bound)
    const int smem = (int)(tile_bytes_of(op.m, sizeof(S)) + xs_bytes_of(sizeof(S)) + 16);
    auto kf = k_seg_forward<Tr, kFP64>;
    auto kb = k_seg_backward<Tr, !kFP64>;
    if (cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(kb, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    const unsigned grid = (unsigned)((long long)op.ngroups * op.P);
    if (kFP64) {
        kf<<<grid, 32, smem, st>>>(op, static_cast<const S *>(in), static_cast<S *>(out), static_cast<double *>(ws));
    } else {
        // the rows k_seg_ends copies in (seg_ends_rows), the largest over the chunk classes
        int rows = 0;
        for (int cl = 0; cl < (op.cls_each ? 1 : op.ncls); ++cl) {
            const int jp = op.jpi32[cl], tail = jp + 8;
            const int r = (jp + tail >= op.m || jp + 3 >= op.m - tail - 3) ? op.m : (jp + 3) + (tail + 3);
            rows = r > rows ? r : rows;
        }
        const int smem_e = (int)(tile_bytes_of(rows, sizeof(S)) + 16);
        auto ke = k_seg_ends<Tr>;
        if (cudaFuncSetAttribute(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_e) != cudaSuccess)
            return TDS_ERR_CUDA;
        ke<<<grid, 32, smem_e, st>>>(op, static_cast<const S *>(in), static_cast<double *>(ws));
    }
    kb<<<grid, 32, smem, st>>>(op, static_cast<const S *>(in), static_cast<S *>(out), static_cast<const double *>(ws));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

template <typename Tr, int V, int MODE>
tds_status launch_resident_t(const DevOp &op, const TileMaps &tm, const void *in, void *out, int smem,
                             cudaStream_t st) {
    using S = typename Tr::S;
    auto kern = k_resident<Tr, V, MODE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    const unsigned grid = (unsigned)((long long)op.ngroups * (kSZ / Tr::W));
    kern<<<grid, op.P * (Tr::W / V), smem, st>>>(op, tm, static_cast<const S *>(in), static_cast<S *>(out));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

template <typename Tr, int MODE>
tds_status launch_pipe_t(const DevOp &op, const TileMaps &tm, const void *in, void *out, int nbuf, int smem,
                         int grid, cudaStream_t st) {
    using S = typename Tr::S;
    auto kern = k_resident_pipe<Tr, 1, MODE>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    kern<<<grid, op.P * Tr::W, smem, st>>>(op, tm, static_cast<const S *>(in), static_cast<S *>(out), nbuf);
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

template <typename Tr>
tds_status launch_pipe_w(const tds_plan *p, int which, const TileMaps &tm, const void *in, void *out,
                         cudaStream_t st) {
    const DevOp &op = p->op[which];
    const int smem = (int)pipe_smem_bytes(p->n, p->P, p->dtype, p->pipe_nbuf, Tr::W);
    const long long units = (long long)op.ngroups * (kSZ / Tr::W);
    const int grid = units < p->pipe_grid ? (int)units : p->pipe_grid;
    if (op.adjoint == 2) return TDS_ERR_ARG;   // the solve alone runs resident or streaming
    return op.adjoint ? launch_pipe_t<Tr, 1>(op, tm, in, out, p->pipe_nbuf, smem, grid, st)
                      : launch_pipe_t<Tr, 0>(op, tm, in, out, p->pipe_nbuf, smem, grid, st);
}

template <typename Tr, int V>
tds_status launch_resident_v(const tds_plan *p, int which, const TileMaps &tm, const void *in, void *out,
                             cudaStream_t st) {
    const DevOp &op = p->op[which];
    if (op.adjoint == 2) {   // the solve alone: one line per thread
        if constexpr (V == 1) return launch_resident_t<Tr, 1, 2>(op, tm, in, out, p->resident_smem, st);
        else return TDS_ERR_ARG;
    }
    return op.adjoint ? launch_resident_t<Tr, V, 1>(op, tm, in, out, p->resident_smem, st)
                      : launch_resident_t<Tr, V, 0>(op, tm, in, out, p->resident_smem, st);
}

// Whether an FP64 plan's operator runs the split-precision sweep (TrSplit): the plan asks for it
// (tds_plan_set_arith) and the operator has the forward form (the stencil right-hand side:
// derivatives and their adjoints on periodic lines, the filter, the mid-point interpolation and
// its transpose on periodic lines).  The closed-line adjoints and the solve alone run native.
bool split_sweep(const tds_plan *p, const DevOp &op) {
    return p->dtype == TDS_F64 && p->split && op.adjoint == 0;
}

// cuTensorMapEncodeTiled, looked up once through the runtime (no link against the driver API).
using EncodeTiledFn = PFN_cuTensorMapEncodeTiled_v12000;
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// The field at `base` as a [rows][32] tensor with box [box_rows][w].
bool encode_rows(CUtensorMap *map, const void *base, tds_dtype dt, long long rows, int w, int box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t es = (dt == TDS_F64) ? 8 : 4;
    const cuuint64_t dims[2] = {(cuuint64_t)kSZ, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kSZ * es};
    const cuuint32_t box[2] = {(cuuint32_t)w, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, dt == TDS_F64 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
              const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


// Lines per thread (tds_plan::lanes): FP32 1, 2 or 4; FP64 1 or 2.  More lanes spread the per-row
// work (plan records, addressing, loop control) over more points and give each thread
// independent recurrences; fewer lanes give more threads.
// Tensor maps of this call's fields when the plan's CTAs hold fewer than 32 lines.
bool tile_maps(const tds_plan *p, const void *in, void *out, TileMaps *tm) {
    std::memset(tm, 0, sizeof(*tm));
    tm->box_rows = p->box_rows;
    if (p->width == kSZ) return true;
    const long long rows = (long long)p->n * (p->nlines / kSZ);
    if (!encode_rows(&tm->in, in, p->dtype, rows, p->width, p->box_rows)) return false;
    return p->dtype != TDS_F32 || encode_rows(&tm->out, out, p->dtype, rows, p->width, p->box_rows);
}


// ilv: one CTA per (unit, operator) (k_resident_ilv), else one CTA per unit sweeping the
// operators in turn (k_resident_multi)
template <typename Tr>
tds_status launch_multi_t(const MultiArgs &ma, const MultiMaps &mm, const void *in, int smem, bool ilv,
                          cudaStream_t st) {
    using S = typename Tr::S;
    auto kern = ilv ? k_resident_ilv<Tr> : k_resident_multi<Tr>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    const long long units = (long long)ma.op[0].ngroups * (kSZ / Tr::W);
    const unsigned grid = (unsigned)(ilv ? units * ma.count : units);
    kern<<<grid, ma.op[0].P * Tr::W, smem, st>>>(ma, mm, static_cast<const S *>(in));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

// Which form of the fused pass runs: one CTA per (unit, operator) -- measured faster for both
// precisions at 512^3 (FP64 5.53 -> 5.40 ms, FP32 0.540 -> 0.523 ms for D1 + D2 + D1^T) --
// unless TDS_MULTI_FORM = "seq" asks for the one-CTA-per-unit form (tuning)
bool multi_ilv() {
    if (const char *e = std::getenv("TDS_MULTI_FORM")) {
        if (std::strcmp(e, "seq") == 0) return false;
    }
    return true;
}

template <typename Tr, int V>
tds_status launch_transport_v(const TransportArgs &ta, const MultiMaps &mm, const void *ui, const void *uj,
                              void *out, int smem, cudaStream_t st) {
    using S = typename Tr::S;
    auto kern = k_resident_transport<Tr, V>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return TDS_ERR_CUDA;
    const unsigned grid = (unsigned)((long long)ta.op1.ngroups * (kSZ / Tr::W));
    kern<<<grid, ta.op1.P * Tr::W / V, smem, st>>>(ta, mm, static_cast<const S *>(ui), static_cast<const S *>(uj),
                                                    static_cast<S *>(out));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

// lanes: lines per thread as in launch_resident (whole-group CTAs only: FP32 1, 2 or 4, FP64 1
// or 2); a CTA keeps at least one warp
template <typename Tr>
tds_status launch_transport_t(const TransportArgs &ta, const MultiMaps &mm, const void *ui, const void *uj,
                              void *out, int smem, int lanes, cudaStream_t st) {
    if constexpr (Tr::W == kSZ) {
        const int threads = ta.op1.P * Tr::W;
        if constexpr (sizeof(typename Tr::S) == 4) {
            if (lanes == 4 && threads / 4 >= 32) return launch_transport_v<Tr, 4>(ta, mm, ui, uj, out, smem, st);
        }
        if (lanes >= 2 && threads / 2 >= 32) return launch_transport_v<Tr, 2>(ta, mm, ui, uj, out, smem, st);
    }
    return launch_transport_v<Tr, 1>(ta, mm, ui, uj, out, smem, st);
}

// ---- arithmetic families: the kernels of one trait family at the plan's CTA width ----
struct FamF64 {
    template <int W> using T = TrNative<double, W>;
    static constexpr bool kSplit = false;
    static constexpr int kMaxLanes = 2;
};
struct FamF32 {
    template <int W> using T = TrNative<float, W>;
    static constexpr bool kSplit = false;
    static constexpr int kMaxLanes = 4;
};
struct FamF32c {   // FP32 with FP64 closure rows (closed lines with a high end gain)
    template <int W> using T = TrNative<float, W, true>;
    static constexpr bool kSplit = false;
    static constexpr int kMaxLanes = 4;
};
struct FamSplit {
    template <int W> using T = TrSplit<W>;
    static constexpr bool kSplit = true;
    static constexpr int kMaxLanes = 1;
};

template <class Fam>
tds_status fam_resident(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    TileMaps tm;
    if (!tile_maps(p, in, out, &tm)) return TDS_ERR_CUDA;
    const int W = p->width;
    if constexpr (Fam::kSplit) {
        const DevOp &op = p->op[which];
        return W == 16 ? launch_resident_t<typename Fam::template T<16>, 1, 0>(op, tm, in, out, p->resident_smem, st)
             : W == 8  ? launch_resident_t<typename Fam::template T<8>, 1, 0>(op, tm, in, out, p->resident_smem, st)
                       : launch_resident_t<typename Fam::template T<kSZ>, 1, 0>(op, tm, in, out, p->resident_smem, st);
    } else {
        const int lanes = (p->op[which].adjoint == 2) ? 1 : p->lanes;
        if (W == 16) return launch_resident_v<typename Fam::template T<16>, 1>(p, which, tm, in, out, st);
        if (W == 8) return launch_resident_v<typename Fam::template T<8>, 1>(p, which, tm, in, out, st);
        if constexpr (Fam::kMaxLanes >= 4) {
            if (lanes == 4) return launch_resident_v<typename Fam::template T<kSZ>, 4>(p, which, tm, in, out, st);
        }
        return lanes == 2 ? launch_resident_v<typename Fam::template T<kSZ>, 2>(p, which, tm, in, out, st)
                          : launch_resident_v<typename Fam::template T<kSZ>, 1>(p, which, tm, in, out, st);
    }
}

template <class Fam>
tds_status fam_pipelined(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    TileMaps tm;
    if (!tile_maps(p, in, out, &tm)) return TDS_ERR_CUDA;
    const int W = p->width;
    return W == 16 ? launch_pipe_w<typename Fam::template T<16>>(p, which, tm, in, out, st)
         : W == 8  ? launch_pipe_w<typename Fam::template T<8>>(p, which, tm, in, out, st)
                   : launch_pipe_w<typename Fam::template T<kSZ>>(p, which, tm, in, out, st);
}

template <class Fam>
tds_status fam_multi(const tds_plan *const *plans, const int *which, int count, const void *in,
                     void *const *outs, cudaStream_t st) {
    const tds_plan *p = plans[0];
    MultiArgs ma;
    MultiMaps mm;
    std::memset(&ma, 0, sizeof(ma));
    std::memset(&mm, 0, sizeof(mm));
    ma.count = count;
    mm.box_rows = p->box_rows;
    const long long rows = (long long)p->n * (p->nlines / kSZ);
    for (int i = 0; i < count; ++i) {
        ma.op[i] = plans[i]->op[which[i]];
        ma.out[i] = outs[i];
        if (p->width < kSZ && p->dtype == TDS_F32 &&
            !encode_rows(&mm.out[i], outs[i], p->dtype, rows, p->width, p->box_rows))
            return TDS_ERR_CUDA;
    }
    if (p->width < kSZ && !encode_rows(&mm.in, in, p->dtype, rows, p->width, p->box_rows)) return TDS_ERR_CUDA;
    const int W = p->width, smem = p->resident_smem;
    const bool ilv = multi_ilv();
    return W == 16 ? launch_multi_t<typename Fam::template T<16>>(ma, mm, in, smem, ilv, st)
         : W == 8  ? launch_multi_t<typename Fam::template T<8>>(ma, mm, in, smem, ilv, st)
                   : launch_multi_t<typename Fam::template T<kSZ>>(ma, mm, in, smem, ilv, st);
}

template <class Fam>
tds_status fam_transport(const tds_plan *d1, const tds_plan *d2, const void *ui, const void *uj, double nu,
                         void *out, cudaStream_t st) {
    TransportArgs ta;
    MultiMaps mm;
    std::memset(&ta, 0, sizeof(ta));
    std::memset(&mm, 0, sizeof(mm));
    ta.op1 = d1->op[0];
    ta.op2 = d2->op[0];
    ta.nu = nu;
    mm.box_rows = d1->box_rows;
    if (d1->width < kSZ &&
        !encode_rows(&mm.in, ui, d1->dtype, (long long)d1->n * (d1->nlines / kSZ), d1->width, d1->box_rows))
        return TDS_ERR_CUDA;
    const int W = d1->width, smem = d1->resident_smem, L = d1->lanes;
    if constexpr (Fam::kSplit) {
        return W == 16 ? launch_transport_v<typename Fam::template T<16>, 1>(ta, mm, ui, uj, out, smem, st)
             : W == 8  ? launch_transport_v<typename Fam::template T<8>, 1>(ta, mm, ui, uj, out, smem, st)
                       : launch_transport_v<typename Fam::template T<kSZ>, 1>(ta, mm, ui, uj, out, smem, st);
    } else {
        return W == 16 ? launch_transport_t<typename Fam::template T<16>>(ta, mm, ui, uj, out, smem, L, st)
             : W == 8  ? launch_transport_t<typename Fam::template T<8>>(ta, mm, ui, uj, out, smem, L, st)
                       : launch_transport_t<typename Fam::template T<kSZ>>(ta, mm, ui, uj, out, smem, L, st);
    }
}

template <class Fam>
tds_status fam_segmented(const tds_plan *p, int which, const void *in, void *out, void *ws, cudaStream_t st) {
    const DevOp &op = which ? p->seg_adj : p->seg;
    if (!op.P || op.adjoint) return TDS_ERR_ARG;
    return launch_segmented_t<typename Fam::template T<kSZ>>(op, in, out, ws, st);
}

// This unit's status word, then reset (the device has been synchronised by the caller).
tds_status take_status() {
    int v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_device_status, sizeof(int)) != cudaSuccess) return TDS_ERR_CUDA;
    if (cudaMemcpyToSymbol(g_device_status, &zero, sizeof(int)) != cudaSuccess) return TDS_ERR_CUDA;
    return (tds_status)v;
}

} // namespace

// Entry points of one family's translation unit (tds_fam_<tag>.cu).
#define TDS_FAMILY_DECLARE(tag)                                                                          \
    tds_status launch_resident_##tag(const tds_plan *, int, const void *, void *, cudaStream_t);         \
    tds_status launch_pipelined_##tag(const tds_plan *, int, const void *, void *, cudaStream_t);        \
    tds_status launch_multi_##tag(const tds_plan *const *, const int *, int, const void *, void *const *, \
                                  cudaStream_t);                                                          \
    tds_status launch_transport_##tag(const tds_plan *, const tds_plan *, const void *, const void *,      \
                                      double, void *, cudaStream_t);                                      \
    tds_status launch_segmented_##tag(const tds_plan *, int, const void *, void *, void *, cudaStream_t); \
    tds_status status_##tag();
TDS_FAMILY_DECLARE(f64)
TDS_FAMILY_DECLARE(f32)
TDS_FAMILY_DECLARE(f32c)
TDS_FAMILY_DECLARE(split)

#define TDS_FAMILY_DEFINE(tag, Fam)                                                                        \
    tds_status launch_resident_##tag(const tds_plan *p, int w, const void *in, void *out, cudaStream_t st) { \
        return fam_resident<Fam>(p, w, in, out, st);                                                        \
    }                                                                                                       \
    tds_status launch_multi_##tag(const tds_plan *const *p, const int *w, int c, const void *in,            \
                                  void *const *o, cudaStream_t st) {                                        \
        return fam_multi<Fam>(p, w, c, in, o, st);                                                          \
    }                                                                                                       \
    tds_status launch_transport_##tag(const tds_plan *d1, const tds_plan *d2, const void *ui, const void *uj, \
                                      double nu, void *out, cudaStream_t st) {                              \
        return fam_transport<Fam>(d1, d2, ui, uj, nu, out, st);                                             \
    }                                                                                                       \
    tds_status status_##tag() { return take_status(); }

// the pipelined and segmented kernels exist for the native families
#define TDS_FAMILY_DEFINE_NATIVE(tag, Fam)                                                                 \
    TDS_FAMILY_DEFINE(tag, Fam)                                                                             \
    tds_status launch_pipelined_##tag(const tds_plan *p, int w, const void *in, void *out, cudaStream_t st) { \
        return fam_pipelined<Fam>(p, w, in, out, st);                                                       \
    }                                                                                                       \
    tds_status launch_segmented_##tag(const tds_plan *p, int w, const void *in, void *out, void *ws,        \
                                      cudaStream_t st) {                                                    \
        return fam_segmented<Fam>(p, w, in, out, ws, st);                                                   \
    }

} // namespace tds
