// tds_reorder.cu -- permutations between the Cartesian layout and the direction layouts of
// the interleaved group data structure (Sec. 4.1: the layout is specific to the derivative
// direction and data is reordered when the direction changes; Table transport counts these
// reorders as one read and one write per point).
//
// With nx and ny multiples of 32, every 32-element row of the Cartesian, y and z layouts is a
// run of 32 consecutive x at fixed (y, z), and every row of the x layout is a run of 32
// consecutive y at fixed (x, z).  So:
//   Cartesian <-> y <-> z        : a permutation of whole rows (both sides coalesced);
//   x <-> {Cartesian, y, z}      : a 32 x 32 (x, y) tile transpose through shared memory.
// The ADD forms accumulate, out += reorder(in): the transport right-hand side (Sec. 5) adds the
// y and z terms back into the x-layout result with one pass each (Table transport counts a
// separate reorder and accumulation).
#include "tds_internal.h"

namespace tds {
namespace {

constexpr int R = kSZ;  // row length

// One 16-byte vector of T stored at dst, or added to what dst holds (ADD).
template <typename T, bool ADD>
__device__ __forceinline__ void put16(T *dst, float4 v) {
    if (ADD) {
        const float4 o = *reinterpret_cast<const float4 *>(dst);
        T *e = reinterpret_cast<T *>(&v);
        const T *f = reinterpret_cast<const T *>(&o);
#pragma unroll
        for (int u = 0; u < 16 / (int)sizeof(T); ++u) e[u] += f[u];
    }
    *reinterpret_cast<float4 *>(dst) = v;
}

// Offset of the row holding x = 32*xb .. 32*xb+31 at (y, z) in a layout whose rows run in x.
__device__ __forceinline__ size_t xrun_row(tds_layout L, int xb, int y, int z, int nx, int ny,
                                           int nz) {
    const size_t xg = (size_t)nx / R;
    switch (L) {
    case TDS_LAYOUT_CART: return (size_t)xb * R + (size_t)nx * ((size_t)y + (size_t)ny * z);
    case TDS_LAYOUT_Y: return (size_t)R * ((size_t)y + (size_t)ny * ((size_t)xb + xg * z));
    default: /* Z */ return (size_t)R * ((size_t)z + (size_t)nz * ((size_t)xb + xg * y));
    }
}

// Offset of the x-layout row holding y = 32*yb .. 32*yb+31 at (x, z).
__device__ __forceinline__ size_t xlayout_row(int x, int yb, int z, int nx, int ny) {
    const size_t yg = (size_t)ny / R;
    return (size_t)R * ((size_t)x + (size_t)nx * ((size_t)yb + yg * z));
}

// Row permutation between two x-run layouts, in 16-byte vectors: a block copies the rows of
// kRowsY consecutive y at one z; each thread moves kVecPerThread independent vectors (all
// loads issued before the stores, so several are in flight per thread).
constexpr int kRowsY = 8;
constexpr int kVecPerThread = 4;

template <typename T, bool ADD>
__global__ void __launch_bounds__(256) k_rows(const T *__restrict__ in, T *__restrict__ out, int nx,
                                             int ny, int nz, tds_layout from, tds_layout to) {
    constexpr int vpr = R * sizeof(T) / 16;      // 16-byte vectors per row
    constexpr int epv = 16 / sizeof(T);          // elements per vector
    const int xg = nx / R, z = blockIdx.y, y0 = blockIdx.x * kRowsY;
    const int ylim = (ny - y0 < kRowsY) ? ny - y0 : kRowsY;
    const int total = ylim * xg * vpr;
    for (int base = threadIdx.x; base < total; base += 256 * kVecPerThread) {
        float4 v[kVecPerThread];
        size_t dst[kVecPerThread];
#pragma unroll
        for (int u = 0; u < kVecPerThread; ++u) {
            const int idx = base + u * 256;
            dst[u] = (size_t)-1;
            if (idx < total) {
                const int vi = idx % vpr, rowi = idx / vpr;
                const int xb = rowi % xg, y = y0 + rowi / xg;
                v[u] = __ldg(reinterpret_cast<const float4 *>(in + xrun_row(from, xb, y, z, nx, ny, nz) + vi * epv));
                dst[u] = xrun_row(to, xb, y, z, nx, ny, nz) + vi * epv;
            }
        }
#pragma unroll
        for (int u = 0; u < kVecPerThread; ++u)
            if (dst[u] != (size_t)-1) put16<T, ADD>(out + dst[u], v[u]);
    }
}

// 32 x 32 (x, y) tile transposes between the x layout and an x-run layout, kTilesZ
// consecutive z per block (all loads of a block are issued before its stores).  Global memory
// moves in 16-byte vectors on both sides: a row of 32 elements is VPR vectors, a pass of 256
// threads covers 256/VPR rows of a tile; the shared tile is padded to 33 columns.
// grid (nx/32, ny/32, ceil(nz/kTilesZ)), 256 threads.  to_x selects the direction.
constexpr int kTilesZ = 4;

template <typename T, bool ADD>
__global__ void __launch_bounds__(256) k_transpose(const T *__restrict__ in, T *__restrict__ out,
                                                  int nx, int ny, int nz, tds_layout other,
                                                  int to_x) {
    constexpr int epv = 16 / sizeof(T);        // elements per 16-byte vector
    constexpr int vpr = R / epv;               // vectors per 32-element row
    constexpr int rpp = 256 / vpr;             // rows per pass
    __shared__ T tile[kTilesZ][R][R + 1];
    const int xb = blockIdx.x, yb = blockIdx.y, z0 = blockIdx.z * kTilesZ;
    const int vg = threadIdx.x % vpr, rr = threadIdx.x / vpr;
    const int nt = (nz - z0 < kTilesZ) ? nz - z0 : kTilesZ;
    for (int q = 0; q < nt; ++q) {
        const int z = z0 + q;
#pragma unroll
        for (int i = rr; i < R; i += rpp) {
            const T *src = to_x ? in + xrun_row(other, xb, yb * R + i, z, nx, ny, nz)
                                : in + xlayout_row(xb * R + i, yb, z, nx, ny);
            const float4 v = __ldg(reinterpret_cast<const float4 *>(src) + vg);
            const T *e = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int u = 0; u < epv; ++u) tile[q][i][vg * epv + u] = e[u];
        }
    }
    __syncthreads();
    for (int q = 0; q < nt; ++q) {
        const int z = z0 + q;
#pragma unroll
        for (int i = rr; i < R; i += rpp) {
            float4 v;
            T *e = reinterpret_cast<T *>(&v);
#pragma unroll
            for (int u = 0; u < epv; ++u) e[u] = tile[q][vg * epv + u][i];
            T *dst = to_x ? out + xlayout_row(xb * R + i, yb, z, nx, ny)
                          : out + xrun_row(other, xb, yb * R + i, z, nx, ny, nz);
            put16<T, ADD>(dst + vg * epv, v);
        }
    }
}

// from == to only with ADD (a plain copy is a memcpy): the identity row permutation of the
// Cartesian layout touches every element once, whatever layout the arrays hold.
template <typename T, bool ADD>
tds_status launch_t(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                    tds_layout to, cudaStream_t st) {
    const T *src = static_cast<const T *>(in);
    T *dst = static_cast<T *>(out);
    if (from == to) from = to = TDS_LAYOUT_CART;
    if (from != TDS_LAYOUT_X && to != TDS_LAYOUT_X) {
        dim3 grid((unsigned)((ny + kRowsY - 1) / kRowsY), (unsigned)nz);
        k_rows<T, ADD><<<grid, 256, 0, st>>>(src, dst, nx, ny, nz, from, to);
    } else {
        dim3 grid((unsigned)(nx / R), (unsigned)(ny / R), (unsigned)((nz + kTilesZ - 1) / kTilesZ));
        const int to_x = (to == TDS_LAYOUT_X);
        k_transpose<T, ADD><<<grid, 256, 0, st>>>(src, dst, nx, ny, nz, to_x ? from : to, to_x);
    }
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

} // namespace

tds_status launch_reorder(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                          tds_layout to, size_t elem, cudaStream_t st) {
    if (from == to) {
        const size_t bytes = (size_t)nx * ny * nz * elem;
        return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess
                   ? TDS_OK : TDS_ERR_CUDA;
    }
    return elem == 8 ? launch_t<double, false>(in, out, nx, ny, nz, from, to, st)
                     : launch_t<float, false>(in, out, nx, ny, nz, from, to, st);
}

tds_status launch_reorder_add(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                              tds_layout to, size_t elem, cudaStream_t st) {
    return elem == 8 ? launch_t<double, true>(in, out, nx, ny, nz, from, to, st)
                     : launch_t<float, true>(in, out, nx, ny, nz, from, to, st);
}

namespace {
// Fan-out copy: every 16-byte vector of `in` read once and written to each of `count` outputs
// (the traffic of the fused multi-operator pass: one read, one write per result).  Each thread
// loads kFanVec vectors before it stores them, so several loads are in flight per thread.
constexpr int kFanVec = 4;

struct FanArgs {
    void *out[kMaxMulti];
    int count;
};

__global__ void __launch_bounds__(256) k_fanout(const float4 *__restrict__ in, const __grid_constant__ FanArgs fa,
                                               size_t nvec) {
    const size_t stride = (size_t)gridDim.x * blockDim.x * kFanVec;
    for (size_t base = ((size_t)blockIdx.x * blockDim.x * kFanVec) + threadIdx.x; base < nvec; base += stride) {
        float4 v[kFanVec];
#pragma unroll
        for (int u = 0; u < kFanVec; ++u) {
            const size_t i = base + (size_t)u * blockDim.x;
            if (i < nvec) v[u] = __ldcs(in + i);
        }
        for (int o = 0; o < fa.count; ++o) {
            float4 *dst = static_cast<float4 *>(fa.out[o]);
#pragma unroll
            for (int u = 0; u < kFanVec; ++u) {
                const size_t i = base + (size_t)u * blockDim.x;
                if (i < nvec) dst[i] = v[u];
            }
        }
    }
}
} // namespace

tds_status launch_fanout(const void *in, void *const *outs, int count, size_t bytes, int nsm, cudaStream_t st) {
    FanArgs fa;
    for (int o = 0; o < kMaxMulti; ++o) fa.out[o] = (o < count) ? outs[o] : nullptr;
    fa.count = count;
    const size_t nvec = bytes / 16;
    const size_t need = (nvec + 256 * kFanVec - 1) / (256 * kFanVec);
    const unsigned grid = (unsigned)(need < (size_t)nsm * 8 ? (need ? need : 1) : (size_t)nsm * 8);
    k_fanout<<<grid, 256, 0, st>>>(static_cast<const float4 *>(in), fa, nvec);
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

} // namespace tds
