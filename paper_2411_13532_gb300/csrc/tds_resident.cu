// tds_resident.cu -- host side of the resident DistD2 kernels (tds_resident.cuh): shared-memory
// sizes, and the dispatch of each call to the translation unit of its arithmetic family
// (tds_fam_f64.cu, tds_fam_f32.cu, tds_fam_f32c.cu, tds_fam_split.cu), plus the self-test of the
// bounded waits and the device status word.
#include "tds_resident.cuh"

namespace tds {

size_t resident_smem_bytes(int n, int P, tds_dtype dtype, int w) {
    const size_t es = (dtype == TDS_F64) ? 8 : 4;
    return tile_bytes_of(n, es, w) + xs_bytes_of(es, w) + (size_t)2 * P * w * 8 + (size_t)P * 8;
}

int resident_box_rows(int n, int m, tds_dtype dtype, int w) {
    const size_t es = (dtype == TDS_F64) ? 8 : 4;
    if (w == kSZ) return m;
    int box = 0;
    for (int d = 256; d >= 1; --d)
        if (m % d == 0) { box = d; break; }
    // every box destination (chunk starts and box starts in the tile) 128-byte aligned
    if (((size_t)box * w * es) % 128 != 0 || ((size_t)m * w * es) % 128 != 0 || n % box != 0) return 0;
    return box;
}

size_t pipe_smem_bytes(int n, int P, tds_dtype dtype, int nbuf, int w) {
    const size_t es = (dtype == TDS_F64) ? 8 : 4;
    return (size_t)nbuf * tile_bytes_of(n, es, w) + xs_bytes_of(es, w) + (size_t)2 * P * w * 8 + (size_t)nbuf * 8;
}

bool runs_split(const tds_plan *p, int which) { return split_sweep(p, p->op[which]); }

tds_status launch_resident(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    if (split_sweep(p, p->op[which])) return launch_resident_split(p, which, in, out, st);
    if (p->dtype == TDS_F64) return launch_resident_f64(p, which, in, out, st);
    if (p->op[which].e64) return launch_resident_f32c(p, which, in, out, st);
    return launch_resident_f32(p, which, in, out, st);
}

tds_status launch_pipelined(const tds_plan *p, int which, const void *in, void *out, cudaStream_t st) {
    if (p->dtype == TDS_F64) return launch_pipelined_f64(p, which, in, out, st);
    if (p->op[which].e64) return launch_pipelined_f32c(p, which, in, out, st);
    return launch_pipelined_f32(p, which, in, out, st);
}

tds_status launch_resident_multi(const tds_plan *const *plans, const int *which, int count, const void *in,
                                 void *const *outs, cudaStream_t st) {
    if (count < 1 || count > kMaxMulti) return TDS_ERR_ARG;
    bool split = true, e64 = false;
    for (int i = 0; i < count; ++i) {
        split = split && split_sweep(plans[i], plans[i]->op[which[i]]);
        e64 = e64 || plans[i]->op[which[i]].e64;
    }
    if (split) return launch_multi_split(plans, which, count, in, outs, st);
    if (plans[0]->dtype == TDS_F64) return launch_multi_f64(plans, which, count, in, outs, st);
    if (e64) return launch_multi_f32c(plans, which, count, in, outs, st);
    return launch_multi_f32(plans, which, count, in, outs, st);
}

tds_status launch_resident_transport(const tds_plan *d1, const tds_plan *d2, const void *ui, const void *uj,
                                     double nu, void *out, cudaStream_t st) {
    if (split_sweep(d1, d1->op[0]) && split_sweep(d2, d2->op[0]))
        return launch_transport_split(d1, d2, ui, uj, nu, out, st);
    if (d1->dtype == TDS_F64) return launch_transport_f64(d1, d2, ui, uj, nu, out, st);
    if (d1->op[0].e64 || d2->op[0].e64) return launch_transport_f32c(d1, d2, ui, uj, nu, out, st);
    return launch_transport_f32(d1, d2, ui, uj, nu, out, st);
}

namespace {
// Self-test of the bounded-wait path: waits on an mbarrier whose phase nothing completes; the
// wait gives up after `limit_ns`, records TDS_ERR_TIMEOUT and the kernel returns normally.
__global__ void k_selftest_wait(unsigned long long limit_ns) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 2);   // two arrivals expected, none ever made
        fence_mbar_init();
    }
    __syncwarp();
    if (!mbar_wait(&bar, 0, limit_ns) && threadIdx.x == 0) record_timeout();
}
} // namespace

tds_status launch_selftest_wait(double seconds, cudaStream_t st) {
    if (!(seconds > 0.0) || seconds > 2.0) return TDS_ERR_ARG;
    k_selftest_wait<<<1, 32, 0, st>>>((unsigned long long)(seconds * 1e9));
    return cudaGetLastError() == cudaSuccess ? TDS_OK : TDS_ERR_CUDA;
}

size_t segmented_ws_bytes(const tds_plan *p) {
    return ((size_t)p->nlines * p->seg.P * 2 * sizeof(double) + 255) & ~(size_t)255;
}

tds_status launch_segmented(const tds_plan *p, int which, const void *in, void *out, void *ws, cudaStream_t st) {
    const DevOp &op = which ? p->seg_adj : p->seg;
    if (p->dtype == TDS_F64) return launch_segmented_f64(p, which, in, out, ws, st);
    if (op.e64) return launch_segmented_f32c(p, which, in, out, ws, st);
    return launch_segmented_f32(p, which, in, out, ws, st);
}

// The first non-zero status word among the translation units' (each is reset).
tds_status read_device_status() {
    if (cudaDeviceSynchronize() != cudaSuccess) return TDS_ERR_CUDA;
    const tds_status words[5] = {take_status(), status_f64(), status_f32(), status_f32c(), status_split()};
    for (tds_status w : words)
        if (w != TDS_OK) return w;
    return TDS_OK;
}

} // namespace tds
