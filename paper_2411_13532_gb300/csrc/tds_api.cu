// tds_api.cu -- the extern "C" entry points of libtds (declared and documented in tds.h):
// argument and shape validation, variant selection, and the launches.
//
// Plan configuration, in finish_plan / tds_plan_set_variant:
//   width   : lines per resident CTA (32, 16, 8): FP32 the largest, FP64 the smallest that leaves
//             room for two CTAs per SM;
//   variant : AUTO = resident when the lines fit a CTA, unless FP64 CTAs would leave < 6 warps per
//             SM (then segmented); segmented when they do not fit; else streaming;
//   sub     : AUTO, FP32, resident CTAs with < 8 warps per SM: a finer-chunk copy of the plan runs in
//             its place (make_sub); every entry point launches through eff(plan), except
//             tds_deriv_noalloc (tds_noalloc.cu), which runs the plan's own chunks.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "tds_internal.h"

using namespace tds;

namespace {

int extent(int nx, int ny, int nz, tds_dir d) { return d == TDS_DIR_X ? nx : (d == TDS_DIR_Y ? ny : nz); }

bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bbytes && y < x + abytes;
}

bool aligned(const void *p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

size_t elem_size(tds_dtype dt) { return dt == TDS_F64 ? 8 : 4; }

size_t ws_need(const tds_plan *p) {
    if (p->sub) return ws_need(p->sub);
    if (p->variant == TDS_VARIANT_STREAMING) return streaming_ws_bytes(p);
    if (p->variant == TDS_VARIANT_SEGMENTED) {
        // the adjoint of a segmented plan runs the streaming pipeline
        const size_t a = segmented_ws_bytes(p), b = streaming_ws_bytes(p);
        return a > b ? a : b;
    }
    return 0;
}

// The plan whose kernels run for p: its finer-chunk plan when AUTO chose one (see make_sub).
const tds_plan *eff(const tds_plan *p) { return (p && p->sub) ? p->sub : p; }

// Warps per SM that the plan's resident CTAs leave (one line per thread): CTAs per SM by shared
// memory times warps per CTA.
int resident_warps_per_sm(const tds_plan *p) {
    if (!p->resident_smem) return 0;
    const int ctas = (int)((size_t)p->smem_sm / ((size_t)p->resident_smem + 1024));
    return ctas * (p->P * p->width / 32);
}

// Whether the resident kernel can run with w lines per CTA; two: and leave room for a second CTA
// on the SM.  Below 32 lines a CTA keeps at least two warps, its rows move as TMA tensor boxes
// (row coordinates below 2^31, 128-byte aligned box destinations).
bool resident_width_ok(const tds_plan *p, int w, bool two) {
    if (w != 32 && w != 16 && w != 8) return false;
    if ((long long)p->P * w > kMaxResidentP * kSZ) return false;   // one thread per line and chunk
    const size_t sm = resident_smem_bytes(p->n, p->P, p->dtype, w);
    if (sm > (size_t)p->smem_optin) return false;
    if (two && 2 * (sm + 1024) > (size_t)p->smem_sm) return false;
    if (w < kSZ) {
        const long long rows = (long long)p->n * (p->nlines / kSZ);
        if (p->P * w < 64 || rows >= (1ll << 31) || resident_box_rows(p->n, p->m, p->dtype, w) == 0)
            return false;
    }
    return true;
}

void configure_pipe(tds_plan *p);

// Resident kernel width (lines per CTA: 32, 16 or 8), among those that let two CTAs share an
// SM.  FP32 sweeps (bound by HBM) and split-precision FP64 sweeps (bound by the issue rate of the
// FP32 pipes): the largest such width (fewest per-CTA overheads, the longest contiguous copies;
// measured for the split FP64 fused pass at 512^3: 16 lines 3.28 ms, 8 lines 4.21 ms).  Native
// FP64 sweeps are bound by the FP64 pipe: on periodic lines the smallest (most CTAs per SM keep
// the pipe busy through each CTA's copy and reduced-system phases); on closed lines the largest
// too, so that the first and last chunks' closure rows do not run on a few lanes of a warp
// whose other lanes wait (measured at 512^3, P = 8, D1 / D2: 8 lines 2.197 / 2.179 ms, 16 lines
// 2.099 / 2.158, 32 lines 2.082 / 2.168).  Else 32 if a whole group fits at all.  The rule follows
// the sweep the plan's operator actually runs: a split-precision plan whose operator has no split
// sweep runs native and takes the native rule.
void pick_width(tds_plan *p) {
    p->width = 0;
    if (p->dtype == TDS_F64 && !runs_split(p, 0) && p->bc == TDS_BC_PERIODIC) {
        for (int w = 8; w <= kSZ; w *= 2)
            if (resident_width_ok(p, w, true)) { p->width = w; break; }
    } else {
        for (int w = kSZ; w >= 8; w /= 2)
            if (resident_width_ok(p, w, true)) { p->width = w; break; }
    }
    if (!p->width && resident_width_ok(p, kSZ, false)) p->width = kSZ;
    p->resident_smem = p->width ? (int)resident_smem_bytes(p->n, p->P, p->dtype, p->width) : 0;
    p->box_rows = p->width ? resident_box_rows(p->n, p->m, p->dtype, p->width) : 0;
    configure_pipe(p);
}

// Persistent pipelined kernel at the plan's width: two tile buffers per CTA (one in use, one
// loading) when they fit, else one; as many such CTAs as fit on every SM.  TDS_PIPE_NBUF (1..4)
// overrides the buffer count (tuning).
void configure_pipe(tds_plan *p) {
    p->pipe_nbuf = 0;
    p->pipe_grid = 0;
    if (!p->width) return;
    int want = 2;
    if (const char *e = std::getenv("TDS_PIPE_NBUF")) {
        const int v = std::atoi(e);
        if (v >= 1 && v <= 4) want = v;
    }
    for (int nb = want; nb >= 1; --nb)
        if (pipe_smem_bytes(p->n, p->P, p->dtype, nb, p->width) <= (size_t)p->smem_optin) {
            p->pipe_nbuf = nb;
            break;
        }
    if (!p->pipe_nbuf) return;
    const size_t per = pipe_smem_bytes(p->n, p->P, p->dtype, p->pipe_nbuf, p->width);
    const int ctas = (int)((size_t)p->smem_sm / (per + 1024));
    p->pipe_grid = p->nsm * (ctas > 0 ? ctas : 1);
}

// Arguments of one call (device buffers): TDS_OK or the error to return before any launch.
tds_status check_call(const tds_plan *p, const void *in, const void *out, const void *ws, size_t ws_bytes) {
    if (!p || !in || !out) return TDS_ERR_ARG;
    if (!aligned(in, 16) || !aligned(out, 16)) return TDS_ERR_ARG;
    const size_t bytes = (size_t)p->n * p->nlines * elem_size(p->dtype);
    if (overlaps(in, bytes, out, bytes)) return TDS_ERR_ALIAS;
    const size_t need = ws_need(p);
    if (need) {
        if (!ws || ws_bytes < need || !aligned(ws, 256)) return TDS_ERR_WORKSPACE;
        if (overlaps(ws, need, in, bytes) || overlaps(ws, need, out, bytes)) return TDS_ERR_ALIAS;
    }
    return TDS_OK;
}

// The plan's variant on device buffers (arguments already checked).  which: 0 the derivative,
// 1 its adjoint, 2 the solve alone (resident when the lines fit a CTA, else streaming).
tds_status launch(const tds_plan *p, int which, const void *in, void *out, void *ws, cudaStream_t st) {
    if (p->sub) return launch(p->sub, which, in, out, ws, st);
    if (which == 2) {
        if (p->variant != TDS_VARIANT_STREAMING && p->resident_smem) return launch_resident(p, 2, in, out, st);
        return launch_streaming(p, 2, in, out, ws, st);
    }
    if (p->variant == TDS_VARIANT_RESIDENT) return launch_resident(p, which, in, out, st);
    if (p->variant == TDS_VARIANT_PIPELINED) return launch_pipelined(p, which, in, out, st);
    if (p->variant == TDS_VARIANT_SEGMENTED) {
        // the adjoint: on the segment partition when it has the forward form (periodic lines),
        // else resident when CTAs holding the lines leave at least 4 warps per SM (measured, FP64
        // closed lines of 512 at P = 1: one 32-thread CTA per SM took 8.3 ms where the forward
        // pass takes 1.9), else the streaming pipeline
        if (which == 0 || p->seg_adj.P) return launch_segmented(p, which, in, out, ws, st);
        if (p->resident_smem && resident_warps_per_sm(p) >= 4) return launch_resident(p, which, in, out, st);
    }
    return launch_streaming(p, which, in, out, ws, st);
}

tds_status run(const tds_plan *p, int which, const void *in, void *out, void *ws, size_t ws_bytes,
               void *stream) {
    if (p && p->band && which != 2) return TDS_ERR_ARG;   // a band plan has no stencil
    const tds_status s = check_call(p, in, out, ws, ws_bytes);
    if (s != TDS_OK) return s;
    return launch(p, which, in, out, ws, static_cast<cudaStream_t>(stream));
}

// The plan restricted to groups [g0, g1) of its lines: the same operator arrays, fewer lines.
// Groups are independent and contiguous (group g occupies elements [g n 32, (g+1) n 32)), so
// the slab runs on the buffers offset by g0 n 32 elements.
tds_plan slab_of(const tds_plan *p, int g0, int g1) {
    tds_plan q = *eff(p);
    q.sub = nullptr;
    q.nlines = (g1 - g0) * kSZ;
    for (DevOp *o : {&q.op[0], &q.op[1], &q.op[2], &q.seg, &q.seg_adj}) {
        o->nlines = q.nlines;
        o->ngroups = g1 - g0;
    }
    return q;
}

// Host buffers: the lines are cut into up to kHostSlabs slabs of whole groups; slab s is copied
// in on the plan's input copy stream, computed on `stream` once it has landed, and copied out on
// the output copy stream once computed, so the copies of one slab overlap the compute of the
// next.  Ordered on `stream`: the call starts after the work already queued there, and work
// queued after it starts once host_out is complete.
tds_status run_host(const tds_plan *p, int which, const void *host_in, void *host_out, void *d_in,
                    void *d_out, void *ws, size_t ws_bytes, void *stream) {
    if (!p || !host_out || !d_in || !d_out || p->band) return TDS_ERR_ARG;
    tds_status s = check_call(p, d_in, d_out, ws, ws_bytes);
    if (s != TDS_OK) return s;
    const size_t gbytes = (size_t)p->n * kSZ * elem_size(p->dtype);
    const int G = p->nlines / kSZ;
    const int S = G < kHostSlabs ? G : kHostSlabs;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const cudaEvent_t *ev = p->ev;
    auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    if (!ok(cudaEventRecord(ev[0], st)) || !ok(cudaStreamWaitEvent(p->copy_in, ev[0], 0)) ||
        !ok(cudaStreamWaitEvent(p->copy_out, ev[0], 0)))
        return TDS_ERR_CUDA;
    for (int k = 0; k < S; ++k) {
        const int g0 = (int)((long long)G * k / S), g1 = (int)((long long)G * (k + 1) / S);
        const size_t off = (size_t)g0 * gbytes, len = (size_t)(g1 - g0) * gbytes;
        char *di = static_cast<char *>(d_in) + off;
        char *dout = static_cast<char *>(d_out) + off;
        if (host_in) {
            if (!ok(cudaMemcpyAsync(di, static_cast<const char *>(host_in) + off, len, cudaMemcpyHostToDevice,
                                    p->copy_in)) ||
                !ok(cudaEventRecord(ev[2 + k], p->copy_in)) || !ok(cudaStreamWaitEvent(st, ev[2 + k], 0)))
                return TDS_ERR_CUDA;
        }
        const tds_plan q = slab_of(p, g0, g1);
        s = launch(&q, which, di, dout, ws, st);
        if (s != TDS_OK) return s;
        if (!ok(cudaEventRecord(ev[2 + kHostSlabs + k], st)) ||
            !ok(cudaStreamWaitEvent(p->copy_out, ev[2 + kHostSlabs + k], 0)) ||
            !ok(cudaMemcpyAsync(static_cast<char *>(host_out) + off, dout, len, cudaMemcpyDeviceToHost,
                                p->copy_out)))
            return TDS_ERR_CUDA;
    }
    if (!ok(cudaEventRecord(ev[1], p->copy_out)) || !ok(cudaStreamWaitEvent(st, ev[1], 0))) return TDS_ERR_CUDA;
    return TDS_OK;
}

// Shape rules shared by every plan (TDS_ERR_SHAPE).
tds_status check_shape(int nx, int ny, int nz, tds_dir dir, int P) {
    if (nx < 1 || ny < 1 || nz < 1) return TDS_ERR_SHAPE;
    const int n = extent(nx, ny, nz, dir);
    const long long lines = (long long)nx * ny * nz / n;
    if (n < 8 || n % P != 0 || n / P < 4 || lines % kSZ != 0 || lines > (1ll << 31) - 1 ||
        (long long)n * lines > (1ll << 40))
        return TDS_ERR_SHAPE;
    return TDS_OK;
}

tds_plan *new_plan(int nx, int ny, int nz, tds_dir dir, tds_bc bc, int P, tds_dtype dtype, tds_reduced mode) {
    tds_plan *p = new (std::nothrow) tds_plan;
    if (!p) return nullptr;
    std::memset(p, 0, sizeof(*p));
    const int n = extent(nx, ny, nz, dir);
    p->nx = nx; p->ny = ny; p->nz = nz; p->dir = dir; p->bc = bc; p->P = P;
    p->dtype = dtype; p->mode = mode;
    p->n = n; p->m = n / P; p->nlines = (int)((long long)nx * ny * nz / n);
    return p;
}

// The operators (host preprocessing and upload), the kernel configuration for this device, the
// host entry points' streams and events, and the AUTO variant; destroys p on failure.
tds_status finish_plan(tds_plan *p, tds_plan **out) {
    const tds_dtype dtype = p->dtype;
    tds_status s = build_plan(p);
    if (s != TDS_OK) { tds_plan_destroy(p); return s; }

    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        tds_plan_destroy(p);
        return TDS_ERR_CUDA;
    }
    int smem_sm = 0, nsm = 0;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        tds_plan_destroy(p);
        return TDS_ERR_CUDA;
    }
    p->smem_optin = optin;
    p->smem_sm = smem_sm;
    p->nsm = nsm;
    pick_width(p);
    // lines per thread in the resident kernels; TDS_RESIDENT_LANES overrides (tuning)
    p->lanes = 1;
    if (const char *e = std::getenv("TDS_RESIDENT_LANES")) {
        const int v = std::atoi(e);
        if (v == 1 || v == 2 || (v == 4 && dtype == TDS_F32)) p->lanes = v;
    }
    if (p->order == 4) p->lanes = 1;   // the half-point stencil forms run one line per thread
    if (cudaStreamCreateWithFlags(&p->copy_in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->copy_out, cudaStreamNonBlocking) != cudaSuccess) {
        tds_plan_destroy(p);
        return TDS_ERR_CUDA;
    }
    for (cudaEvent_t &e : p->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            tds_plan_destroy(p);
            return TDS_ERR_CUDA;
        }
    tds_plan_set_variant(p, TDS_VARIANT_AUTO);
    *out = p;
    return TDS_OK;
}

// AUTO, FP32: when the plan's resident CTAs would leave fewer than 8 warps per SM (long chunks:
// one warp per chunk and few CTAs per SM, e.g. P = 1 with 512- or 1024-point lines), the same
// operator on finer chunks, P x 2^k (chunks of at least 64 rows), runs in its place.  The result
// is the same to rounding: the reduced system over all chunk ends is solved exactly (EXACT mode
// only; the paper-drop approximation depends on the chunks).  Measured, FP32 D1 on 2^30 points:
// n = 512, P = 1: 0.60 -> 0.91 of the copy rate; n = 1024, P = 1: 0.26 -> 0.82.
void make_sub(tds_plan *p) {
    if (p->sub) { tds_plan_destroy(p->sub); p->sub = nullptr; }
    if (p->is_sub || p->dtype != TDS_F32 || p->mode != TDS_REDUCED_EXACT || p->band ||
        p->variant != TDS_VARIANT_RESIDENT || resident_warps_per_sm(p) >= 8)
        return;
    for (int s = 2; p->m % s == 0 && p->m / s >= 64 && p->P * s * 8 <= kMaxResidentP * kSZ; s *= 2) {
        tds_plan *c = new_plan(p->nx, p->ny, p->nz, p->dir, p->bc, p->P * s, p->dtype, p->mode);
        if (!c) return;
        c->order = p->order;
        c->h = p->h;
        c->is_sub = true;
        tds_plan *done = nullptr;
        if (finish_plan(c, &done) != TDS_OK) return;   // finish_plan destroyed c
        if (done->variant == TDS_VARIANT_RESIDENT && resident_warps_per_sm(done) >= 8) {
            p->sub = done;
            return;
        }
        tds_plan_destroy(done);
    }
}


} // namespace

extern "C" {

const char *tds_status_string(tds_status s) {
    switch (s) {
    case TDS_OK: return "ok";
    case TDS_ERR_ARG: return "invalid argument";
    case TDS_ERR_SHAPE: return "shape rule violated";
    case TDS_ERR_ALIAS: return "input and output overlap";
    case TDS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case TDS_ERR_CUDA: return "CUDA error";
    case TDS_ERR_TIMEOUT: return "device-side wait timed out";
    case TDS_ERR_NOMEM: return "out of memory";
    }
    return "unknown status";
}

tds_status tds_plan_create(tds_plan **out, int nx, int ny, int nz, tds_dir dir, int order,
                           tds_bc bc, int P, double h, tds_dtype dtype, int sz, tds_reduced mode) {
    if (!out) return TDS_ERR_ARG;
    *out = nullptr;
    if (dir < TDS_DIR_X || dir > TDS_DIR_Z || (order != 1 && order != 2) ||
        (bc != TDS_BC_PERIODIC && bc != TDS_BC_CLOSED) || (dtype != TDS_F64 && dtype != TDS_F32) ||
        (mode != TDS_REDUCED_EXACT && mode != TDS_REDUCED_PAPER_DROP) || sz != kSZ ||
        !(h > 0.0) || !std::isfinite(h) || P < 1)
        return TDS_ERR_ARG;
    const tds_status sh = check_shape(nx, ny, nz, dir, P);
    if (sh != TDS_OK) return sh;
    tds_plan *p = new_plan(nx, ny, nz, dir, bc, P, dtype, mode);
    if (!p) return TDS_ERR_NOMEM;
    p->order = order;
    p->h = h;
    return finish_plan(p, out);
}

tds_status tds_plan_create_filter(tds_plan **out, int nx, int ny, int nz, tds_dir dir, double alpha_f,
                                  tds_bc bc, int P, tds_dtype dtype, int sz, tds_reduced mode) {
    if (!out) return TDS_ERR_ARG;
    *out = nullptr;
    if (dir < TDS_DIR_X || dir > TDS_DIR_Z || (bc != TDS_BC_PERIODIC && bc != TDS_BC_CLOSED) ||
        (dtype != TDS_F64 && dtype != TDS_F32) ||
        (mode != TDS_REDUCED_EXACT && mode != TDS_REDUCED_PAPER_DROP) || sz != kSZ ||
        !(alpha_f > -0.5 && alpha_f < 0.5) || P < 1)
        return TDS_ERR_ARG;
    const tds_status sh = check_shape(nx, ny, nz, dir, P);
    if (sh != TDS_OK) return sh;
    tds_plan *p = new_plan(nx, ny, nz, dir, bc, P, dtype, mode);
    if (!p) return TDS_ERR_NOMEM;
    p->order = 3;
    p->h = alpha_f;   // the filter's parameter takes the grid spacing's place
    return finish_plan(p, out);
}

tds_status tds_plan_create_interp(tds_plan **out, int nx, int ny, int nz, tds_dir dir, tds_bc bc, int P,
                                  tds_dtype dtype, int sz, tds_reduced mode) {
    if (!out) return TDS_ERR_ARG;
    *out = nullptr;
    if (dir < TDS_DIR_X || dir > TDS_DIR_Z || (bc != TDS_BC_PERIODIC && bc != TDS_BC_CLOSED) ||
        (dtype != TDS_F64 && dtype != TDS_F32) ||
        (mode != TDS_REDUCED_EXACT && mode != TDS_REDUCED_PAPER_DROP) || sz != kSZ || P < 1)
        return TDS_ERR_ARG;
    const tds_status sh = check_shape(nx, ny, nz, dir, P);
    if (sh != TDS_OK) return sh;
    tds_plan *p = new_plan(nx, ny, nz, dir, bc, P, dtype, mode);
    if (!p) return TDS_ERR_NOMEM;
    p->order = 4;
    p->h = 1.0;
    return finish_plan(p, out);
}

tds_status tds_plan_create_band(tds_plan **out, int nx, int ny, int nz, tds_dir dir, const double *a,
                                const double *b, const double *c, tds_bc bc, int P, tds_dtype dtype,
                                int sz, tds_reduced mode) {
    if (!out) return TDS_ERR_ARG;
    *out = nullptr;
    if (!a || !b || !c || dir < TDS_DIR_X || dir > TDS_DIR_Z ||
        (bc != TDS_BC_PERIODIC && bc != TDS_BC_CLOSED) || (dtype != TDS_F64 && dtype != TDS_F32) ||
        (mode != TDS_REDUCED_EXACT && mode != TDS_REDUCED_PAPER_DROP) || sz != kSZ || P < 1)
        return TDS_ERR_ARG;
    const tds_status sh = check_shape(nx, ny, nz, dir, P);
    if (sh != TDS_OK) return sh;
    const int n = extent(nx, ny, nz, dir);
    for (int j = 0; j < n; ++j)
        if (!std::isfinite(a[j]) || !std::isfinite(b[j]) || !std::isfinite(c[j])) return TDS_ERR_ARG;
    tds_plan *p = new_plan(nx, ny, nz, dir, bc, P, dtype, mode);
    if (!p) return TDS_ERR_NOMEM;
    p->band = static_cast<double *>(std::malloc(sizeof(double) * 3 * (size_t)n));
    if (!p->band) { tds_plan_destroy(p); return TDS_ERR_NOMEM; }
    std::memcpy(p->band, a, sizeof(double) * n);
    std::memcpy(p->band + n, b, sizeof(double) * n);
    std::memcpy(p->band + 2 * n, c, sizeof(double) * n);
    p->order = 0;
    p->h = 1.0;
    return finish_plan(p, out);
}

tds_status tds_plan_set_variant(tds_plan *p, tds_variant v) {
    if (!p) return TDS_ERR_ARG;
    const bool autov = (v == TDS_VARIANT_AUTO);
    if (v == TDS_VARIANT_AUTO) {
        // resident unless, for FP64 sweeps (bound by the FP64 pipe, which needs warps), its CTAs
        // would leave fewer than 6 warps per SM (few chunks, large tiles) while the lines split
        // into at least two segments (one warp per segment keeps more warps per SM; measured:
        // 256^3 P = 1, 3 warps per SM, segmented 26 % faster; P = 2, 6 warps per SM, resident
        // 7 % faster).  FP32 sweeps stay resident (thin FP32 plans run on finer chunks instead,
        // make_sub), except lines long enough to need 8-line CTAs (n above ~1800): their
        // segments read the input ~1.2 times (k_seg_ends), which beats the few, narrow resident
        // CTAs (measured at n = 2048: 1.52x against 1.73x the time of a copy).  Then segmented,
        // else streaming.
        bool thin = false;
        if (p->dtype == TDS_F64 && p->resident_smem && p->seg.P >= 2) {
            const int ctas = (int)((size_t)p->smem_sm / ((size_t)p->resident_smem + 1024));
            thin = ctas * (p->P * p->width / 32) < 6;
        }
        if (p->dtype == TDS_F32 && p->resident_smem && p->width == 8 && p->seg.P >= 2) thin = true;
        v = (p->resident_smem && !thin) ? TDS_VARIANT_RESIDENT
          : p->seg.P ? TDS_VARIANT_SEGMENTED
          : p->resident_smem ? TDS_VARIANT_RESIDENT : TDS_VARIANT_STREAMING;
    }
    if (v == TDS_VARIANT_RESIDENT && !p->resident_smem) return TDS_ERR_ARG;
    if (v == TDS_VARIANT_PIPELINED && !p->pipe_nbuf) return TDS_ERR_ARG;
    if (v == TDS_VARIANT_SEGMENTED && !p->seg.P) return TDS_ERR_ARG;
    if (v != TDS_VARIANT_RESIDENT && v != TDS_VARIANT_STREAMING && v != TDS_VARIANT_PIPELINED &&
        v != TDS_VARIANT_SEGMENTED)
        return TDS_ERR_ARG;
    p->variant = v;
    // AUTO may hand the work to finer chunks; a variant the caller fixes runs on the plan's own
    if (autov) {
        make_sub(p);
    } else if (p->sub) {
        tds_plan_destroy(p->sub);
        p->sub = nullptr;
    }
    return TDS_OK;
}

tds_status tds_plan_set_width(tds_plan *p, int lines) {
    if (!p || !resident_width_ok(p, lines, false)) return TDS_ERR_ARG;
    if (p->sub) {   // a width the caller fixes applies to the plan's own chunks
        tds_plan_destroy(p->sub);
        p->sub = nullptr;
    }
    p->width = lines;
    p->resident_smem = (int)resident_smem_bytes(p->n, p->P, p->dtype, lines);
    p->box_rows = resident_box_rows(p->n, p->m, p->dtype, lines);
    configure_pipe(p);
    return TDS_OK;
}

tds_status tds_plan_set_arith(tds_plan *p, tds_arith arith) {
    if (!p || p->dtype != TDS_F64 || p->band || (arith != TDS_ARITH_NATIVE && arith != TDS_ARITH_SPLIT))
        return TDS_ERR_ARG;
    const int split = (arith == TDS_ARITH_SPLIT) ? 1 : 0;
    if (split == p->split) return TDS_OK;
    // the width rule follows the arithmetic; AUTO chooses the variant again for that width
    p->split = split;
    pick_width(p);
    return tds_plan_set_variant(p, TDS_VARIANT_AUTO);
}

tds_status tds_plan_info(const tds_plan *q, int *n, int *nlines, int *P, int *variant, int *smem) {
    if (!q) return TDS_ERR_ARG;
    if (n) *n = q->n;
    if (nlines) *nlines = q->nlines;
    if (P) *P = q->P;
    const tds_plan *p = eff(q);   // the kernels that run
    if (variant) *variant = (int)p->variant;
    if (smem)
        *smem = p->variant == TDS_VARIANT_RESIDENT ? p->resident_smem
              : p->variant == TDS_VARIANT_PIPELINED ? (int)pipe_smem_bytes(p->n, p->P, p->dtype, p->pipe_nbuf, p->width)
              : 0;
    return TDS_OK;
}

tds_status tds_plan_run_chunks(const tds_plan *p, int *chunks) {
    if (!p || !chunks) return TDS_ERR_ARG;
    *chunks = eff(p)->P;
    return TDS_OK;
}

tds_status tds_plan_width(const tds_plan *p, int *lines) {
    if (!p || !lines) return TDS_ERR_ARG;
    *lines = eff(p)->width;
    return TDS_OK;
}

tds_status tds_workspace_bytes(const tds_plan *p, size_t *bytes) {
    if (!p || !bytes) return TDS_ERR_ARG;
    *bytes = ws_need(p);
    return TDS_OK;
}

tds_status tds_deriv(const tds_plan *p, const void *in, void *out, void *ws, size_t ws_bytes,
                     void *stream) {
    return run(p, 0, in, out, ws, ws_bytes, stream);
}

tds_status tds_deriv_adjoint(const tds_plan *p, const void *g, void *out, void *ws,
                             size_t ws_bytes, void *stream) {
    return run(p, 1, g, out, ws, ws_bytes, stream);
}

tds_status tds_solve(const tds_plan *p, const void *d, void *x, void *ws, size_t ws_bytes, void *stream) {
    return run(p, 2, d, x, ws, ws_bytes, stream);
}

tds_status tds_deriv_thomas(const tds_plan *p, const void *in, void *out, void *stream) {
    if (!p || !in || !out || p->band || !p->thomas_mem) return TDS_ERR_ARG;
    if (!aligned(in, 16) || !aligned(out, 16)) return TDS_ERR_ARG;
    const size_t bytes = (size_t)p->n * p->nlines * elem_size(p->dtype);
    if (overlaps(in, bytes, out, bytes)) return TDS_ERR_ALIAS;
    return launch_thomas(p, in, out, static_cast<cudaStream_t>(stream));
}

tds_status tds_deriv_multi(int count, const tds_plan *const *plans, const int *adjoint, const void *in,
                           void *const *outs, void *ws, size_t ws_bytes, void *stream) {
    if (count < 1 || count > kMaxMulti || !plans || !adjoint || !outs) return TDS_ERR_ARG;
    if (!plans[0]) return TDS_ERR_ARG;
    const tds_plan *run_plans[kMaxMulti];   // the plans whose kernels run
    for (int i = 0; i < count; ++i) {
        if (!plans[i]) return TDS_ERR_ARG;
        run_plans[i] = eff(plans[i]);
    }
    const tds_plan *p0 = run_plans[0];
    const size_t bytes = (size_t)p0->n * p0->nlines * elem_size(p0->dtype);
    int which[kMaxMulti];
    bool fused = true;
    for (int i = 0; i < count; ++i) {
        const tds_plan *p = run_plans[i];
        if (!p || p->band || (adjoint[i] != 0 && adjoint[i] != 1)) return TDS_ERR_ARG;
        which[i] = adjoint[i];
        // every operator maps the same field shape in the same direction layout
        if (p->nx != p0->nx || p->ny != p0->ny || p->nz != p0->nz || p->dir != p0->dir ||
            p->dtype != p0->dtype)
            return TDS_ERR_ARG;
        const tds_status s = check_call(p, in, outs[i], ws, ws_bytes);
        if (s != TDS_OK) return s;
        for (int j = 0; j < i; ++j)
            if (overlaps(outs[i], bytes, outs[j], bytes)) return TDS_ERR_ALIAS;
        // one pass needs resident plans of one geometry and width, forward-form operators; split-
        // precision FP64 plans run one launch per operator (their sweeps, not HBM reads, bound
        // them: measured at 512^3, D1 + D2 + D1^T 2.93 ms as three launches, 3.30 ms fused)
        fused = fused && p->variant == TDS_VARIANT_RESIDENT && p->lanes == 1 && p->P == p0->P &&
                p->width == p0->width && p->op[which[i]].adjoint == 0 && !p->split;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (fused) return launch_resident_multi(run_plans, which, count, in, outs, st);
    for (int i = 0; i < count; ++i) {
        const tds_status s = launch(run_plans[i], which[i], in, outs[i], ws, st);
        if (s != TDS_OK) return s;
    }
    return TDS_OK;
}

tds_status tds_transport(const tds_plan *d1, const tds_plan *d2, const void *ui, const void *uj, double nu,
                         void *out, void *stream) {
    if (!d1 || !d2 || !ui || !uj || !out || d1->band || d2->band || d1->order != 1 || d2->order != 2)
        return TDS_ERR_ARG;
    d1 = eff(d1);   // the plans whose kernels run
    d2 = eff(d2);
    // one geometry: the same field in the same direction layout, cut the same way
    if (d1->nx != d2->nx || d1->ny != d2->ny || d1->nz != d2->nz || d1->dir != d2->dir ||
        d1->dtype != d2->dtype || d1->P != d2->P || d1->width != d2->width)
        return TDS_ERR_ARG;
    // the fused kernel is resident: a CTA must hold its lines of a group
    if (!d1->resident_smem || !d2->resident_smem) return TDS_ERR_ARG;
    if (!aligned(ui, 16) || !aligned(uj, 16) || !aligned(out, 16)) return TDS_ERR_ARG;
    const size_t bytes = (size_t)d1->n * d1->nlines * elem_size(d1->dtype);
    if (overlaps(out, bytes, ui, bytes) || overlaps(out, bytes, uj, bytes)) return TDS_ERR_ALIAS;
    return launch_resident_transport(d1, d2, ui, uj, nu, out, static_cast<cudaStream_t>(stream));
}

tds_status tds_deriv_host(const tds_plan *p, const void *host_in, void *host_out, void *d_in,
                          void *d_out, void *ws, size_t ws_bytes, void *stream) {
    return run_host(p, 0, host_in, host_out, d_in, d_out, ws, ws_bytes, stream);
}

tds_status tds_deriv_adjoint_host(const tds_plan *p, const void *host_g, void *host_out, void *d_in,
                                  void *d_out, void *ws, size_t ws_bytes, void *stream) {
    return run_host(p, 1, host_g, host_out, d_in, d_out, ws, ws_bytes, stream);
}

tds_status tds_reorder(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                       tds_layout to, tds_dtype dtype, int sz, void *stream) {
    if (!in || !out || sz != kSZ || (dtype != TDS_F64 && dtype != TDS_F32) ||
        from < TDS_LAYOUT_CART || from > TDS_LAYOUT_Z || to < TDS_LAYOUT_CART || to > TDS_LAYOUT_Z)
        return TDS_ERR_ARG;
    if (!aligned(in, 16) || !aligned(out, 16)) return TDS_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || nx % kSZ || ny % kSZ || nz > 65535 || ny > 65535 ||
        (long long)nx * ny * nz > (1ll << 40))
        return TDS_ERR_SHAPE;
    const size_t bytes = (size_t)nx * ny * nz * elem_size(dtype);
    if (overlaps(in, bytes, out, bytes)) return TDS_ERR_ALIAS;
    return launch_reorder(in, out, nx, ny, nz, from, to, elem_size(dtype),
                          static_cast<cudaStream_t>(stream));
}

tds_status tds_reorder_add(const void *in, void *out, int nx, int ny, int nz, tds_layout from,
                           tds_layout to, tds_dtype dtype, int sz, void *stream) {
    if (!in || !out || sz != kSZ || (dtype != TDS_F64 && dtype != TDS_F32) ||
        from < TDS_LAYOUT_CART || from > TDS_LAYOUT_Z || to < TDS_LAYOUT_CART || to > TDS_LAYOUT_Z)
        return TDS_ERR_ARG;
    if (!aligned(in, 16) || !aligned(out, 16)) return TDS_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || nx % kSZ || ny % kSZ || nz > 65535 || ny > 65535 ||
        (long long)nx * ny * nz > (1ll << 40))
        return TDS_ERR_SHAPE;
    const size_t bytes = (size_t)nx * ny * nz * elem_size(dtype);
    if (overlaps(in, bytes, out, bytes)) return TDS_ERR_ALIAS;
    return launch_reorder_add(in, out, nx, ny, nz, from, to, elem_size(dtype),
                              static_cast<cudaStream_t>(stream));
}

tds_status tds_fanout_copy(const void *in, void *const *outs, int count, size_t bytes, void *stream) {
    if (!in || !outs || count < 1 || count > kMaxMulti || bytes % 16 || !aligned(in, 16)) return TDS_ERR_ARG;
    for (int o = 0; o < count; ++o) {
        if (!outs[o] || !aligned(outs[o], 16)) return TDS_ERR_ARG;
        if (overlaps(in, bytes, outs[o], bytes)) return TDS_ERR_ALIAS;
        for (int q = 0; q < o; ++q)
            if (overlaps(outs[q], bytes, outs[o], bytes)) return TDS_ERR_ALIAS;
    }
    if (bytes == 0) return TDS_OK;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return TDS_ERR_CUDA;
    }
    return launch_fanout(in, outs, count, bytes, nsm, static_cast<cudaStream_t>(stream));
}

void tds_plan_destroy(tds_plan *p) {
    if (!p) return;
    tds_plan_destroy(p->sub);
    std::free(p->band);
    for (cudaEvent_t e : p->ev)
        if (e) cudaEventDestroy(e);
    if (p->copy_in) cudaStreamDestroy(p->copy_in);
    if (p->copy_out) cudaStreamDestroy(p->copy_out);
    if (p->dmem) cudaFree(p->dmem);
    if (p->thomas_mem) cudaFree(p->thomas_mem);
    std::free(p->hmem);
    delete p;
}

tds_status tds_device_status(void) { return read_device_status(); }

tds_status tds_selftest_timeout(double seconds, void *stream) {
    return launch_selftest_wait(seconds, static_cast<cudaStream_t>(stream));
}

tds_status tds_plan_reduced_coeffs(const tds_plan *p, double *sub, double *sup) {
    if (!p || !sub || !sup) return TDS_ERR_ARG;
    std::memcpy(sub, p->red_sub_host[0], sizeof(double) * 2 * p->P);
    std::memcpy(sup, p->red_sup_host[0], sizeof(double) * 2 * p->P);
    return TDS_OK;
}

tds_status tds_reduced_solve(const tds_plan *p, const double *rhs, double *x, void *stream) {
    if (!p || !rhs || !x) return TDS_ERR_ARG;
    const size_t rb = sizeof(double) * 2 * p->P * (size_t)p->nlines;
    if (overlaps(rhs, rb, x, rb)) return TDS_ERR_ALIAS;
    return launch_reduced_only(p, rhs, x, static_cast<cudaStream_t>(stream));
}

} // extern "C"
