// tds_noalloc.cu -- tds_deriv_noalloc: the derivative for callers that cannot allocate device
// memory, for example code running where cudaMalloc is not available or not allowed (a host
// that hands out only pre-registered buffers, a real-time loop that must never allocate, a
// plugin whose host application owns all device memory).  Such callers cannot provide the
// workspace that tds_deriv's streaming pipeline needs for the chunk ends, so this entry point
// takes that scratch from a fixed array compiled into the library instead.
#include <mutex>

#include <cudaTypedefs.h>

#include "tds_internal.h"

namespace {

// Scratch for the chunk ends (FP64, 16 bytes per line and chunk) of the streaming pipeline.
// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TDS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 256;
struct ScratchAddr {
    unsigned long long ctx_id;   // the context the address belongs to (0: none looked up yet)
    void *addr;
};
ScratchAddr g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mutex;

// The driver's identity of the current context, unique for the life of the process (a context
// that a device reset destroys and the runtime re-creates gets a new one); 0 if unavailable.
unsigned long long current_context_id() {
    using GetCurrentFn = PFN_cuCtxGetCurrent_v4000;
    using GetIdFn = PFN_cuCtxGetId_v12000;
    static const GetCurrentFn get_current = []() -> GetCurrentFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<GetCurrentFn>(f);
    }();
    static const GetIdFn get_id = []() -> GetIdFn {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<GetIdFn>(f);
    }();
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

// Address of the scratch array on the current device.  In host code the array's name is only
// a host-side stand-in, so the device address is looked up with the device current, once per
// device and context, and cached; a new context on the device (after cudaDeviceReset, say)
// gets a fresh lookup.  With no context current yet on this thread (or without the driver's
// context identity) the lookup, which makes the device's primary context current, runs again.
tds_status scratch_on_current_device(void **addr) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return TDS_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return TDS_ERR_ARG;
    const unsigned long long id = current_context_id();
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchAddr &c = g_scratch_addr[dev];
    if (id == 0 || c.ctx_id != id || !c.addr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TDS_ERR_CUDA;
        }
        c.addr = p;
        c.ctx_id = id;
    }
    *addr = c.addr;
    return TDS_OK;
}

bool overlap(const void *a, const void *b, size_t bytes) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bytes && y < x + bytes;
}

} // namespace

extern "C" TDS_API tds_status tds_deriv_noalloc(const tds_plan *plan, const void *in, void *out,
                                                void *stream) {
    if (!plan || !in || !out || plan->band) return TDS_ERR_ARG;   // a band plan has no stencil
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return TDS_ERR_ARG;
    const size_t bytes = (size_t)plan->n * plan->nlines * (plan->dtype == TDS_F64 ? 8 : 4);
    if (overlap(in, out, bytes)) return TDS_ERR_ALIAS;
    // chunk ends of the forward streaming pipeline: 2 FP64 values per line and chunk
    const size_t need = (size_t)plan->nlines * plan->P * 2 * sizeof(double);
    if (need > (size_t)TDS_NOALLOC_SCRATCH_BYTES) return TDS_ERR_WORKSPACE;
    void *scratch = nullptr;
    const tds_status s = scratch_on_current_device(&scratch);
    if (s != TDS_OK) return s;
    // every scratch entry the pipeline reads is written earlier in the same call: nothing needs
    // to start at zero.  The plan's own chunks run (not the finer-chunk copy an AUTO FP32 plan may
    // carry for tds_deriv): the scratch need stays 16 N P bytes.
    return tds::launch_streaming(plan, 0, in, out, scratch, static_cast<cudaStream_t>(stream));
}
