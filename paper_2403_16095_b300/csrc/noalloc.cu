// gs_bin_tiles_noalloc: tile binning for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) at the point
// where they bin: a real-time tracking thread that must never block on the
// allocator, a host process whose device memory is entirely owned by another
// framework's pool, or a plug-in that may only use memory declared when it was
// loaded. This entry point takes the same inputs and outputs as gs_bin_tiles
// but needs no caller workspace: its scratch is the file-scope device array
// below, which every GPU that loads libgs holds until the process exits.
//
// Set-up: the first call on each device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress and caches it with the
// device's current CUDA context; in host code the array's name is only a
// host-side stand-in, never a device address. Make that first call before any
// stream capture. A call that finds another context current (the old one was
// destroyed, e.g. by cudaDeviceReset, and the module loaded again) looks the
// address up again: it is again a first call. All calls share the array
// and it keeps the last call's contents: the binning writes every scratch word
// it reads later in the same call and clears its counters itself, so nothing
// leaks from one call to the next; calls that overlap on the GPU (different
// streams, or the same device from several threads without ordering) race on
// the array.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "gs_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)12 << 20;  // holds the workspace of GS_NOALLOC_MAX_PAIRS pairs
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bin_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};
void *g_scratch_ctx[kMaxDevices] = {};  // the context the cached address belongs to

// The current CUDA context (cuCtxGetCurrent, resolved through the runtime's
// driver entry points so that libgs links no driver library), or NULL.
void *current_context() {
    using Fn = int (*)(void **);
    static Fn fn = nullptr;
    static bool tried = false;
    if (!tried) {  // under g_mu
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(p);
    }
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

gs_status na_fail(gs_status st, const char *msg) {
    char buf[256];
    snprintf(buf, sizeof(buf), "gs_bin_tiles_noalloc: %s", msg);
    gs::set_error_message(buf);
    return st;
}

// Device address of the scratch array on the current device (set-up on first use).
gs_status scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(GS_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(GS_ERR_UNSUPPORTED, "device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_mu);
    void *ctx = current_context();
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess || !p) return na_fail(GS_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context();  // the lookup may have made the context current
    }
    *out = g_scratch_addr[dev];
    return GS_OK;
}

}  // namespace

extern "C" gs_status gs_bin_tiles_noalloc(const gs_projected *proj, int n_frames, const gs_camera *cams,
                                          const gs_opts *opts, gs_tiles *tiles, int32_t *status, gs_stream stream) {
    if (!proj || !tiles || !opts || !cams || !status) return na_fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (tiles->capacity < 1 || tiles->capacity > GS_NOALLOC_MAX_PAIRS) {
        char buf[160];
        snprintf(buf, sizeof(buf), "capacity %d outside 1..%d pairs (use gs_bin_tiles with a caller workspace)",
                 tiles->capacity, GS_NOALLOC_MAX_PAIRS);
        return na_fail(GS_ERR_INVALID_ARG, buf);
    }
    const long long records = (long long)proj->n_gaussians * (n_frames > 0 ? n_frames : 0);
    if (proj->n_gaussians < 0 || records > INT32_MAX) return na_fail(GS_ERR_INVALID_ARG, "bad record count");
    const size_t need = gs_bin_tiles_workspace_size((int)records, tiles->capacity);
    if (need == 0 || need > kScratchBytes) return na_fail(GS_ERR_INVALID_ARG, "scratch needed exceeds the static array");
    void *ws = nullptr;
    const gs_status st = scratch_address(&ws);
    if (st != GS_OK) return st;
    // the regular entry point validates the rest and launches the same kernels
    return gs_bin_tiles(proj, n_frames, cams, opts, tiles, status, ws, kScratchBytes, stream);
}
