// Forward with a fixed, library-owned scratch area instead of the plan's
// workspaces, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc once they are running: a process whose
// device memory is all reserved up front by another framework's caching
// allocator (a fresh cudaMalloc fails or fragments that pool), or a
// latency-bound serving loop that avoids cudaMalloc because it may
// synchronise the whole device.  Such a caller creates its plans at start-up;
// grav_forward_static_scratch then lets it run a forward without the plan's
// own workspaces, e.g. a second forward on the same plan on another stream,
// without asking for more memory.
//
// The scratch is one file-scope __device__ array of GRAV_STATIC_SCRATCH_BYTES
// that every GPU loading the library holds until the process exits.  Host
// code must not pass the array's name to a kernel (on the host it is only a
// stand-in symbol); the device address is looked up with
// cudaGetSymbolAddress, with the device current, on the first call made on
// that device, and again only if the device's CUDA context has changed since
// (after cudaDeviceReset the old address belongs to a context that no longer
// exists).  Every call shares the array: two calls whose work overlaps on
// the GPU race, whatever plans they use.  The forward writes every scratch
// element it later reads, so nothing has to be cleared between calls.
#include <mutex>

#include "grav_internal.h"

namespace grav {

namespace {

constexpr size_t kScratchBytes = (size_t)GRAV_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);

// cuCtxGetCurrent from the driver, looked up once through the runtime.
CtxGetCurrentFn ctx_get_current() {
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return reinterpret_cast<CtxGetCurrentFn>(p);
    }();
    return fn;
}

// Device address of the static scratch on the current device, looked up on
// the first call and again whenever the device's context is a new one.
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("grav_forward_static_scratch: device ordinal %d beyond %d", dev, kMaxDevices);
        return GRAV_EINVAL;
    }
    CtxGetCurrentFn get_ctx = ctx_get_current();
    CUcontext ctx = nullptr;
    if (get_ctx && get_ctx(&ctx) == CUDA_SUCCESS && !ctx) {
        // a host thread that has not used the runtime yet: cudaSetDevice
        // makes the device's primary context current on it
        cudaError_t e = cudaSetDevice(dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
        get_ctx(&ctx);
    }
    if (!get_ctx || !ctx) {
        set_error("grav_forward_static_scratch: no current CUDA context (cuCtxGetCurrent)");
        return GRAV_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev] || g_scratch_ctx[dev] != ctx) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_addr[dev];
    return GRAV_OK;
}

template <typename R>
int forward_static(grav_plan* p, const void* rho, void* out, unsigned char* scratch, size_t x_bytes,
                   cudaStream_t s) {
    void* X = scratch;
    void* Y = scratch + x_bytes;
    cudaError_t e = launch_row_r2c<R>(p->log_px, (const R*)rho, (size_t)p->ny * p->nx, (size_t)p->nx, p->nx, p->ny,
                                      p->nz, X, p->ny_pad, p->tw, p->log_t, s, Batch(), p->err_flag);
    if (e != cudaSuccess) return cuda_fail(e, "static-scratch forward row transform");
    ColumnArgs a{p->ny, p->ny_pad, p->nz, p->ncomp, p->kx_count, p->jp, p->imag_mask, p->oddv_mask,
                 p->log_t - (p->log_py - 1), p->log_t - p->log_py};
    e = launch_forward_columns<R>(p->log_py - 1, a, X, (const R*)p->spec, Y, p->tw, p->err_flag, s, Batch());
    if (e != cudaSuccess) return cuda_fail(e, "static-scratch forward column stage");
    const size_t half = (size_t)p->kx_count * p->ncomp * p->ny_pad * 2 * sizeof(R);
    e = launch_row_c2r<R>(p->log_px, Y, (const unsigned char*)Y + half, p->ny, p->ncomp, p->ny_pad, (R*)out,
                          (size_t)p->nx, p->nx, p->tw, p->log_t, s, Batch());
    if (e != cudaSuccess) return cuda_fail(e, "static-scratch forward inverse row transform");
    return GRAV_OK;
}

}  // namespace

}  // namespace grav

using namespace grav;

extern "C" int grav_forward_static_scratch(grav_plan* plan, const void* rho_dev, void* out_dev, void* stream) {
    if (!plan || !rho_dev || !out_dev) {
        set_error("grav_forward_static_scratch: null plan or buffer");
        return GRAV_EINVAL;
    }
    if (plan->kind != 0) {
        set_error("grav_forward_static_scratch: the plan was made by grav_plan_create3d");
        return GRAV_EINVAL;
    }
    const size_t real = plan->fp64 ? sizeof(double) : sizeof(float);
    size_t x_bytes = (size_t)plan->kx_count * plan->nz * plan->ny_pad * 2 * real;
    x_bytes = (x_bytes + 255) / 256 * 256;
    const size_t y_bytes = (size_t)2 * plan->kx_count * plan->ncomp * plan->ny_pad * 2 * real;
    if (x_bytes + y_bytes > kScratchBytes) {
        set_error("grav_forward_static_scratch: this plan needs %zu bytes of scratch, the static area holds %zu",
                  x_bytes + y_bytes, kScratchBytes);
        return GRAV_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != plan->device) {
        set_error("grav_forward_static_scratch: plan lives on device %d, current device is %d", plan->device, dev);
        return GRAV_EINVAL;
    }
    void* scratch = nullptr;
    int rc = scratch_address(dev, &scratch);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    return plan->fp64 ? forward_static<double>(plan, rho_dev, out_dev, (unsigned char*)scratch, x_bytes, s)
                      : forward_static<float>(plan, rho_dev, out_dev, (unsigned char*)scratch, x_bytes, s);
}
