// fic_decode_static: decoding that allocates nothing.
//
// Some callers cannot call cudaMalloc: applications that reserve all device memory up front and
// hand libraries only the buffers they need (engines and media frameworks that own the memory
// budget), and latency-critical loops in which an allocation could block on, or synchronise,
// the device. fic_decode needs one image of scratch besides its output (the two planes of 2x2
// averages it iterates on, or with odd strides the second buffer of the Jacobi iteration), which
// those callers cannot provide on demand. This variant keeps that
// scratch in a fixed array in the library's device memory instead: every GPU that loads the
// library holds the array (kStaticDecodeMaxPixels floats, 4 MiB) until the process exits.
//
// The array's device address is looked up (cudaGetSymbolAddress, with the device current) on the
// first call made with a device current, and again after that device's context was re-created;
// host code must not use the array's name directly, which on the host only names a stand-in, not device memory. Every call
// shares the one array and leaves its last contents behind: nothing here reads scratch that the
// same call has not written first, and calls whose GPU work overlaps (other streams, other host
// threads) race on it.
#include <cstdio>
#include <mutex>

#include "fic_internal.cuh"

namespace fic {

constexpr size_t kStaticDecodeMaxPixels = (size_t)FIC_DECODE_STATIC_MAX_PIXELS;

static __device__ __align__(256) float g_decode_scratch[kStaticDecodeMaxPixels];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
struct ScratchEntry {
    void *ctx = nullptr;  // the context (CUcontext) the address belongs to
    float *ptr = nullptr;
};
ScratchEntry g_scratch[kMaxDevices];

// Device address of g_decode_scratch in the current device's current context, looked up once per
// (device, context): the module, and with it the array, is loaded again when a context is
// re-created, so an address cached for an earlier context is not reused.
cudaError_t scratch_for_current_device(float **ptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *ctx = nullptr;
    if (!current_context(&ctx)) return cudaErrorDeviceUninitialized;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    ScratchEntry &ent = g_scratch[dev];
    if (!ctx || !ent.ptr || ent.ctx != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_decode_scratch);  // makes the primary context current if none is
        if (e != cudaSuccess) return e;
        if (!current_context(&ctx) || !ctx) return cudaErrorDeviceUninitialized;
        ent.ptr = static_cast<float *>(p);
        ent.ctx = ctx;
    }
    *ptr = ent.ptr;
    return cudaSuccess;
}
}  // namespace

}  // namespace fic

extern "C" fic_status fic_decode_static(const fic_codes *codes, const fic_geom *gm, const fic_params *p,
                                        int32_t iters, const float *x0, float *out, void *stream) {
    using namespace fic;
    NvtxRange nvtx_range("fic_decode_static");
    // geometry and parameters pass the same checks, and give the same grids, as in fic_decode
    Geo g{};
    const fic_status gs = make_geometry(gm, p, &g);
    if (gs != FIC_OK) return gs;
    if (!codes || !codes->dom || !codes->iso || !codes->s || !codes->o || !out || iters < 0) {
        set_error("fic_decode_static: null code or output pointer, or negative iters");
        return FIC_ERR_INVALID_ARG;
    }
    const size_t img = (size_t)gm->H * gm->W;
    if (img > kStaticDecodeMaxPixels) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "fic_decode_static: %d x %d = %zu pixels exceeds the fixed scratch of %zu pixels; "
                 "use fic_decode with a workspace",
                 gm->H, gm->W, img, kStaticDecodeMaxPixels);
        set_error(msg);
        return FIC_ERR_INVALID_ARG;
    }
    float *tmp = nullptr;
    cudaError_t e = scratch_for_current_device(&tmp);
    if (e != cudaSuccess) {
        set_error(cudaGetErrorString(e));
        return FIC_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (iters == 0) {
        e = x0 ? cudaMemcpyAsync(out, x0, img * sizeof(float), cudaMemcpyDeviceToDevice, st)
               : launch_fill(out, img, 128.f, st);
    } else {
        // the same launches as fic_decode, with the fixed array as its scratch
        e = launch_decode_iterate(*codes, g, iters, x0, out, tmp, st);
    }
    if (e != cudaSuccess) {
        set_error(cudaGetErrorString(e));
        return FIC_ERR_CUDA;
    }
    return FIC_OK;
}
