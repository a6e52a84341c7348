// fr_loss_noalloc: the photometric loss (blur + L1 + adjoint) for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application may own the whole
// device memory budget through its own pool and forbid libraries from
// allocating behind its back, and a latency-critical loop cannot afford the
// implicit synchronisation an allocation may cause.  Such callers pass their
// own input and output buffers; the one scratch buffer the loss needs (the
// sign of the blurred residual) lives in the file-scope device array below
// instead of in a context.
//
// The array is sized for images of at most FR_LOSS_NOALLOC_MAX_PIXELS pixels
// (512 x 512: 3 MiB).  Every GPU that loads this library holds it until the
// process exits.  All calls share it and it keeps the last call's contents;
// each call overwrites the part it reads before reading it, so nothing needs
// clearing, but two calls whose kernels overlap on the GPU (unordered streams)
// race on it and must be serialised by the caller.
#include <cstdio>
#include <mutex>

#include "../../include/facert.h"
#include "common.cuh"
#include "kernels.h"

#define FR_LOSS_NOALLOC_MAX_PIXELS (512 * 512)
#define FR_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) float g_loss_sign_scratch[FR_LOSS_NOALLOC_MAX_PIXELS * 3];

namespace {

std::mutex g_setup_mutex;
float* g_scratch_ptr[FR_NOALLOC_MAX_DEVICES] = {};
thread_local char g_noalloc_err[256];

fr_status noalloc_fail(fr_status code, const char* msg) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%s", msg);
    return code;
}

// Device address of the scratch array on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device, with that device current, and cached.
fr_status scratch_on_current_device(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(FR_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= FR_NOALLOC_MAX_DEVICES) return noalloc_fail(FR_EINVAL, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        float* p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_loss_sign_scratch);
        if (e != cudaSuccess) return noalloc_fail(FR_ECUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return FR_OK;
}

}  // namespace

extern "C" fr_status fr_loss_noalloc(int32_t height, int32_t width, const float* image, const float* target,
                                     double* loss, float* adj_image, float* blurred, void* stream) {
    if (!image || !target || !loss) return noalloc_fail(FR_EINVAL, "fr_loss_noalloc: null argument");
    if (height < 1 || width < 1 || (long)height * width > FR_LOSS_NOALLOC_MAX_PIXELS)
        return noalloc_fail(FR_EINVAL, "fr_loss_noalloc: image larger than the 512x512-pixel static scratch");
    float* sign = nullptr;
    fr_status s = scratch_on_current_device(&sign);
    if (s != FR_OK) return s;
    launch_loss(height, width, image, target, loss, sign, blurred, adj_image, static_cast<cudaStream_t>(stream));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FR_ECUDA, cudaGetErrorString(e));
    return FR_OK;
}

extern "C" const char* fr_loss_noalloc_error(void) { return g_noalloc_err; }
