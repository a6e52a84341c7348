// fr_loss_noalloc: the photometric loss (blur + L1 + adjoint) for callers that
// must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application may own the whole
// device memory budget through its own pool and forbid libraries from
// allocating behind its back, and a latency-critical loop cannot afford the
// implicit synchronisation an allocation may cause.  Such callers pass their
// own input and output buffers; the scratch the loss needs (the sign of the
// blurred residual and the per-block partial sums of the loss) lives in the
// file-scope device arrays below instead of in a context.
//
// The arrays are sized for images of at most FR_LOSS_NOALLOC_MAX_PIXELS pixels
// (512 x 512: 3 MiB of signs, 8 KiB of partials).  Every GPU that loads this
// library holds them until the process exits.  All calls share them and they
// keep the last call's contents; each call overwrites the part it reads before
// reading it, so nothing needs clearing, but two calls whose kernels overlap
// on the GPU (unordered streams) race on them and must be serialised by the
// caller.
#include <cstdio>

#include "../../include/facert.h"
#include "common.cuh"
#include "kernels.h"

#define FR_LOSS_NOALLOC_MAX_PIXELS (512 * 512)

static __device__ __align__(256) float g_loss_sign_scratch[FR_LOSS_NOALLOC_MAX_PIXELS * 3];
static __device__ __align__(256) double g_loss_part_scratch[FR_LOSS_PARTS];

namespace {

thread_local char g_noalloc_err[256];

fr_status noalloc_fail(fr_status code, const char* msg) {
    snprintf(g_noalloc_err, sizeof(g_noalloc_err), "%s", msg);
    return code;
}

// Device addresses of the scratch arrays on the current device.  In host code
// an array's name is only a host-side stand-in, so the addresses are looked up
// with the device current.  They are looked up on every call rather than
// cached: a cached address would go stale if the caller reset the device
// (cudaDeviceReset) and the library's module were loaded again.  The first
// call on a device may load the library's module there, so it should come
// before any stream capture.
fr_status scratch_on_current_device(float** sign, double** part) {
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(sign), g_loss_sign_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(part), g_loss_part_scratch);
    if (e != cudaSuccess) return noalloc_fail(FR_ECUDA, cudaGetErrorString(e));
    return FR_OK;
}

}  // namespace

extern "C" fr_status fr_loss_noalloc(int32_t height, int32_t width, const float* image, const float* target,
                                     double* loss, float* adj_image, float* blurred, void* stream) {
    if (!image || !target || !loss) return noalloc_fail(FR_EINVAL, "fr_loss_noalloc: null argument");
    if (height < 1 || width < 1 || (long)height * width > FR_LOSS_NOALLOC_MAX_PIXELS)
        return noalloc_fail(FR_EINVAL, "fr_loss_noalloc: image larger than the 512x512-pixel static scratch");
    // an error left pending by an earlier, unrelated call is reported as such
    // and left in place for its owner, so that the error read after the
    // launches below belongs to them
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        snprintf(g_noalloc_err, sizeof(g_noalloc_err), "fr_loss_noalloc: an earlier CUDA error is pending: %s",
                 cudaGetErrorString(e));
        return FR_ECUDA;
    }
    float* sign = nullptr;
    double* part = nullptr;
    fr_status s = scratch_on_current_device(&sign, &part);
    if (s != FR_OK) return s;
    launch_loss(height, width, image, target, loss, sign, part, blurred, adj_image, static_cast<cudaStream_t>(stream));
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(FR_ECUDA, cudaGetErrorString(e));
    return FR_OK;
}

extern "C" const char* fr_loss_noalloc_error(void) { return g_noalloc_err; }
