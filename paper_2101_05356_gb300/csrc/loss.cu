// Photometric loss of Sec. 4 (Eq. energy) on the smoothed render ("Variance
// Reduction": 3x3 Gaussian, sigma 1): blurred = G * image (replicate border),
// loss = sum |blurred - target| reduced in FP64, and its adjoint
// dloss/dimage = G^T * sign(blurred - target) by gather (no atomics).
#include "common.cuh"
#include "kernels.h"

namespace {

FR_D float gw(int dx, int dy) {
    const float e1 = expf(-0.5f), e2 = expf(-1.0f);
    const float z = 1.0f + 4.0f * e1 + 4.0f * e2;
    const int r2 = dx * dx + dy * dy;
    return (r2 == 0 ? 1.0f : (r2 == 1 ? e1 : e2)) / z;
}

__global__ void __launch_bounds__(256) k_blur_loss(int H, int W, const float* __restrict__ img,
                                                   const float* __restrict__ tgt, double* loss,
                                                   float* __restrict__ sgn, float* __restrict__ blurred) {
    __shared__ double part[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;   // over H * W * 3
    double l = 0.0;
    if (i < H * W * 3) {
        const int k = i % 3, p = i / 3, x = p % W, y = p / W;
        float acc = 0.0f;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = min(max(y + dy, 0), H - 1), xx = min(max(x + dx, 0), W - 1);
                acc += gw(dx, dy) * img[3 * (yy * W + xx) + k];
            }
        const float r = acc - tgt[i];
        l = fabs((double)r);
        sgn[i] = (float)((r > 0.0f) - (r < 0.0f));
        if (blurred) blurred[i] = acc;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
        if (s != 0.0) atomicAdd(loss, s);
    }
}

// adj_q = sum over (p, delta) with clamp(p + delta) == q of w(delta) sgn_p
__global__ void __launch_bounds__(256) k_blur_adjoint(int H, int W, const float* __restrict__ sgn,
                                                      float* __restrict__ adj) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * W * 3) return;
    const int k = i % 3, q = i / 3, qx = q % W, qy = q / W;
    float acc = 0.0f;
    for (int py = max(qy - 2, 0); py <= min(qy + 2, H - 1); ++py)
        for (int px = max(qx - 2, 0); px <= min(qx + 2, W - 1); ++px)
            for (int dy = -1; dy <= 1; ++dy) {
                if (min(max(py + dy, 0), H - 1) != qy) continue;
                for (int dx = -1; dx <= 1; ++dx)
                    if (min(max(px + dx, 0), W - 1) == qx) acc += gw(dx, dy) * sgn[3 * (py * W + px) + k];
            }
    adj[i] = acc;
}

}  // namespace

void launch_loss(int H, int W, const float* image, const float* target, double* loss, float* sign,
                 float* blurred, float* adj_image, cudaStream_t st) {
    const int n = H * W * 3;
    cudaMemsetAsync(loss, 0, sizeof(double), st);
    k_blur_loss<<<(n + 255) / 256, 256, 0, st>>>(H, W, image, target, loss, sign, blurred);
    fr_count_launches(1);
    if (adj_image) {
        k_blur_adjoint<<<(n + 255) / 256, 256, 0, st>>>(H, W, sign, adj_image);
        fr_count_launches(1);
    }
}
