// Photometric loss of Sec. 4 (Eq. energy) on the smoothed render ("Variance
// Reduction": 3x3 Gaussian, sigma 1): blurred = G * image (replicate border),
// loss = sum |blurred - target| reduced in FP64, and its adjoint
// dloss/dimage = G^T * sign(blurred - target) by gather (no atomics).
// Batched over images through blockIdx.y; arguments travel by value.
//
// The loss sum does not depend on how blocks are scheduled: block b of an
// image always sums the same elements (a grid-stride loop over a fixed number
// of blocks per image) in the same order, writes its FP64 partial to its own
// slot, and a finishing kernel adds the partials in block order and stores the
// result.  Repeated calls therefore give bitwise the same loss.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int LOSS_THREADS = 256;

FR_D float gw(int dx, int dy) {
    const float e1 = expf(-0.5f), e2 = expf(-1.0f);
    const float z = 1.0f + 4.0f * e1 + 4.0f * e2;
    const int r2 = dx * dx + dy * dy;
    return (r2 == 0 ? 1.0f : (r2 == 1 ? e1 : e2)) / z;
}

FR_HD int loss_blocks(int px3) {
    const int nb = (px3 + LOSS_THREADS - 1) / LOSS_THREADS;
    return nb < FR_LOSS_PARTS ? (nb > 0 ? nb : 1) : FR_LOSS_PARTS;
}

__global__ void __launch_bounds__(LOSS_THREADS) k_blur_loss(LossTable t) {
    __shared__ double part[LOSS_THREADS / 32];
    const LossItem& L = t.it[blockIdx.y];
    const int H = L.H, W = L.W, n = H * W * 3;
    const int nb = loss_blocks(n);
    if ((int)blockIdx.x >= nb) return;                  // block-uniform
    double l = 0.0;
    for (int i = blockIdx.x * LOSS_THREADS + threadIdx.x; i < n; i += nb * LOSS_THREADS) {
        const int k = i % 3, p = i / 3, x = p % W, y = p / W;
        float acc = 0.0f;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int yy = min(max(y + dy, 0), H - 1), xx = min(max(x + dx, 0), W - 1);
                acc += gw(dx, dy) * L.image[3 * (yy * W + xx) + k];
            }
        const float r = acc - L.target[i];
        l += fabs((double)r);
        L.sign[i] = (float)((r > 0.0f) - (r < 0.0f));
        if (L.blurred) L.blurred[i] = acc;
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < LOSS_THREADS / 32; ++w) s += part[w];
        L.part[blockIdx.x] = s;
    }
}

// loss = sum of the image's block partials in block order (one block per image)
__global__ void __launch_bounds__(LOSS_THREADS) k_loss_finish(LossTable t) {
    __shared__ double part[LOSS_THREADS];
    const LossItem& L = t.it[blockIdx.x];
    const int nb = loss_blocks(L.H * L.W * 3);
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += LOSS_THREADS) s += L.part[b];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = LOSS_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *L.loss = part[0];
}

// adj_q = sum over (p, delta) with clamp(p + delta) == q of w(delta) sgn_p
__global__ void __launch_bounds__(LOSS_THREADS) k_blur_adjoint(LossTable t) {
    const LossItem& L = t.it[blockIdx.y];
    if (!L.adj) return;
    const int H = L.H, W = L.W;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= H * W * 3) return;
    const int k = i % 3, q = i / 3, qx = q % W, qy = q / W;
    float acc = 0.0f;
    for (int py = max(qy - 2, 0); py <= min(qy + 2, H - 1); ++py)
        for (int px = max(qx - 2, 0); px <= min(qx + 2, W - 1); ++px)
            for (int dy = -1; dy <= 1; ++dy) {
                if (min(max(py + dy, 0), H - 1) != qy) continue;
                for (int dx = -1; dx <= 1; ++dx)
                    if (min(max(px + dx, 0), W - 1) == qx) acc += gw(dx, dy) * L.sign[3 * (py * W + px) + k];
            }
    L.adj[i] = acc;
}

}  // namespace

void launch_loss(const LossTable& t, cudaStream_t st) {
    if (t.n <= 0) return;
    k_blur_loss<<<dim3(loss_blocks(t.max_px3), t.n), LOSS_THREADS, 0, st>>>(t);
    k_loss_finish<<<t.n, LOSS_THREADS, 0, st>>>(t);
    k_blur_adjoint<<<dim3((t.max_px3 + LOSS_THREADS - 1) / LOSS_THREADS, t.n), LOSS_THREADS, 0, st>>>(t);
    fr_count_launches(3);
}

void launch_loss(int H, int W, const float* image, const float* target, double* loss, float* sign, double* part,
                 float* blurred, float* adj_image, cudaStream_t st) {
    LossTable t;
    t.n = 1;
    t.max_px3 = H * W * 3;
    t.it[0] = LossItem{H, W, image, target, loss, sign, part, blurred, adj_image};
    launch_loss(t, st);
}
