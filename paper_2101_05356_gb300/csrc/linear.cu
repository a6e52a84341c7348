// Linear models y_b = mean + basis * coef_b for the faces of a batch, in FP32
// on the CUDA cores, and their transpose for the adjoint:
//   * the shape morph of Sec. 3.1, v = a_s + Sigma_s alpha + Sigma_e delta
//     (rows = 3N vertex coordinates);
//   * the statistical albedos of Sec. 3.2 in UV texture space,
//     C = a_r + Sigma_r beta and S = a_b + Sigma_b gamma (rows = 3 M^2 texels).
// Both are HBM-bound at any batch size a call holds (one pass over the basis
// per launch), so the kernels stream the basis once with float4 loads; the
// BF16 tensor-core form of the forward is in morph_tc.cu.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int LIN_THREADS = 256;
constexpr int ADJ_ROWS4 = 8192;          // float4 rows summed by one adjoint block

// Thread i owns float4 i of the rows: acc = mean + sum_k c_k basis[k], with
// the face's coefficients staged in shared memory.
__global__ void __launch_bounds__(LIN_THREADS) k_linear(const float* __restrict__ mean,
                                                        const float* __restrict__ basis, int ld, int rows, int K,
                                                        LinearTable t) {
    __shared__ float c[FR_MAX_BASIS];
    const int b = blockIdx.y;
    for (int k = threadIdx.x; k < K; k += blockDim.x) c[k] = t.coef[b][k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * i >= rows) return;
    const int ld4 = ld / 4;
    float4 acc = __ldg(reinterpret_cast<const float4*>(mean) + i);
    const float4* bp = reinterpret_cast<const float4*>(basis) + i;
    int k = 0;
    for (; k + 4 <= K; k += 4) {
        const float4 b0 = __ldg(bp + (size_t)(k + 0) * ld4), b1 = __ldg(bp + (size_t)(k + 1) * ld4);
        const float4 b2 = __ldg(bp + (size_t)(k + 2) * ld4), b3 = __ldg(bp + (size_t)(k + 3) * ld4);
        acc.x += c[k] * b0.x + c[k + 1] * b1.x + c[k + 2] * b2.x + c[k + 3] * b3.x;
        acc.y += c[k] * b0.y + c[k + 1] * b1.y + c[k + 2] * b2.y + c[k + 3] * b3.y;
        acc.z += c[k] * b0.z + c[k + 1] * b1.z + c[k + 2] * b2.z + c[k + 3] * b3.z;
        acc.w += c[k] * b0.w + c[k + 1] * b1.w + c[k + 2] * b2.w + c[k + 3] * b3.w;
    }
    for (; k < K; ++k) {
        const float4 bk = __ldg(bp + (size_t)k * ld4);
        acc.x += c[k] * bk.x; acc.y += c[k] * bk.y; acc.z += c[k] * bk.z; acc.w += c[k] * bk.w;
    }
    float* o = t.out[b] + 4 * (size_t)i;
    if (4 * i + 4 <= rows) {
        *reinterpret_cast<float4*>(o) = acc;
    } else {                                   // ragged tail: rows not a multiple of 4
        o[0] = acc.x;
        if (4 * i + 1 < rows) o[1] = acc.y;
        if (4 * i + 2 < rows) o[2] = acc.z;
    }
}

// Adjoint, first pass: block (chunk, k, b) sums basis[k][i] * g_b[i] over its
// chunk of rows (FP32 products, FP64 sum) into part[b][k][chunk].
__global__ void __launch_bounds__(LIN_THREADS) k_linear_adj_part(const float* __restrict__ basis, int ld, int rows,
                                                                 int K, LinearAdjTable t, double* part,
                                                                 int n_chunks) {
    __shared__ double w[LIN_THREADS / 32];
    const int chunk = blockIdx.x, k = blockIdx.y, b = blockIdx.z;
    double acc = 0.0;
    if (t.g_coef[b]) {
        const float* g = t.g[b];
        const float4* bp = reinterpret_cast<const float4*>(basis + (size_t)k * ld);
        const int lo = chunk * ADJ_ROWS4, hi = std::min(lo + ADJ_ROWS4, (rows + 3) / 4);
        for (int i = lo + (int)threadIdx.x; i < hi; i += LIN_THREADS) {
            const float4 bb = __ldg(bp + i);
            const int e = 4 * i;
            float s;
            if (e + 4 <= rows) {
                const float4 gg = *reinterpret_cast<const float4*>(g + e);
                s = bb.x * gg.x + bb.y * gg.y + bb.z * gg.z + bb.w * gg.w;
            } else {
                s = bb.x * g[e];
                if (e + 1 < rows) s += bb.y * g[e + 1];
                if (e + 2 < rows) s += bb.z * g[e + 2];
            }
            acc += (double)s;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int q = 0; q < LIN_THREADS / 32; ++q) s += w[q];
        part[((size_t)b * K + k) * n_chunks + chunk] = s;
    }
}

// Adjoint, second pass: g_coef_b[k] += sum of the chunk partials in chunk
// order (a fixed order, so the result does not depend on scheduling).
__global__ void k_linear_adj_finish(const double* __restrict__ part, int K, int n_chunks, LinearAdjTable t) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (k >= K || !t.g_coef[b]) return;
    const double* p = part + ((size_t)b * K + k) * n_chunks;
    double s = 0.0;
    for (int c = 0; c < n_chunks; ++c) s += p[c];
    t.g_coef[b][k] += (float)s;
}

int nb(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int linear_adj_chunks(int rows) { return std::max(1, nb((rows + 3) / 4, ADJ_ROWS4)); }

void launch_linear(const float* mean, const float* basis, int ld, int rows, int K, const LinearTable& t,
                   cudaStream_t st) {
    if (t.n <= 0 || rows <= 0) return;
    k_linear<<<dim3(nb((rows + 3) / 4, LIN_THREADS), t.n), LIN_THREADS, 0, st>>>(mean, basis, ld, rows, K, t);
    fr_count_launches(1);
}

void launch_linear_adjoint(const float* basis, int ld, int rows, int K, const LinearAdjTable& t, double* part,
                           cudaStream_t st) {
    if (t.n <= 0 || K <= 0 || rows <= 0) return;
    const int n_chunks = linear_adj_chunks(rows);
    k_linear_adj_part<<<dim3(n_chunks, K, t.n), LIN_THREADS, 0, st>>>(basis, ld, rows, K, t, part, n_chunks);
    k_linear_adj_finish<<<dim3(nb(K, 128), t.n), 128, 0, st>>>(part, K, n_chunks, t);
    fr_count_launches(2);
}
