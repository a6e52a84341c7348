// Linear models y_b = mean + basis * coef_b for the faces of a batch, in FP32
// on the CUDA cores, and their transpose for the adjoint:
//   * the shape morph of Sec. 3.1, v = a_s + Sigma_s alpha + Sigma_e delta
//     (rows = 3N vertex coordinates);
//   * the statistical albedos of Sec. 3.2 in UV texture space,
//     C = a_r + Sigma_r beta and S = a_b + Sigma_b gamma (rows = 3 M^2 texels).
// Both are HBM-bound at any batch size a call holds, so the kernels stream the
// basis with float4 loads, once per group of up to eight faces; the BF16
// tensor-core form of the forward is in morph_tc.cu.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int LIN_THREADS = 256;
constexpr int ADJ_ROWS4 = 1024;          // float4 rows summed by one adjoint block

// Faces per pass over the basis: a launch reads each basis float4 once per
// group of LIN_GROUP faces (blockIdx.y is the group), so a batch streams the
// basis ceil(n / LIN_GROUP) times instead of n times.
constexpr int LIN_GROUP = 8;

// Thread i owns float4 i of the rows: y_b = mean + (sum_k c_bk basis[k]) for
// the G faces b of its group, with their coefficients staged in shared memory.
// The basis terms are summed apart from the mean (they are much smaller), so
// the large mean is rounded into the result once.
template <int G>
__global__ void __launch_bounds__(LIN_THREADS) k_linear(const float* __restrict__ mean,
                                                        const float* __restrict__ basis, int ld, int rows, int K,
                                                        LinearTable t) {
    __shared__ float c[G][FR_MAX_BASIS];
    const int b0 = blockIdx.y * G, nb_ = min(G, t.n - b0);
    for (int q = threadIdx.x; q < G * K; q += blockDim.x) {
        const int b = q / K, k = q % K;
        c[b][k] = b < nb_ ? t.coef[b0 + b][k] : 0.0f;
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * i >= rows) return;
    const int ld4 = ld / 4;
    const float4 m = __ldg(reinterpret_cast<const float4*>(mean) + i);
    float4 acc[G];
#pragma unroll
    for (int b = 0; b < G; ++b) acc[b] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    const float4* bp = reinterpret_cast<const float4*>(basis) + i;
    // unrolled so that several basis rows are in flight per thread (the grid
    // of one face is small: 3N / 4 threads)
#pragma unroll 8
    for (int k = 0; k < K; ++k) {
        const float4 bk = __ldg(bp + (size_t)k * ld4);
#pragma unroll
        for (int b = 0; b < G; ++b) {
            const float ck = c[b][k];
            acc[b].x += ck * bk.x; acc[b].y += ck * bk.y; acc[b].z += ck * bk.z; acc[b].w += ck * bk.w;
        }
    }
#pragma unroll
    for (int b = 0; b < G; ++b) {
        if (b >= nb_) break;
        acc[b] = make_float4(m.x + acc[b].x, m.y + acc[b].y, m.z + acc[b].z, m.w + acc[b].w);
        float* o = t.out[b0 + b] + 4 * (size_t)i;
        if (4 * i + 4 <= rows) {
            *reinterpret_cast<float4*>(o) = acc[b];
        } else {                               // ragged tail: rows not a multiple of 4
            o[0] = acc[b].x;
            if (4 * i + 1 < rows) o[1] = acc[b].y;
            if (4 * i + 2 < rows) o[2] = acc[b].z;
        }
    }
}

// Adjoint, first pass: block (chunk, k-group, face group) sums
// basis[k][i] * g_b[i] over its chunk of rows for KG consecutive k and the G
// faces b of its group into part[b][k][chunk].  A thread sums its few rows of
// the chunk (ADJ_ROWS4 / LIN_THREADS float4 rows, 16 products) and the warp
// its 32 threads in FP32; the block, chunk and batch sums are FP64 (the FP64
// pipe is narrow, so it only sees one value per warp).  Each basis float4 is read once per face
// group and each gradient float4 once per k-group.
template <int G, int KG>
__global__ void __launch_bounds__(LIN_THREADS) k_linear_adj_part(const float* __restrict__ basis, int ld, int rows,
                                                                 int K, LinearAdjTable t, double* part,
                                                                 int n_chunks) {
    __shared__ double w[LIN_THREADS / 32][KG][G];
    const int chunk = blockIdx.x, k0 = blockIdx.y * KG, b0 = blockIdx.z * G;
    const int nb_ = min(G, t.n - b0), nk = min(KG, K - k0);
    float acc[KG][G];
#pragma unroll
    for (int q = 0; q < KG; ++q)
#pragma unroll
        for (int b = 0; b < G; ++b) acc[q][b] = 0.0f;
    const int lo = chunk * ADJ_ROWS4, hi = std::min(lo + ADJ_ROWS4, (rows + 3) / 4);
    for (int i = lo + (int)threadIdx.x; i < hi; i += LIN_THREADS) {
        const int e = 4 * i;
        float4 gg[G];
#pragma unroll
        for (int b = 0; b < G; ++b) {
            gg[b] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (b >= nb_ || !t.g_coef[b0 + b]) continue;
            const float* g = t.g[b0 + b];
            if (e + 4 <= rows) {
                gg[b] = *reinterpret_cast<const float4*>(g + e);
            } else {                                   // ragged tail
                gg[b].x = g[e];
                if (e + 1 < rows) gg[b].y = g[e + 1];
                if (e + 2 < rows) gg[b].z = g[e + 2];
            }
        }
#pragma unroll
        for (int q = 0; q < KG; ++q) {
            if (q >= nk) break;
            const float4 bb = __ldg(reinterpret_cast<const float4*>(basis + (size_t)(k0 + q) * ld) + i);
#pragma unroll
            for (int b = 0; b < G; ++b)
                acc[q][b] += bb.x * gg[b].x + bb.y * gg[b].y + bb.z * gg[b].z + bb.w * gg[b].w;
        }
    }
    // warp sums in FP32 (32 partials of a few products each, in a fixed
    // order); FP64 from the block sum on
#pragma unroll
    for (int q = 0; q < KG; ++q)
#pragma unroll
        for (int b = 0; b < G; ++b) {
            float v = acc[q][b];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5][q][b] = (double)v;
        }
    __syncthreads();
    const int q = threadIdx.x / G, b = threadIdx.x % G;
    if (q < nk && b < nb_) {
        double s = 0.0;
        for (int r = 0; r < LIN_THREADS / 32; ++r) s += w[r][q][b];
        part[((size_t)(b0 + b) * K + k0 + q) * n_chunks + chunk] = s;
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
    const dim3 grid(nb((rows + 3) / 4, LIN_THREADS), nb(t.n, LIN_GROUP));
    if (t.n == 1)      // one face: smaller blocks spread its few rows over more SMs
        k_linear<1><<<nb((rows + 3) / 4, LIN_THREADS / 2), LIN_THREADS / 2, 0, st>>>(mean, basis, ld, rows, K, t);
    else
        k_linear<LIN_GROUP><<<grid, LIN_THREADS, 0, st>>>(mean, basis, ld, rows, K, t);
    fr_count_launches(1);
}

void launch_linear_adjoint(const float* basis, int ld, int rows, int K, const LinearAdjTable& t, double* part,
                           cudaStream_t st) {
    if (t.n <= 0 || K <= 0 || rows <= 0) return;
    const int n_chunks = linear_adj_chunks(rows);
    if (t.n == 1)
        k_linear_adj_part<1, 8><<<dim3(n_chunks, nb(K, 8), 1), LIN_THREADS, 0, st>>>(basis, ld, rows, K, t, part,
                                                                                     n_chunks);
    else
        k_linear_adj_part<LIN_GROUP, 4><<<dim3(n_chunks, nb(K, 4), nb(t.n, LIN_GROUP)), LIN_THREADS, 0, st>>>(
            basis, ld, rows, K, t, part, n_chunks);
    k_linear_adj_finish<<<dim3(nb(K, 128), t.n), 128, 0, st>>>(part, K, n_chunks, t);
    fr_count_launches(2);
}
