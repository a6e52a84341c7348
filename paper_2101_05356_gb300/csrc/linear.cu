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
    // One face: U basis rows are loaded before any is summed, so that U loads
    // are in flight per thread (its grid is small, 3N / 4 threads, a few warps
    // per SM, and its time is the K / U dependent round trips to HBM).  A group
    // keeps many warps per SM and unrolls by 8.  The sums run over k in order
    // either way, so a face's result is the same in both.
    if constexpr (G > 1) {
#pragma unroll 8
        for (int k = 0; k < K; ++k) {
            const float4 bk = __ldg(bp + (size_t)k * ld4);
#pragma unroll
            for (int b = 0; b < G; ++b) {
                const float ck = c[b][k];
                acc[b].x += ck * bk.x; acc[b].y += ck * bk.y; acc[b].z += ck * bk.z; acc[b].w += ck * bk.w;
            }
        }
    } else {
        constexpr int U = 36;
        for (int k0 = 0; k0 < K; k0 += U) {
            float4 bk[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (k0 + u < K) bk[u] = __ldg(bp + (size_t)(k0 + u) * ld4);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (k0 + u >= K) break;
#pragma unroll
                for (int b = 0; b < G; ++b) {
                    const float ck = c[b][k0 + u];
                    acc[b].x += ck * bk[u].x; acc[b].y += ck * bk[u].y; acc[b].z += ck * bk[u].z; acc[b].w += ck * bk[u].w;
                }
            }
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

// Adjoint, first pass.  Block (chunk of ADJ_ROWS4 float4 rows, face group of
// G, k-slice z) stages the chunk's gradients g_b of its faces in shared memory
// once; its warp w takes the column groups z * 8 + w, then every 8 * gridDim.z
// after, of KG consecutive k, and sums basis[k][i] * g_b[i] over the chunk (a
// lane its ADJ_ROWS4 / 32 rows in order, the warp its lanes by a butterfly, all
// FP32) into part[chunk][b][k] (FP64; chunk-major, so that the second pass
// reads it coalesced).  Each basis float4 is read once per face group and each
// gradient float4 once per k-slice.  The order of every (face, k) sum depends
// only on the chunking, not on G, KG or the k-split, so the one-face kernel
// below, which keeps that order, gives a face's gradient bitwise the same
// alone and in a batch.
constexpr int ADJ_ROWS4 = 256;

// The models of one transpose launch (up to two: the two statistical albedos
// share one).  start[m] is model m's first block (first pass of a batch) or
// first warp item (one face); the kernels read the table in place.
struct AdjLaunch {
    int n_models;
    int start[3];
    const float* basis[2];
    int ld[2], rows[2], K[2], chunks[2];
    double* part[2];
    LinearAdjTable t[2];
};

template <int NM>
__device__ __forceinline__ int adj_model(const AdjLaunch& L, long x) {
    return (NM > 1 && x >= L.start[1]) ? 1 : 0;
}
template <int G, int KG, int MIN_BLOCKS>
__global__ void __launch_bounds__(LIN_THREADS, MIN_BLOCKS) k_linear_adj_part(const __grid_constant__ AdjLaunch L) {
    __shared__ float4 gs[G][ADJ_ROWS4];
    const int m = adj_model<2>(L, blockIdx.x);
    const float* __restrict__ basis = L.basis[m];
    const int ld = L.ld[m], rows = L.rows[m], K = L.K[m];
    const LinearAdjTable& t = L.t[m];
    double* part = L.part[m];
    const int chunk = blockIdx.x - L.start[m], b0 = blockIdx.y * G;
    const int nb_ = min(G, t.n - b0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int rows4 = (rows + 3) / 4, lo = chunk * ADJ_ROWS4;
    for (int q = threadIdx.x; q < G * ADJ_ROWS4; q += LIN_THREADS) {
        const int b = q / ADJ_ROWS4, r = q % ADJ_ROWS4, i = lo + r, e = 4 * i;
        float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (b < nb_ && t.g_coef[b0 + b] && i < rows4) {
            const float* g = t.g[b0 + b];
            if (e + 4 <= rows) {
                v = *reinterpret_cast<const float4*>(g + e);
            } else {                                   // ragged tail
                v.x = g[e];
                if (e + 1 < rows) v.y = g[e + 1];
                if (e + 2 < rows) v.z = g[e + 2];
            }
        }
        gs[b][r] = v;
    }
    __syncthreads();
    const int n_kg = (K + KG - 1) / KG, warps = LIN_THREADS / 32;
    for (int kg = blockIdx.z * warps + warp; kg < n_kg; kg += warps * gridDim.z) {
        const int k0 = kg * KG, nk = min(KG, K - k0);
        float acc[KG][G];
#pragma unroll
        for (int q = 0; q < KG; ++q)
#pragma unroll
            for (int b = 0; b < G; ++b) acc[q][b] = 0.0f;
#pragma unroll 1
        for (int r = lane; r < ADJ_ROWS4; r += 32) {
            const int i = lo + r;
            if (i >= rows4) break;
            float4 bb[KG];
#pragma unroll
            for (int q = 0; q < KG; ++q)
                bb[q] = q < nk ? __ldg(reinterpret_cast<const float4*>(basis + (size_t)(k0 + q) * ld) + i)
                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int b = 0; b < G; ++b) {
                const float4 gg = gs[b][r];
#pragma unroll
                for (int q = 0; q < KG; ++q)
                    acc[q][b] += bb[q].x * gg.x + bb[q].y * gg.y + bb[q].z * gg.z + bb[q].w * gg.w;
            }
        }
        // the butterfly leaves the same sum, bitwise, on every lane
#pragma unroll
        for (int q = 0; q < KG; ++q)
#pragma unroll
            for (int b = 0; b < G; ++b) {
                float v = acc[q][b];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == ((q * G + b) & 31) && q < nk && b < nb_)
                    part[((size_t)chunk * t.n + b0 + b) * K + k0 + q] = (double)v;
            }
    }
}

// Adjoint of one face, first pass: warp (chunk, column group of KG) sums
// basis[k][i] * g[i] over the chunk exactly as the batched kernel above does
// for each of its faces (the same rows per lane, the same expressions, the
// same butterfly), so the partials are bitwise those of the face in a batch.
// The gradient is read from global memory (consecutive warps share a chunk, so
// it is an L1 hit after the first), which leaves no shared staging to balance
// over the block's warps.
template <int KG>
__global__ void __launch_bounds__(LIN_THREADS) k_linear_adj_one(const __grid_constant__ AdjLaunch L) {
    const int lane = threadIdx.x & 31;
    const long gitem = (long)blockIdx.x * (LIN_THREADS / 32) + (threadIdx.x >> 5);
    const int m = adj_model<1>(L, gitem);       // one model per launch (see the launcher)
    const float* __restrict__ basis = L.basis[m];
    const int ld = L.ld[m], rows = L.rows[m], K = L.K[m], n_chunks = L.chunks[m];
    const LinearAdjTable& t = L.t[m];
    double* part = L.part[m];
    const int n_kg = (K + KG - 1) / KG;
    const long item = gitem - L.start[m];
    if (item >= (long)n_chunks * n_kg || !t.g_coef[0]) return;      // warp-uniform
    const int chunk = (int)(item / n_kg), k0 = (int)(item % n_kg) * KG, nk = min(KG, K - k0);
    const int rows4 = (rows + 3) / 4, lo = chunk * ADJ_ROWS4;
    const float* g = t.g[0];
    float acc[KG];
#pragma unroll
    for (int q = 0; q < KG; ++q) acc[q] = 0.0f;
#pragma unroll 1
    for (int r = lane; r < ADJ_ROWS4; r += 32) {
        const int i = lo + r, e = 4 * i;
        if (i >= rows4) break;
        float4 gg = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (e + 4 <= rows) {
            gg = *reinterpret_cast<const float4*>(g + e);
        } else {                                       // ragged tail
            gg.x = g[e];
            if (e + 1 < rows) gg.y = g[e + 1];
            if (e + 2 < rows) gg.z = g[e + 2];
        }
        float4 bb[KG];
#pragma unroll
        for (int q = 0; q < KG; ++q)
            bb[q] = q < nk ? __ldg(reinterpret_cast<const float4*>(basis + (size_t)(k0 + q) * ld) + i)
                           : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < KG; ++q) acc[q] += bb[q].x * gg.x + bb[q].y * gg.y + bb[q].z * gg.z + bb[q].w * gg.w;
    }
#pragma unroll
    for (int q = 0; q < KG; ++q) {
        float v = acc[q];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == (q & 31) && q < nk) part[((size_t)chunk * t.n) * K + k0 + q] = (double)v;
    }
}

// Adjoint, second pass: g_coef_b[k] += the sum of the chunk partials.  Block
// (FIN_K consecutive k, face b): FIN_STREAMS streams per k each sum the chunks
// stream + FIN_STREAMS * m in order (FP64; a warp reads four chunks' rows of
// FIN_K partials), then a fixed tree over the streams: a fixed order, so the
// result does not depend on scheduling.
constexpr int FIN_THREADS = 1024, FIN_K = 8, FIN_STREAMS = FIN_THREADS / FIN_K;
__global__ void __launch_bounds__(FIN_THREADS) k_linear_adj_finish(const __grid_constant__ AdjLaunch L) {
    __shared__ double ws[FIN_STREAMS][FIN_K];
    const int m = blockIdx.z;
    const double* __restrict__ part = L.part[m];
    const int K = L.K[m], n_chunks = L.chunks[m];
    const LinearAdjTable& t = L.t[m];
    const int kk = threadIdx.x % FIN_K, stream = threadIdx.x / FIN_K;
    const int k = blockIdx.x * FIN_K + kk, b = blockIdx.y;
    double s = 0.0;
    if (k < K) {
#pragma unroll 4
        for (int c = stream; c < n_chunks; c += FIN_STREAMS) s += part[((size_t)c * t.n + b) * K + k];
    }
    ws[stream][kk] = s;
    __syncthreads();
    for (int h = FIN_STREAMS / 2; h > 0; h >>= 1) {
        if (stream < h) ws[stream][kk] += ws[stream + h][kk];
        __syncthreads();
    }
    if (stream == 0 && k < K && t.g_coef[b]) t.g_coef[b][k] += (float)ws[0][kk];
}

int nb(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

int linear_adj_chunks(int rows) { return std::max(1, nb((rows + 3) / 4, ADJ_ROWS4)); }

void launch_linear(const float* mean, const float* basis, int ld, int rows, int K, const LinearTable& t,
                   cudaStream_t st) {
    if (t.n <= 0 || rows <= 0) return;
    const dim3 grid(nb((rows + 3) / 4, LIN_THREADS), nb(t.n, LIN_GROUP));
    // one face: small blocks spread its few rows evenly over the SMs.  (Splitting
    // the columns over several threads per row would keep more loads in flight,
    // but its sums would differ from the batched kernel's in the last bits, and
    // a face must render bitwise the same alone and in a batch.)
    if (t.n == 1)
        k_linear<1><<<nb((rows + 3) / 4, LIN_THREADS / 4), LIN_THREADS / 4, 0, st>>>(mean, basis, ld, rows, K, t);
    else
        k_linear<LIN_GROUP><<<grid, LIN_THREADS, 0, st>>>(mean, basis, ld, rows, K, t);
    fr_count_launches(1);
}

void launch_linear_adjoint(const LinearAdjModel* models, int n_models, cudaStream_t st) {
    AdjLaunch L;
    L.n_models = 0;
    int n = 0, kmax = 0;
    for (int q = 0; q < n_models && L.n_models < 2; ++q) {
        const LinearAdjModel& md = models[q];
        if (md.t.n <= 0 || md.K <= 0 || md.rows <= 0) continue;
        const int m = L.n_models++;
        L.basis[m] = md.basis;
        L.ld[m] = md.ld;
        L.rows[m] = md.rows;
        L.K[m] = md.K;
        L.chunks[m] = linear_adj_chunks(md.rows);
        L.part[m] = md.part;
        L.t[m] = md.t;
        n = md.t.n;                                   // the same faces for every model of a launch
        kmax = std::max(kmax, md.K);
    }
    if (L.n_models == 0) return;
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    const int n_groups = nb(n, LIN_GROUP);
    L.start[0] = 0;
    if (n == 1) {
        // one launch per model: the model's table is then constant in the kernel
        // (48 registers; selecting the model per warp took 57 and measured slower)
        for (int m = 0; m < L.n_models; ++m) {
            AdjLaunch L1 = L;
            L1.n_models = 1;
            L1.basis[0] = L.basis[m]; L1.ld[0] = L.ld[m]; L1.rows[0] = L.rows[m]; L1.K[0] = L.K[m];
            L1.chunks[0] = L.chunks[m]; L1.part[0] = L.part[m]; L1.t[0] = L.t[m];
            L1.start[0] = 0;
            L1.start[1] = L.chunks[m] * nb(L.K[m], 8);
            k_linear_adj_one<8><<<nb(L1.start[1], LIN_THREADS / 32), LIN_THREADS, 0, st>>>(L1);
        }
        fr_count_launches(L.n_models - 1);
    } else {
        for (int m = 0; m < L.n_models; ++m) L.start[m + 1] = L.start[m] + L.chunks[m];
        // split the columns over grid.z until about eight blocks per SM are in flight
        // (measured on GB300, albedo batch 8, both models: two columns per warp at six
        // blocks per SM (40 registers) 0.163 ms; at five 0.183-0.189 ms, at seven or
        // eight (spilling) 0.228 ms, four columns at four 0.185 ms)
        const int most = nb(nb(kmax, 2), LIN_THREADS / 32);
        const int z = std::max(1, std::min(most, nb(8L * sms, (long)L.start[L.n_models] * n_groups)));
        k_linear_adj_part<LIN_GROUP, 2, 6><<<dim3(L.start[L.n_models], n_groups, z), LIN_THREADS, 0, st>>>(L);
    }
    k_linear_adj_finish<<<dim3(nb(kmax, FIN_K), n, L.n_models), FIN_THREADS, 0, st>>>(L);
    fr_count_launches(2);
}
