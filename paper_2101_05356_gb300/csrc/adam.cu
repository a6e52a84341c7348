// Fused multi-tensor Adam with the regularisers of the two-stage optimisation
// (Sec. 4, Eq. loss1 and loss3): shape prior, light prior, soft box
// constraints (expression, intensities, light-stage geometry, textures),
// texture symmetry, chromaticity consistency and smoothness.  One
// launch updates every parameter group of a stage; each thread owns one
// element, adds the regulariser gradient (texture stencils read neighbours) to
// the render gradient, and applies the Adam step with per-group learning rate.
#include "../../include/facert.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int ADAM_THREADS = 256;

struct GroupTable {
    fr_opt_group g[FR_MAX_OPT_GROUPS];
    int block_start[FR_MAX_OPT_GROUPS + 1];
    int n_groups;
    float beta1, beta2, eps;
    float bc1[FR_MAX_OPT_GROUPS], bc2[FR_MAX_OPT_GROUPS];   // bias corrections 1 - beta^t per group
};

FR_D float sgnf(float x) { return (float)((x > 0.0f) - (x < 0.0f)); }

// Regulariser gradient and energy contribution of element i of group G.
FR_D float reg_grad(const fr_opt_group& G, int i, float x, double* energy) {
    float g = 0.0f;
    double e = 0.0;
    switch (G.kind) {
    case FR_GROUP_COEF: {
        if (i < G.n_prior) {                       // w_i sum (alpha_k / sigma_k)^2, sigma_k = 1
            g += 2.0f * G.w_prior * x;
            e += (double)G.w_prior * x * x;
        } else {                                   // soft box delta in [0, 1]
            const float lo = fminf(x, 0.0f), hi = fmaxf(x - 1.0f, 0.0f);
            g += 2.0f * G.w_box * (lo + hi);
            e += (double)G.w_box * (lo * lo + hi * hi);
        }
        break;
    }
    case FR_GROUP_LIGHT: {                         // w1 sum_j |I_j - m_j|^2, I = scale * i, m = mean(I) fixed
        const int j = i / 3;
        float sc;
        if (G.aux) {
            sc = G.aux[j];
        } else {                                   // scale d^2 / a from the stage geometry [d | a | p]
            const float d = G.aux2[j], a = G.aux2[G.n / 3 + j];
            sc = a > 0.0f ? d * d / a : 0.0f;
        }
        const float* base = G.x + 3 * j;
        const float m = sc * (base[0] + base[1] + base[2]) * (1.0f / 3.0f);
        const float d = sc * x - m;
        g += 2.0f * G.w_prior * d * sc;
        e += (double)G.w_prior * d * d;
        const float lo = fminf(x, 0.0f);          // soft box i > 0
        g += 2.0f * G.w_box * lo;
        e += (double)G.w_box * lo * lo;
        break;
    }
    case FR_GROUP_STAGE: {                         // light geometry [d | a | p0 p1] of N_L lights
        const int NL = G.n / 4;
        const float* X = G.x;
        if (i < 2 * NL) {
            const int j = i < NL ? i : i - NL;
            const float d = X[j], a = X[NL + j];
            float dE_ds = 0.0f;                    // light prior through s = d^2 / a
            if (a > 0.0f) {
                const float s = d * d / a;
                const float* ij = G.aux + 3 * j;
                const float m = s * (ij[0] + ij[1] + ij[2]) * (1.0f / 3.0f);
                for (int c = 0; c < 3; ++c) dE_ds += (s * ij[c] - m) * ij[c];
                dE_ds *= 2.0f * G.w_prior;
            }
            if (i < NL) {                          // d: prior, soft box d >= 0
                if (a > 0.0f) g += dE_ds * 2.0f * d / a;
                const float lo = fminf(d, 0.0f);
                g += 2.0f * G.w_box * lo;
                e += (double)G.w_box * lo * lo;
            } else {                               // a: prior, soft box [0, 1], inside-face term through sqrt(a)
                if (a > 0.0f) g += dE_ds * (-(d * d / a) / a);
                const float lo = fminf(a, 0.0f), hi = fmaxf(a - 1.0f, 0.0f);
                g += 2.0f * G.w_box * (lo + hi);
                e += (double)G.w_box * (lo * lo + hi * hi);
                if (a > 0.0f) {
                    const float ra = sqrtf(a), r = ra * (1.0f / 3.0f);
                    const float p0 = X[2 * NL + 2 * j], p1 = X[2 * NL + 2 * j + 1];
                    const float in = fminf(p0 - r, 0.0f) + fminf(p1 - r, 0.0f) + fminf(1.0f - p0 - p1 - r, 0.0f);
                    g += 2.0f * G.w_box * in * (-1.0f / (6.0f * ra));
                }
            }
        } else {                                   // p_jm: corners inside the homothetic face
            const int q = i - 2 * NL, j = q >> 1, mm = q & 1;
            const float a = X[NL + j];
            const float r = sqrtf(fmaxf(a, 0.0f)) * (1.0f / 3.0f);
            const float p0 = X[2 * NL + 2 * j], p1 = X[2 * NL + 2 * j + 1];
            const float in0 = fminf(p0 - r, 0.0f), in1 = fminf(p1 - r, 0.0f), in2 = fminf(1.0f - p0 - p1 - r, 0.0f);
            g += 2.0f * G.w_box * ((mm == 0 ? in0 : in1) - in2);
            if (mm == 0) e += (double)G.w_box * ((double)in0 * in0 + (double)in1 * in1 + (double)in2 * in2);
        }
        break;
    }
    case FR_GROUP_TEX_RGB:
    case FR_GROUP_TEX_MONO: {
        const int C = G.kind == FR_GROUP_TEX_RGB ? 3 : 1;
        const int M = G.width;
        const int ch = i % C, t = i / C, col = t % M, row = t / M;
        const float* X = G.x;
        if (G.w_smooth != 0.0f) {                  // sum_i sum_{j in N4(i)} |X_j - X_i|^2
            float s = 0.0f;
            double es = 0.0;
            const int nb[4][2] = {{row, col - 1}, {row, col + 1}, {row - 1, col}, {row + 1, col}};
            for (int k = 0; k < 4; ++k) {
                const int rr = nb[k][0], cc = nb[k][1];
                if (rr < 0 || rr >= M || cc < 0 || cc >= M) continue;
                const float d = x - X[(rr * M + cc) * C + ch];
                s += d;
                es += (double)d * d;
            }
            g += 4.0f * G.w_smooth * s;
            e += (double)G.w_smooth * es;              // each ordered pair once here; summed over i
        }
        if (G.w_sym != 0.0f) {                     // sum |X(x) - X(flip x)|, flip: column -> M - 1 - column
            const int fc = M - 1 - col;
            if (fc != col) {
                const float d = x - X[(row * M + fc) * C + ch];
                g += 2.0f * G.w_sym * sgnf(d);
                e += (double)G.w_sym * fabsf(d);
            }
        }
        if (G.w_chroma != 0.0f && C == 3 && G.aux) {   // sum |kappa(X) - kappa(X0)|, kappa(c) = c / (sum c + 1e-6)
            const float* p = X + t * 3;
            const float* q = G.aux + t * 3;
            const float S = p[0] + p[1] + p[2] + 1e-6f, S0 = q[0] + q[1] + q[2] + 1e-6f;
            float gc = 0.0f;
            for (int k = 0; k < 3; ++k) {
                const float kk = p[k] / S;
                const float sg = sgnf(kk - q[k] / S0);
                gc += sg * (((k == ch) ? 1.0f : 0.0f) - kk) / S;
                if (k == ch) e += (double)G.w_chroma * fabsf(kk - q[k] / S0);
            }
            g += G.w_chroma * gc;
        }
        if (G.w_box != 0.0f) {                     // soft box [0, 1]
            const float lo = fminf(x, 0.0f), hi = fmaxf(x - 1.0f, 0.0f);
            g += 2.0f * G.w_box * (lo + hi);
            e += (double)G.w_box * (lo * lo + hi * hi);
        }
        break;
    }
    default:
        break;
    }
    *energy += e;
    return g;
}

// Pass 1: gradient (render + regularisers) into m/v, reading x only; pass 2
// applies the parameter update, so stencils read the pre-step values.
FR_D int group_of_block(const GroupTable& T) {
    int lo = 0, hi = T.n_groups - 1;          // last group whose start <= blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.block_start[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(ADAM_THREADS) k_adam_moments(GroupTable T, double* energy) {
    __shared__ double part[ADAM_THREADS / 32];
    const int gi = group_of_block(T);
    const fr_opt_group& G = T.g[gi];
    const int i = (blockIdx.x - T.block_start[gi]) * ADAM_THREADS + threadIdx.x;
    double e = 0.0;
    if (i < G.n) {
        const float x = G.x[i];
        float g = G.g ? G.g[i] : 0.0f;
        g += reg_grad(G, i, x, &e);
        const float m = T.beta1 * G.m[i] + (1.0f - T.beta1) * g;
        const float v = T.beta2 * G.v[i] + (1.0f - T.beta2) * g * g;
        G.m[i] = m;
        G.v[i] = v;
    }
    if (energy) {
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = e;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < ADAM_THREADS / 32; ++w) s += part[w];
            if (s != 0.0) atomicAdd(energy, s);
        }
    }
}

__global__ void __launch_bounds__(ADAM_THREADS) k_adam_apply(GroupTable T) {
    const int gi = group_of_block(T);
    const fr_opt_group& G = T.g[gi];
    const int i = (blockIdx.x - T.block_start[gi]) * ADAM_THREADS + threadIdx.x;
    if (i >= G.n) return;
    const float mh = G.m[i] / T.bc1[gi], vh = G.v[i] / T.bc2[gi];
    float x = G.x[i] - G.lr * mh / (sqrtf(vh) + T.eps);
    if (G.clamp_lo < G.clamp_hi) x = fminf(fmaxf(x, G.clamp_lo), G.clamp_hi);
    G.x[i] = x;
}

}  // namespace

extern "C" fr_status fr_adam(const fr_opt_group* groups, int32_t n_groups, int32_t step, float beta1, float beta2,
                             float eps, double* reg_energy, void* stream) {
    if (!groups || n_groups < 1 || n_groups > FR_MAX_OPT_GROUPS || step < 1) return FR_EINVAL;
    GroupTable T;
    int blocks = 0;
    for (int k = 0; k < n_groups; ++k) {
        const fr_opt_group& G = groups[k];
        if (!G.x || !G.m || !G.v || G.n < 0) return FR_EINVAL;
        if ((G.kind == FR_GROUP_TEX_RGB || G.kind == FR_GROUP_TEX_MONO) &&
            (G.width < 1 || (long)G.width * G.width * (G.kind == FR_GROUP_TEX_RGB ? 3 : 1) != G.n))
            return FR_EINVAL;
        if (G.kind == FR_GROUP_LIGHT && ((!G.aux && !G.aux2) || G.n % 3 != 0)) return FR_EINVAL;
        if (G.kind == FR_GROUP_STAGE && (!G.aux || G.n % 4 != 0)) return FR_EINVAL;
        T.g[k] = G;
        const int st_k = G.step > 0 ? G.step : step;
        T.bc1[k] = (float)(1.0 - pow((double)beta1, st_k));
        T.bc2[k] = (float)(1.0 - pow((double)beta2, st_k));
        T.block_start[k] = blocks;
        blocks += (G.n + ADAM_THREADS - 1) / ADAM_THREADS;
    }
    T.block_start[n_groups] = blocks;
    T.n_groups = n_groups;
    T.beta1 = beta1;
    T.beta2 = beta2;
    T.eps = eps;
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (reg_energy) cudaMemsetAsync(reg_energy, 0, sizeof(double), st);
    if (blocks > 0) {
        k_adam_moments<<<blocks, ADAM_THREADS, 0, st>>>(T, reg_energy);
        k_adam_apply<<<blocks, ADAM_THREADS, 0, st>>>(T);
        fr_count_launches(2);
    }
    return cudaGetLastError() == cudaSuccess ? FR_OK : FR_ECUDA;
}
