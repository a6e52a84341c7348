// Batched linear model on the 5th-generation tensor cores, for every face of a
// batch at once: the morph of Sec. 3.1 (v = a_s + [Sigma_s | Sigma_e]
// [alpha; delta]) and the statistical albedos of Sec. 3.2 (C = a_r +
// Sigma_r beta, S = a_b + Sigma_b gamma in texture space):
//     D[i][b] = sum_k basis[i][k] coef[b][k]      (BF16 x BF16 -> FP32 in TMEM)
//     y_b[i]  = mean[i] + D[i][b]                 (FP32 epilogue)
// One CTA owns 128 rows i of the 3N dimension and all faces of the batch,
// padded to the MMA width N (32, or 64 for batches of 33 to 64 faces).  The
// basis tile (pre-arranged at set-up in the no-swizzle K-major core-matrix
// layout, 8 rows x 16 bytes per core matrix) and the gathered coefficient tile
// arrive by two bulk asynchronous copies completing on one mbarrier; a single
// thread issues K/16 tcgen05.mma instructions into a 128 x N FP32 TMEM
// accumulator; four warps read it back with tcgen05.ld (32 columns at a time)
// and write v_b.
// Every wait is bounded: on a timeout the CTA sets the status word, waits
// (bounded) for its own copies, frees its TMEM and returns.
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int TC_M = 128;        // rows per CTA (TMEM lanes)
constexpr int TC_N_MAX = 64;     // widest MMA: faces per call, padded
constexpr int TC_THREADS = 128;
constexpr unsigned SPIN_LIMIT = 1u << 22;

FR_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the fixed
// version bits 46-48 = 0b001, no swizzle (bits 61-63 = 0).
FR_D uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: D = FP32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28.
template <int N>
__host__ __device__ constexpr uint32_t idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

FR_D void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

FR_D bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned limit = SPIN_LIMIT) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// 32 TMEM columns (one per face) of this thread's row, from column c0
FR_D void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

template <int TC_N>
__global__ void __launch_bounds__(TC_THREADS) k_morph_tc(const uint16_t* __restrict__ basis_tiles, int Kp,
                                                         const uint16_t* __restrict__ coef_tile,
                                                         const float* __restrict__ mean, int n3, LinearTable t,
                                                         int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const int a_bytes = TC_M * Kp * 2, b_bytes = TC_N * Kp * 2;
    unsigned char* sA = smem;
    unsigned char* sB = smem + a_bytes;
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tile = blockIdx.x;

    if (tid == 0) {
        mbar_init(&bar_load, 1);
        mbar_init(&bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (tid == 0) {
        const uint32_t bar = smem_u32(&bar_load);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(a_bytes + b_bytes)
                     : "memory");
        const unsigned char* srcA = reinterpret_cast<const unsigned char*>(basis_tiles) + (size_t)tile * a_bytes;
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(sA)), "l"(srcA), "r"(a_bytes), "r"(bar)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(smem_u32(sB)), "l"(coef_tile), "r"(b_bytes), "r"(bar)
                     : "memory");
    }
    // every thread waits for the operands (bounded); the outcome is made uniform
    const bool go = __syncthreads_and(mbar_wait(&bar_load, 0) ? 1 : 0) != 0;

    const uint32_t tmem = tmem_base;
    if (go && tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // K-major, no swizzle: core matrices adjacent in K are 128 B apart
        // (leading offset), 8-row groups are (Kp / 8) * 128 B apart (stride offset)
        const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
        for (int ks = 0; ks < Kp / 16; ++ks) {
            const uint64_t da = smem_desc(smem_u32(sA) + ks * 256, 128, sbo);
            const uint64_t db = smem_desc(smem_u32(sB) + ks * 256, 128, sbo);
            const uint32_t acc = ks > 0 ? 1u : 0u;
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                ::"r"(tmem), "l"(da), "l"(db), "r"(idesc<TC_N>()), "r"(acc)
                : "memory");
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(smem_u32(&bar_mma))
                     : "memory");
    }
    const bool done = go && __syncthreads_and(mbar_wait(&bar_mma, 0) ? 1 : 0) != 0;
    if (done) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int row = tile * TC_M + tid;
        const float m = row < n3 ? mean[row] : 0.0f;
        // warp w reads TMEM lanes 32w..32w+31 (its rows), 32 columns per load;
        // every warp executes every load (the loads are warp-collective)
#pragma unroll
        for (int c0 = 0; c0 < TC_N; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < n3) {
#pragma unroll
                for (int b = 0; b < 32; ++b)
                    if (c0 + b < t.n) t.out[c0 + b][row] = m + __uint_as_float(r[b]);
            }
        }
    } else if (tid == 0) {
        // a wait gave up: report it, then give this CTA's own copies or MMAs a
        // second bounded wait before its TMEM is freed and it exits
        set_status(status, FR_STATUS_TIMEOUT);
        if (!go) mbar_wait(&bar_load, 0);
        else mbar_wait(&bar_mma, 0);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
    }
}

// The bounded-wait error path on its own: one CTA waits on an mbarrier that
// nothing arrives at, gives up after `limit` polls with the same loop as the
// morph kernel's waits, and reports FR_STATUS_TIMEOUT.
__global__ void k_wait_probe(unsigned limit, int* status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, limit);
    if (!ok && threadIdx.x == 0) set_status(status, FR_STATUS_TIMEOUT);
}

FR_D uint16_t bf16_rne(float f) {
    uint32_t u = __float_as_uint(f);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

// Gather the batch's coefficients into the B-operand tile: face b is row b of
// an N x Kp K-major matrix in core-matrix layout (8 rows x 8 BF16 per 128 B).
__global__ void k_coef_tile(LinearTable t, int K, int Kp, int TC_N, uint16_t* tile) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= TC_N * Kp) return;
    const int b = idx / Kp, k = idx % Kp;
    const float v = (b < t.n && k < K) ? t.coef[b][k] : 0.0f;
    const int g = b >> 3, r = b & 7, c = k >> 3, kk = k & 7;
    tile[((g * (Kp / 8) + c) * 128 + r * 16 + kk * 2) / 2] = bf16_rne(v);
}

}  // namespace

int morph_tc_smem_bytes(int Kp) { return TC_M * Kp * 2 + TC_N_MAX * Kp * 2; }
int morph_tc_coef_tile_elems(int Kp) { return TC_N_MAX * Kp; }

void launch_linear_tc(const uint16_t* tiles, int Kp, int K, uint16_t* coef_tile, const float* mean, int rows,
                      const LinearTable& t, int* status, cudaStream_t st) {
    if (t.n <= 0 || rows <= 0 || t.n > TC_N_MAX) return;
    const int N = t.n <= 32 ? 32 : 64;           // MMA width: the batch padded to 32 or 64 faces
    k_coef_tile<<<(N * Kp + 255) / 256, 256, 0, st>>>(t, K, Kp, N, coef_tile);
    const int n_tiles = (rows + TC_M - 1) / TC_M;
    const int smem = TC_M * Kp * 2 + N * Kp * 2;
    if (N == 32) {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_morph_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_morph_tc<32><<<n_tiles, TC_THREADS, smem, st>>>(tiles, Kp, coef_tile, mean, rows, t, status);
    } else {
        if (smem > 48 * 1024) cudaFuncSetAttribute(k_morph_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k_morph_tc<64><<<n_tiles, TC_THREADS, smem, st>>>(tiles, Kp, coef_tile, mean, rows, t, status);
    }
    fr_count_launches(2);
}

void launch_wait_probe(unsigned limit, int* status, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(limit, status);
    fr_count_launches(1);
}
