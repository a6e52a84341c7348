// Batched linear model on the 5th-generation tensor cores, for every face of a
// batch at once: the morph of Sec. 3.1 (v = a_s + [Sigma_s | Sigma_e]
// [alpha; delta]) and the statistical albedos of Sec. 3.2 (C = a_r +
// Sigma_r beta, S = a_b + Sigma_b gamma in texture space):
//     D[i][b] = sum_k basis[i][k] coef[b][k]      (BF16 x BF16 -> FP32 in TMEM)
//     y_b[i]  = mean[i] + D[i][b]                 (FP32 epilogue)
// The basis is pre-arranged at set-up as 128-row tiles in the no-swizzle
// K-major core-matrix layout (8 rows x 16 bytes per core matrix); every CTA
// gathers the batch's coefficients into one B tile in shared memory (BF16,
// the same layout), padded to the MMA width N (32, or 64 for batches of 33 to
// 64 faces).
//
// The kernel is persistent and warp-specialised: each CTA walks the row tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... of the basis.  A producer warp keeps
// a ring of `stages` shared-memory buffers filled with bulk asynchronous copies
// of the tiles (one "full" and one "empty" mbarrier per buffer); an MMA warp
// issues each tile's K/16 tcgen05.mma instructions into one of two 128 x N
// FP32 TMEM accumulators as soon as its copy has landed and the accumulator is
// free, and commits them to the buffer's "empty" barrier and the accumulator's
// "full" barrier; four epilogue warps read a finished accumulator back with
// tcgen05.ld, write y_b and release it.  So copies, MMAs and epilogues of
// consecutive tiles overlap, and the basis streams from HBM at the copy rate.
// Every wait is bounded: a role whose wait gives up sets the status word and
// stops; the others then give up in turn.  Before the CTA frees its TMEM and
// exits it gives the last copy into every buffer and the last MMAs of both
// accumulators a second bounded wait; if one of those also gives up it sets
// FR_STATUS_TIMEOUT_UNSAFE as well (a late write may land in shared memory or
// TMEM that a later CTA has been given, so the host treats the context as
// unusable from then on).
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr int TC_M = 128;        // rows per tile (TMEM lanes)
constexpr int TC_N_MAX = 64;     // widest MMA: faces per call, padded
constexpr int TC_EPI_WARPS = 4;             // epilogue warps: TMEM lanes 32w..32w+31
constexpr int TC_PRODUCER = 4, TC_MMA = 5;   // warp indices of the copy and MMA roles
constexpr int TC_THREADS = 32 * (TC_EPI_WARPS + 2);
constexpr int TC_MAX_STAGES = 8;
constexpr int TC_STAGE_BYTES = 32 * 1024;   // shared memory given to the ring of basis tiles (at
                                            // least two; measured on GB300, albedo K = 80: two 20 KB
                                            // stages and four CTAs per SM 0.060 ms, three stages 0.062,
                                            // four 0.066, six 0.089)
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

FR_D void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    const uint32_t b = smem_u32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(b)
                 : "memory");
}

FR_D uint16_t bf16_rne(float f) {
    uint32_t u = __float_as_uint(f);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

FR_D void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

FR_D void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar))
                 : "memory");
}

// The models of one launch (up to two, e.g. the diffuse and specular
// albedos): row tiles are numbered across them, model 0's first.
struct TcLaunch {
    int n;                       // models (1 or 2)
    int tiles0;                  // row tiles of model 0 (model 1's follow)
    const uint16_t* basis[2];    // operand tiles [ceil(rows / 128)][128][Kp]
    const float* mean[2];
    int K[2], Kp[2], rows[2];
    LinearTable t[2];
};

template <int TC_N>
__global__ void __launch_bounds__(TC_THREADS) k_morph_tc(TcLaunch L, int n_tiles, int stage_bytes, int stages,
                                                         int* status) {
    extern __shared__ __align__(1024) unsigned char smem[];
    // one B tile per model ([N][Kp] BF16, each a multiple of 1024 bytes), then
    // the ring of stage_bytes buffers for the basis tiles
    unsigned char* sB[2] = {smem, smem + TC_N * L.Kp[0] * 2};
    unsigned char* sA0 = smem + TC_N * L.Kp[0] * 2 + (L.n > 1 ? TC_N * L.Kp[1] * 2 : 0);
    __shared__ __align__(8) uint64_t full[TC_MAX_STAGES], empty[TC_MAX_STAGES], tfull[2], tempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, issued_loads, issued_mma;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this CTA's tiles: blockIdx.x + k * gridDim.x for k < my_n
    const int my_n = ((int)blockIdx.x < n_tiles) ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto tile_of = [&](int k, int& model) {             // local tile index and model of tile k
        const int g = (int)blockIdx.x + k * (int)gridDim.x;
        model = g < L.tiles0 ? 0 : 1;
        return model ? g - L.tiles0 : g;
    };

    if (tid == 0) {
        for (int q = 0; q < stages; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], 32 * TC_EPI_WARPS);
        }
        abort_flag = 0;
        issued_loads = issued_mma = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&tmem_base)), "r"(2 * TC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();                                    // the barriers are initialised
    // the ring's first copies wait on nothing: issue them before the coefficient
    // gather below, so that their latency overlaps the gather's
    const int pre = my_n < stages ? my_n : stages;
    if (warp == TC_PRODUCER && lane == 0) {
        for (int k = 0; k < pre; ++k) {
            int mdl;
            const int lt = tile_of(k, mdl);
            const int a_bytes = TC_M * L.Kp[mdl] * 2;
            bulk_load(sA0 + (size_t)k * stage_bytes,
                      reinterpret_cast<const unsigned char*>(L.basis[mdl]) + (size_t)lt * a_bytes, a_bytes, &full[k]);
        }
    }
    // the B operands: face b is row b of an N x Kp K-major matrix in core-matrix
    // layout (8 rows x 8 BF16 per 128 B), coefficients rounded to nearest even;
    // the loads of both models are issued before any store (one round trip for
    // batches of up to 4 * TC_THREADS / Kp faces); the writes are made visible
    // to the tensor cores' (async proxy) reads
    constexpr int GU = 4;
    const int g_total = TC_N * (L.Kp[0] > L.Kp[1] || L.n < 2 ? L.Kp[0] : L.Kp[1]);
    for (int base = 0; base < g_total; base += GU * TC_THREADS) {
        float v[2][GU];
#pragma unroll
        for (int mdl = 0; mdl < 2; ++mdl) {
            const int Kp = mdl < L.n ? L.Kp[mdl] : 16, K = L.K[mdl];     // (no second model: no loads)
            const LinearTable& t = L.t[mdl];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int idx = base + u * TC_THREADS + tid;
                const int b = idx / Kp, k = idx - b * Kp;
                v[mdl][u] = (mdl < L.n && idx < TC_N * Kp && b < t.n && k < K) ? __ldg(&t.coef[b][k]) : 0.0f;
            }
        }
#pragma unroll
        for (int mdl = 0; mdl < 2; ++mdl) {
            if (mdl >= L.n) break;
            uint16_t* sB16 = reinterpret_cast<uint16_t*>(sB[mdl]);
            const int Kp = L.Kp[mdl];
#pragma unroll
            for (int u = 0; u < GU; ++u) {
                const int idx = base + u * TC_THREADS + tid;
                if (idx < TC_N * Kp) {
                    const int b = idx / Kp, k = idx - b * Kp;
                    const int g = b >> 3, r = b & 7, c = k >> 3, kk = k & 7;
                    sB16[((g * (Kp / 8) + c) * 128 + r * 16 + kk * 2) / 2] = bf16_rne(v[mdl][u]);
                }
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    volatile int* abort_v = &abort_flag;

    if (warp == TC_PRODUCER) {
        if (lane == 0) {
            int k = pre;
            for (; k < my_n && !*abort_v; ++k) {
                const int q = k % stages;
                // the buffer's previous tile (k - stages) must have been consumed
                if (k >= stages && !mbar_wait(&empty[q], (uint32_t)(k / stages - 1) & 1u)) {
                    set_status(status, FR_STATUS_TIMEOUT);
                    *abort_v = 1;
                    break;
                }
                int mdl;
                const int lt = tile_of(k, mdl);
                const int a_bytes = TC_M * L.Kp[mdl] * 2;
                bulk_load(sA0 + (size_t)q * stage_bytes,
                          reinterpret_cast<const unsigned char*>(L.basis[mdl]) + (size_t)lt * a_bytes, a_bytes,
                          &full[q]);
            }
            issued_loads = k;
        }
    } else if (warp == TC_MMA) {
        if (lane == 0) {
            int k = 0;
            for (; k < my_n && !*abort_v; ++k) {
                const int q = k % stages, b = k & 1;
                bool ok = mbar_wait(&full[q], (uint32_t)(k / stages) & 1u);
                // accumulator b is free once the epilogue has read tile k - 2
                if (ok && k >= 2) ok = mbar_wait(&tempty[b], (uint32_t)((k >> 1) - 1) & 1u);
                if (!ok) {
                    set_status(status, FR_STATUS_TIMEOUT);
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                int mdl;
                tile_of(k, mdl);
                const int Kp = L.Kp[mdl];
                // K-major, no swizzle: core matrices adjacent in K are 128 B apart
                // (leading offset), 8-row groups are (Kp / 8) * 128 B apart (stride offset)
                const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
                const unsigned char* sA = sA0 + (size_t)q * stage_bytes;
                const uint32_t acc_addr = tmem + (uint32_t)(b * TC_N);
                for (int ks = 0; ks < Kp / 16; ++ks) {
                    const uint64_t da = smem_desc(smem_u32(sA) + ks * 256, 128, sbo);
                    const uint64_t db = smem_desc(smem_u32(sB[mdl]) + ks * 256, 128, sbo);
                    const uint32_t acc = ks > 0 ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                        ::"r"(acc_addr), "l"(da), "l"(db), "r"(idesc<TC_N>()), "r"(acc)
                        : "memory");
                }
                mma_commit(&empty[q]);          // the buffer may be refilled
                mma_commit(&tfull[b]);          // the accumulator may be read
            }
            issued_mma = k;
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (its rows of the tile),
        // 32 columns per load; every warp executes every load (warp-collective)
        for (int k = 0; k < my_n; ++k) {
            const int b = k & 1;
            // a bounded wait that also gives up as soon as another role has
            const uint32_t a = smem_u32(&tfull[b]);
            bool ok = false;
            for (unsigned it = 0; it < SPIN_LIMIT && !ok; ++it) {
                uint32_t done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(a), "r"((uint32_t)(k >> 1) & 1u)
                    : "memory");
                ok = done != 0;
                if (!ok && *abort_v) break;
            }
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0 && !*abort_v) {
                    set_status(status, FR_STATUS_TIMEOUT);
                    *abort_v = 1;
                }
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int mdl;
            const int row = tile_of(k, mdl) * TC_M + tid;
            const int n3 = L.rows[mdl];
            const LinearTable& t = L.t[mdl];
            const float m = row < n3 ? __ldg(&L.mean[mdl][row]) : 0.0f;
#pragma unroll
            for (int c0 = 0; c0 < TC_N; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(b * TC_N + c0), r);
                if (row < n3) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (c0 + j < t.n) t.out[c0 + j][row] = m + __uint_as_float(r[j]);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&tempty[b]);
        }
    }
    __syncthreads();
    if (tid == 0 && abort_flag) {
        // a wait gave up: give the last copy into every buffer and the last
        // MMAs of both accumulators a second bounded wait before the TMEM is
        // freed and the shared memory released
        bool drained = true;
        for (int q = 0; q < stages; ++q) {
            const int last = issued_loads - 1 - ((issued_loads - 1 - q) % stages + stages) % stages;
            if (last >= 0 && last % stages == q) drained &= mbar_wait(&full[q], (uint32_t)(last / stages) & 1u);
        }
        for (int b = 0; b < 2; ++b) {
            const int last = issued_mma - 1 - (((issued_mma - 1 - b) % 2) + 2) % 2;
            if (last >= 0 && (last & 1) == b) drained &= mbar_wait(&tfull[b], (uint32_t)(last >> 1) & 1u);
        }
        if (!drained) set_status(status, FR_STATUS_TIMEOUT_UNSAFE);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TC_N));
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


}  // namespace

int morph_tc_stages(int Kp) {
    const int a_bytes = TC_M * Kp * 2;
    const int st = TC_STAGE_BYTES / a_bytes;
    return st < 2 ? 2 : (st > TC_MAX_STAGES ? TC_MAX_STAGES : st);
}
int morph_tc_smem_bytes(int Kp) { return 2 * TC_N_MAX * Kp * 2 + morph_tc_stages(Kp) * TC_M * Kp * 2; }

namespace {

// Persistent grid: as many CTAs per SM as its shared memory, its TMEM (512
// columns, two N-column accumulators per CTA) and its threads allow, with the
// shared-memory carveout at its maximum (the kernel uses no L1 data cache to
// speak of).  Queried once per host thread, device, MMA width and ring size.
template <int N>
int morph_tc_grid(int n_tiles, int smem) {
    thread_local int cached_smem = -1, cached_dev = -1, per_sm = 1, sms = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cached_smem != smem || cached_dev != dev) {
        int smem_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncSetAttribute(k_morph_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cudaFuncSetAttribute(k_morph_tc<N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k_morph_tc<N>);
        const int per_cta = smem + (int)fa.sharedSizeBytes + 1024;     // + the per-CTA reservation
        per_sm = smem_sm / per_cta;
        per_sm = per_sm < 512 / (2 * N) ? per_sm : 512 / (2 * N);
        per_sm = per_sm < 2048 / TC_THREADS ? per_sm : 2048 / TC_THREADS;
        if (per_sm < 1) per_sm = 1;
        cached_smem = smem;
        cached_dev = dev;
    }
    const int g = (sms > 0 ? sms : 1) * per_sm;
    return n_tiles < g ? n_tiles : g;
}

}  // namespace

void launch_linear_tc(const TcModel* models, int n_models, int* status, cudaStream_t st) {
    TcLaunch L{};
    int n_faces = 0, max_kp = 0, n_tiles = 0;
    for (int q = 0; q < n_models && L.n < 2; ++q) {
        const TcModel& m = models[q];
        if (m.t.n <= 0 || m.rows <= 0 || m.t.n > TC_N_MAX || m.K <= 0) continue;
        const int i = L.n++;
        L.basis[i] = m.tiles; L.mean[i] = m.mean; L.K[i] = m.K; L.Kp[i] = m.Kp; L.rows[i] = m.rows; L.t[i] = m.t;
        const int nt = (m.rows + TC_M - 1) / TC_M;
        if (i == 0) L.tiles0 = nt;
        n_tiles += nt;
        n_faces = n_faces > m.t.n ? n_faces : m.t.n;
        max_kp = max_kp > m.Kp ? max_kp : m.Kp;
    }
    if (L.n == 0) return;
    const int N = n_faces <= 32 ? 32 : 64;       // MMA width: the batch padded to 32 or 64 faces
    const int stages = morph_tc_stages(max_kp);
    const int stage_bytes = TC_M * max_kp * 2;
    int smem = stages * stage_bytes;
    for (int i = 0; i < L.n; ++i) smem += N * L.Kp[i] * 2;
    if (N == 32) {
        const int g = morph_tc_grid<32>(n_tiles, smem);
        k_morph_tc<32><<<g, TC_THREADS, smem, st>>>(L, n_tiles, stage_bytes, stages, status);
    } else {
        const int g = morph_tc_grid<64>(n_tiles, smem);
        k_morph_tc<64><<<g, TC_THREADS, smem, st>>>(L, n_tiles, stage_bytes, stages, status);
    }
    fr_count_launches(1);
}

void launch_wait_probe(unsigned limit, int* status, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(limit, status);
    fr_count_launches(1);
}
