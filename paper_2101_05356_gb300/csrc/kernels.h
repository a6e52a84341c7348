// Launcher declarations shared between the kernel translation units and the
// C-ABI implementation.  Batched launchers take the device item table (one
// DevItem per face) and the number of items.
#pragma once
#include <vector>

#include "common.cuh"

// process-wide count of kernels launched by this library (api.cu)
void fr_count_launches(int n);

// geometry.cu
void launch_set_items(const DevItem* host_items, int n, DevItem* dev_items, cudaStream_t st);
void launch_zero_accumulators(const DevItem* items, int n, int N, int M, cudaStream_t st);
void launch_tex_flush(const DevItem* items, int n, int M, cudaStream_t st);
void launch_pose(const DevItem* items, int n, int N, cudaStream_t st);
void launch_stage_lights(const DevItem* items, int n, int NL, cudaStream_t st);
void launch_faces(const DevItem* items, int n, const int4* faces, int T, cudaStream_t st);
void launch_vertex_normals(const DevItem* items, int n, const int* vf_off, const int* vf_idx, int N,
                           cudaStream_t st);
void launch_normals_adjoint(const DevItem* items, int n, const int4* faces, const int* vf_off,
                            const int* vf_idx, int N, cudaStream_t st);
void launch_pose_adjoint(const DevItem* items, int n, int N, cudaStream_t st);
void launch_pose_finish(const DevItem* items, int n, int NL, int N, cudaStream_t st);

// linear.cu: y_b = mean + basis * coef_b for the faces of a batch (shape morph,
// statistical albedo); basis [K][ld] FP32, mean [ld], rows <= ld, ld % 4 == 0,
// outputs and adjoint inputs 16-byte aligned.  Tables are passed by value.
struct LinearTable {
    int n;
    const float* coef[FR_MAX_BATCH];     // [K] per face (device)
    float* out[FR_MAX_BATCH];            // [rows] per face (device)
};
struct LinearAdjTable {
    int n;
    const float* g[FR_MAX_BATCH];        // dE/dy_b [rows] (device)
    float* g_coef[FR_MAX_BATCH];         // += basis^T g_b [K] (device; null: skipped)
};
int linear_adj_chunks(int rows);         // size of the adjoint's FP64 partials: n * K * chunks
void launch_linear(const float* mean, const float* basis, int ld, int rows, int K, const LinearTable& t,
                   cudaStream_t st);
// One linear model's transpose: part = its FP64 partials [linear_adj_chunks(rows)][FR_MAX_BATCH][K].
struct LinearAdjModel {
    const float* basis;
    int ld, rows, K;
    double* part;
    LinearAdjTable t;
};
// g_coef_b += basis^T g_b for every model (at most two per launch, the same faces).
void launch_linear_adjoint(const LinearAdjModel* models, int n_models, cudaStream_t st);

// morph_tc.cu: the same forward as one BF16 tensor-core GEMM over the batch
// (tiles: the basis as [ceil(rows / 128)][128][Kp] BF16 operand tiles); one
// launch takes up to two models (the diffuse and specular albedos)
struct TcModel {
    const uint16_t* tiles;
    int Kp, K;
    const float* mean;
    int rows;
    LinearTable t;
};
int morph_tc_smem_bytes(int Kp);
void launch_wait_probe(unsigned limit, int* status, cudaStream_t st);
void launch_linear_tc(const TcModel* models, int n_models, int* status, cudaStream_t st);

// landmark.cu: sparse landmark loss (one block; L <= 256)
struct LandmarkArgs {
    const float* mean;          // shape mean [ld]
    const float* basis;         // shape basis [K][ld]
    int ld, K;
    const int* idx;             // landmark vertex indices [L]
    int L, W, H;
    const float *coef, *rot, *trans, *focal;
    const float* z;             // target pixel positions [L][2]
    float weight;
    double* loss;               // set to weight * E_land
    float* proj;                // projected landmarks [L][2] (may be null)
    float *g_coef, *g_rot, *g_trans, *g_focal;   // += weight * dE_land (each may be null)
};
void launch_landmarks(const LandmarkArgs& a, cudaStream_t st);

// api.cu: what the native server (server.cu) needs to know about a context
struct fr_ctx;
struct CtxInfo {
    int width = 0, height = 0, spp = 0, tex = 0, K = 0, NL = 0, max_batch = 0, n_landmarks = 0;
    int k_diffuse = 0, k_specular = 0;
    uint32_t flags = 0;
    bool ready = false, have_albedo = false, have_stage = false;
    int env_size = 0;                 // environment map side (0: no environment blocks)
    std::vector<float> light_da;      // [d (N_L) | a (N_L)] of the light records
};
void ctx_info(const fr_ctx* c, CtxInfo& out);

// bvh_topology.cu (host): static binned-SAH topology of a mesh, in the
// BvhScratch encoding (child codes ~leaf slot / internal index, root 0)
struct BvhTopology {
    std::vector<int> child, parent_int, parent_leaf, vals;
};
void build_bvh_topology(const float* v, const int* faces, int T, BvhTopology& out);

// lbvh.cu: rebuild = Morton sort + Karras radix tree per call; otherwise the
// items' BvhScratch carries a fixed topology and only the boxes are refitted
void launch_lbvh(const DevItem* items, int n, const int4* faces, int T, int* status, bool rebuild,
                 cudaStream_t st);
void launch_bvh_check(const DevItem* items, int T, int* out, cudaStream_t st);

// render.cu
// the ray kernels process camera samples [q0, q0 + count) of each item, count
// from the block map; records_only: the adjoint's records of that tile only
void launch_forward(const DevItem* items, const BlockMap& map, bool env, long q0, bool records_only,
                    cudaStream_t st);
void launch_adjoint(const DevItem* items, const BlockMap& map, int NL, bool all_recorded, bool any_stage, bool env,
                    long q0, cudaStream_t st);
void launch_edge_order(const DevItem* items, int n, long max_edge, cudaStream_t st);
void launch_edge_primary(const DevItem* items, const BlockMap& map, bool env, cudaStream_t st);
void launch_classify(const DevItem* items, int n, int E, int NL, int T, cudaStream_t st);
void launch_spec_candidates(const DevItem* items, int n, int T, const BlockMap& map, cudaStream_t st);
void launch_edge_specular(const DevItem* items, const BlockMap& map, bool env, cudaStream_t st);
void launch_trace_rays(const DevItem* items, const float* org, const float* dir, int n, int32_t* tri,
                       float* t, cudaStream_t st);

// loss.cu: per-image arguments passed by value (no device table needed).
// part: FR_LOSS_PARTS doubles of scratch for the per-block partial sums.
constexpr int FR_LOSS_PARTS = 1024;
struct LossItem {
    int H, W;
    const float* image;
    const float* target;
    double* loss;
    float* sign;
    double* part;
    float* blurred;
    float* adj;
};
struct LossTable {
    int n;
    int max_px3;
    LossItem it[FR_MAX_BATCH];
};
void launch_loss(const LossTable& t, cudaStream_t st);
void launch_loss(int H, int W, const float* image, const float* target, double* loss, float* sign, double* part,
                 float* blurred, float* adj_image, cudaStream_t st);

// misc
void launch_philox(uint32_t k0, uint32_t k1, const uint32_t* counters, int n, uint32_t* out, cudaStream_t st);
