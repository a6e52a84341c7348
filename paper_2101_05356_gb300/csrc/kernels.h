// Launcher declarations shared between the kernel translation units and the
// C-ABI implementation.
#pragma once
#include "common.cuh"

struct EdgeLists {
    const int4* edges;   // [E] (a, b, f1, f2), a < b, f2 = -1 on the boundary
    int* prim_list;      // [E]   ordered primary silhouettes (compacted list 0)
    int* prim_count;     // [1]
    int* light_list;     // [NL][E] ordered shadow candidates (lists 1..NL)
    int* light_count;    // [NL]
};

struct BvhScratch {
    uint32_t *keys, *keys_alt;
    int *vals, *vals_alt;
    int* hist;           // [256][n_tiles]
    int* child;          // [2 (T - 1)] child codes of internal nodes
    int* parent_int;     // [T - 1]
    int* parent_leaf;    // [T]
    int* flag;           // [T - 1]
    float4* box_int;     // [2 (T - 1)] lo, hi
    float4* box_leaf;    // [2 T]
    unsigned* aabb;      // [6] ordered-int scene bounds
};

// geometry.cu
void launch_morph(const float* mean, const float* basis, int ld, int K, const float* coef, float* v_model,
                  cudaStream_t st);
void launch_pose(const float* v_model, int N, const float* rot, const float* trans, float4* v_cam,
                 unsigned* aabb, cudaStream_t st);
void launch_faces(const float4* v_cam, const int4* faces, int T, const unsigned* aabb, float4* n_face,
                  uint32_t* keys, int* vals, cudaStream_t st);
void launch_vertex_normals(const float4* n_face, const int* vf_off, const int* vf_idx, int N, float4* vn,
                           cudaStream_t st);
void launch_normals_adjoint(const float4* v_cam, const float4* vn, const float* d_n, const int4* faces,
                            const int* vf_off, const int* vf_idx, int N, float* dm, float* d_v,
                            cudaStream_t st);
void launch_pose_adjoint(const float* v_model, int N, int ld, const float* rot, const float* trans,
                         const float* d_v, float* d_vmodel, double* acc12, cudaStream_t st);
void launch_pose_finish(const float* rot, const double* acc12, const double* small, int NL, float* g_rot,
                        float* g_trans, float* g_focal, float* g_light, cudaStream_t st);
void launch_morph_adjoint(const float* basis, int ld, int K, int n3, const float* d_vmodel, float* g_coef,
                          cudaStream_t st);

// lbvh.cu
void launch_lbvh(const float4* v_cam, const int4* faces, int T, BvhScratch& B, BvhNode* nodes, float4* tris,
                 int* status, cudaStream_t st);
void launch_bvh_check(const BvhNode* nodes, const BvhScratch& B, int T, int* out, cudaStream_t st);

// render.cu
void launch_forward(const DevScene& S, const DevParams& P, float* image, int32_t* tri_rec, uint64_t* mask_rec,
                    uint32_t iteration, uint32_t face, cudaStream_t st);
void launch_adjoint(const DevScene& S, const DevParams& P, const DevGrads& G, const EdgeLists& EL,
                    const float* adj_image, uint32_t iteration, uint32_t face, cudaStream_t st);
void launch_edge_primary(const DevScene& S, const DevParams& P, const DevGrads& G, const EdgeLists& EL,
                         const float* adj_image, uint32_t iteration, uint32_t face, cudaStream_t st);
void launch_classify(const DevScene& S, const EdgeLists& EL, uint8_t* flags, cudaStream_t st);
void launch_trace_rays(const DevScene& S, const float* org, const float* dir, int n, int32_t* tri, float* t,
                       cudaStream_t st);

// loss.cu
void launch_loss(int H, int W, const float* image, const float* target, double* loss, float* sign,
                 float* blurred, float* adj_image, cudaStream_t st);

// process-wide count of kernels launched by this library (api.cu)
void fr_count_launches(int n);

// misc
void launch_philox(uint32_t k0, uint32_t k1, const uint32_t* counters, int n, uint32_t* out, cudaStream_t st);
