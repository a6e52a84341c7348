// C-ABI of the facert library: context, slot scratch ownership, argument checks
// and the orchestration of the hot path (include/facert.h documents each call).
//
// A context holds one face model and light stage and `max_batch` slots of
// per-face scratch (geometry, BVH, edge lists, adjoint accumulators, loss
// scratch).  Every compute call is a batch: item k uses slot k, the item table
// is written to device memory by one small kernel, and every stage is one
// launch over all items.  The single-face calls are batches of one.
#include <algorithm>
#include <cstdint>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/facert.h"
#include "common.cuh"
#include "kernels.h"

namespace {

struct Slot {
    float* v_model = nullptr;
    float* d_vmodel = nullptr;
    float4* v_cam = nullptr;
    float4* vn = nullptr;
    float4* n_face = nullptr;
    BvhScratch B{};
    BvhNode* nodes = nullptr;
    float4* tris = nullptr;
    int* slot_of = nullptr;
    uint8_t* sil_flags = nullptr;
    int* lists = nullptr;
    int* counts = nullptr;
    fix64* d_v = nullptr;
    fix64* d_n = nullptr;
    fix64* tex = nullptr;
    float* dm = nullptr;
    fix64* small = nullptr;
    double* pose_part = nullptr;
    float* sign = nullptr;
    double* loss_part = nullptr;     // per-block loss partials [FR_LOSS_PARTS]
    float* adj_image = nullptr;
    LightDev* lights = nullptr;      // lights built from stage parameters [FR_MAX_LIGHTS]
    int* edge_perm = nullptr;        // primary-edge sample order [edge_cap]
    long edge_cap = 0;
    int* spec_list = nullptr;        // specular-boundary candidates [T], their boxes, counts
    float4* spec_box = nullptr;
    int* spec_hist = nullptr;
    int* spec_count = nullptr;
    uint8_t* spec_flag = nullptr;
    int32_t* rec_tri = nullptr;      // hit records: a whole image, or one tile of a larger one
    uint64_t* rec_vis = nullptr;
    long rec_cap = 0;                // camera samples the record buffer holds
};

// A linear model y = mean + basis * coef (shape morph, statistical albedo):
// FP32 mean [ld] and basis [K][ld] with rows padded to ld, the same basis as
// BF16 tensor-core operand tiles, and the adjoint's FP64 partials.
struct LinearModel {
    int rows = 0, K = 0, ld = 0, Kp = 0;
    float* mean = nullptr;
    float* basis = nullptr;
    uint16_t* tiles = nullptr;           // [ceil(rows / 128)][128][Kp] BF16, no-swizzle K-major core matrices
    double* part = nullptr;              // [linear_adj_chunks(rows)][FR_MAX_BATCH][K] (chunk-major)
};

}  // namespace

struct fr_ctx {
    fr_config cfg{};
    int max_batch = 1;
    int N = 0, T = 0, K = 0, NL = 0, E = 0, ld = 0;   // ld = shape.ld
    bool have_mesh = false, have_lights = false;
    bool poisoned = false;                     // a device wait gave up unsafely: refuse further work
    long rec_tile = 0;                         // record tile in camera samples (0: the slots' capacity)
    std::string err;
    // mesh and lights (shared by all slots)
    LinearModel shape;                         // rows 3N
    LinearModel albedo[2];                     // diffuse, specular; rows 3 M^2 (optional)
    bool have_albedo = false;
    // static SAH topology of the mesh (refitted per call unless FR_FLAG_LBVH)
    int *topo_child = nullptr, *topo_parent_int = nullptr, *topo_parent_leaf = nullptr, *topo_vals = nullptr;
    int* landmarks = nullptr;                  // landmark vertex indices [n_landmarks]
    int n_landmarks = 0;
    int4* faces = nullptr;
    float2* uv = nullptr;
    int* vf_off = nullptr;
    int* vf_idx = nullptr;
    int4* edges = nullptr;
    LightDev* lights = nullptr;
    float* stage = nullptr;                    // virtual light stage frame [N_L][12] (null: records only)
    std::vector<float> light_d_h, light_a_h;   // host copies of the lights' d and a
    int env_size = 0;                          // environment map side (0: no environment blocks)
    bool use_stage = false;                    // the last fr_set_lights gave a light-stage frame
    std::vector<Slot> slots;
    DevItem* d_items = nullptr;                // device item table [FR_MAX_BATCH]
    std::vector<DevItem> h_items;
    int* status = nullptr;
    unsigned long long* counters = nullptr;   // [kernel][rays, nodes, triangle tests]
    bool timing = false;
    cudaEvent_t ev[9] = {};
    // a fused step runs the geometry-only part of its reverse pass on `side`,
    // forked from and joined back into the caller's stream, beside the forward
    cudaStream_t side = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr, tail_ev = nullptr;
    std::vector<void*> owned;
};

static std::atomic<unsigned long long> g_launches{0};
void fr_count_launches(int n) { g_launches += (unsigned long long)n; }

namespace {

thread_local std::string g_err;

fr_status fail(fr_ctx* c, fr_status code, const std::string& msg) {
    if (c) c->err = msg; else g_err = msg;
    return code;
}

#define CK(ctx, x)                                                                     \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) return fail(ctx, FR_ECUDA, std::string(#x ": ") + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(x)                         \
    do {                               \
        fr_status s_ = (x);            \
        if (s_ != FR_OK) return s_;    \
    } while (0)

template <class T>
fr_status dalloc(fr_ctx* c, T** p, size_t count) {
    void* q = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
    if (e != cudaSuccess) return fail(c, FR_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    c->owned.push_back(q);
    *p = static_cast<T*>(q);
    return FR_OK;
}

void free_all(fr_ctx* c) {
    for (void* p : c->owned) cudaFree(p);
    c->owned.clear();
}

cudaStream_t S_(void* s) { return static_cast<cudaStream_t>(s); }

void destroy_side(fr_ctx* c) {
    if (c->fork_ev) cudaEventDestroy(c->fork_ev);
    if (c->join_ev) cudaEventDestroy(c->join_ev);
    if (c->tail_ev) cudaEventDestroy(c->tail_ev);
    if (c->side) cudaStreamDestroy(c->side);
    c->fork_ev = c->join_ev = c->tail_ev = nullptr;
    c->side = nullptr;
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// stage marks: 0 start, 1 after build, 2 after forward, 3 after loss,
// 4 after classify, 5 after adjoint, 6 after edge_primary, 7 after chain
void mark(fr_ctx* c, int k, cudaStream_t st) {
    if (c->timing) cudaEventRecord(c->ev[k], st);
}

fr_status check_params(fr_ctx* c, const fr_params* p) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    if (c->poisoned) return fail(c, FR_ECUDA, "context unusable after an unsafe device timeout");
    if (!c->have_mesh || !c->have_lights) return fail(c, FR_EINVAL, "mesh and lights must be set first");
    if (!p || !p->rot || !p->trans || !p->focal || !p->light_i || !p->diffuse || !p->specular || !p->roughness ||
        (c->K > 0 && !p->coef))
        return fail(c, FR_EINVAL, "null parameter pointer");
    if (c->env_size > 0 && !p->env) return fail(c, FR_EINVAL, "environment blocks need the env parameter");
    return FR_OK;
}

// Per-call description of one face before it becomes a DevItem.
struct ItemArgs {
    int W, H, spp, edge_spp;
    uint32_t flags, iteration, face;
    const fr_params* p;
    const fr_grads* g;          // may be null
    float* image;
    const float* adj;           // image-space adjoint (null: the slot's loss adjoint)
    int32_t* tri_rec;
    uint64_t* mask_rec;
    bool records;               // fused step: the adjoint may reuse the forward's hit records
};

DevItem make_item(const fr_ctx* c, int k, const ItemArgs& a) {
    const Slot& sl = c->slots[k];
    DevItem it;
    std::memset(&it, 0, sizeof(it));
    it.rec_from = -1;                       // the forward keeps no records unless set below
    DevScene& s = it.S;
    s.N = c->N; s.T = c->T; s.K = c->K; s.NL = c->NL; s.E = c->E;
    s.W = a.W; s.H = a.H; s.spp = a.spp; s.M = c->cfg.tex_size; s.edge_spp = a.edge_spp;
    s.flags = a.flags; s.seed = c->cfg.seed;
    s.v = sl.v_cam; s.vn = sl.vn; s.uv = c->uv; s.faces = c->faces; s.nodes = sl.nodes; s.tris = sl.tris;
    s.slot_of = sl.slot_of;
    s.lights = c->lights; s.status = c->status; s.counters = c->counters;
    const fr_params* p = a.p;
    it.P = DevParams{p->coef, p->rot, p->trans, p->focal, p->light_i, p->diffuse, p->specular, p->roughness,
                     p->light_d, p->light_a, p->light_p, c->env_size > 0 ? p->env : nullptr};
    s.env_size = c->env_size;
    if (c->use_stage && p->light_d && p->light_a && p->light_p) {   // lights built from (d, a, p)
        s.stage = c->stage;
        s.lights = sl.lights;
        it.lights_w = sl.lights;
    }
    it.G.d_v = sl.d_v;
    it.G.d_n = sl.d_n;
    it.G.tex = sl.tex;
    it.G.small = sl.small;
    if (a.g) {
        it.G.diffuse = a.g->diffuse;
        it.G.specular = a.g->specular;
        it.G.roughness = a.g->roughness;
        it.g_coef = a.g->coef;
        it.g_rot = a.g->rot;
        it.g_trans = a.g->trans;
        it.g_focal = a.g->focal;
        it.g_light = a.g->light_i;
        it.g_light_d = a.g->light_d;
        it.g_light_a = a.g->light_a;
        it.g_light_p = a.g->light_p;
        it.g_env = c->env_size > 0 ? a.g->env : nullptr;
    }
    it.EL.edges = c->edges;
    it.EL.prim_list = sl.lists;
    it.EL.prim_count = sl.counts;
    it.EL.light_list = sl.lists + c->E;
    it.EL.light_count = sl.counts + 1;
    it.B = sl.B;
    if (!(c->cfg.flags & FR_FLAG_LBVH)) {     // refit the static topology
        it.B.child = c->topo_child;
        it.B.parent_int = c->topo_parent_int;
        it.B.parent_leaf = c->topo_parent_leaf;
        it.B.vals = c->topo_vals;
        it.B.keys = nullptr;
    }
    it.nodes = sl.nodes;
    it.tris = sl.tris;
    it.slot_of = sl.slot_of;
    it.v_cam = sl.v_cam;
    it.vn = sl.vn;
    it.v_model = sl.v_model;
    it.d_vmodel = sl.d_vmodel;
    it.n_face = sl.n_face;
    it.dm = sl.dm;
    it.pose_part = sl.pose_part;
    it.sil_flags = sl.sil_flags;
    it.image = a.image;
    it.adj = a.adj ? a.adj : sl.adj_image;
    it.tri_rec = a.tri_rec;
    it.mask_rec = a.mask_rec;
    if ((long)a.W * a.H * a.edge_spp <= sl.edge_cap) it.edge_perm = sl.edge_perm;
    it.spec_list = sl.spec_list;
    it.spec_box = sl.spec_box;
    it.spec_hist = sl.spec_hist;
    it.spec_count = sl.spec_count;
    it.spec_flag = sl.spec_flag;
    // hit records: a fused step's forward writes them when the whole image fits
    // the buffer; otherwise the adjoint recomputes them tile by tile into it.
    // FR_FLAG_RECOMPUTE keeps the adjoint re-tracing every sample instead.
    if (sl.rec_tri && !(a.flags & FR_FLAG_RECOMPUTE)) {
        it.rec_tri = sl.rec_tri;
        it.rec_vis = sl.rec_vis;
        it.rec_cap = c->rec_tile > 0 ? std::min(c->rec_tile, sl.rec_cap) : sl.rec_cap;
        const long total = (long)a.W * a.H * a.spp;
        it.rec_full = a.records && total <= it.rec_cap ? 1 : 0;
        // a larger image: the forward keeps the records of its last tile, which
        // the adjoint (walking the tiles from the last) reads before it
        // recomputes the others into the same buffer
        it.rec_from = a.records ? (total - 1) / it.rec_cap * it.rec_cap : -1;
    }
    it.iteration = a.iteration;
    it.face = a.face;
    return it;
}

// Blocks of a launch over camera samples [q0, q0 + cap) of each item, for the
// items `take` accepts (the others get no blocks).
template <class F>
BlockMap tile_map(const fr_ctx* c, int n, long q0, long cap, F take) {
    BlockMap m;
    m.n = n;
    int b = 0;
    for (int k = 0; k < n; ++k) {
        const DevScene& s = c->h_items[k].S;
        m.block0[k] = b;
        const long left = (long)s.W * s.H * s.spp - q0;
        if (take(c->h_items[k]) && left > 0) b += (int)((std::min(left, cap) + 127) / 128);
    }
    m.block0[n] = b;
    return m;
}

BlockMap map_of(const fr_ctx* c, int n, bool edges) {
    BlockMap m;
    m.n = n;
    int b = 0;
    for (int k = 0; k < n; ++k) {
        const DevScene& s = c->h_items[k].S;
        m.block0[k] = b;
        // primary-edge samples take two threads each (one per side of the edge)
        long work = (long)s.W * s.H * (edges ? ((s.flags & FR_FLAG_NO_PRIMARY_EDGE) ? 0 : 2 * s.edge_spp) : s.spp);
        b += (int)((work + 127) / 128);
    }
    m.block0[n] = b;
    return m;
}

// One block per scanline of the specular-boundary term for each item that has
// the term: (W + H) * max(edge_spp, 1) rows and columns.
BlockMap spec_map(const fr_ctx* c, int n) {
    BlockMap m;
    m.n = n;
    int b = 0;
    for (int k = 0; k < n; ++k) {
        const DevScene& s = c->h_items[k].S;
        m.block0[k] = b;
        if (!(s.flags & (FR_FLAG_NO_SPECULAR_EDGE | FR_FLAG_FLAT))) b += (s.W + s.H) * std::max(s.edge_spp, 1);
    }
    m.block0[n] = b;
    return m;
}

// Upload the item table for items [0, n) (one small kernel on the stream).
fr_status upload(fr_ctx* c, int n, cudaStream_t st) {
    launch_set_items(c->h_items.data(), n, c->d_items, st);
    CK(c, cudaGetLastError());
    return FR_OK;
}

// out_b = mean + basis * coef_b for the n faces of `t`, on the tensor cores
// when the context has FR_FLAG_MORPH_BF16, else in FP32
void linear_forward(fr_ctx* c, const LinearModel& m, const LinearTable& t, cudaStream_t st) {
    if ((c->cfg.flags & FR_FLAG_MORPH_BF16) && m.K > 0) {
        const TcModel tm{m.tiles, m.Kp, m.K, m.mean, m.rows, t};
        launch_linear_tc(&tm, 1, c->status, st);
    } else {
        launch_linear(m.mean, m.basis, m.ld, m.rows, m.K, t, st);
    }
}

void morph(fr_ctx* c, int n, cudaStream_t st) {
    LinearTable t;
    t.n = n;
    for (int k = 0; k < n; ++k) {
        t.coef[k] = c->h_items[k].P.coef;
        t.out[k] = c->slots[k].v_model;
    }
    linear_forward(c, c->shape, t, st);
}

void morph_adjoint(fr_ctx* c, int n, cudaStream_t st) {
    LinearAdjTable t;
    t.n = n;
    for (int k = 0; k < n; ++k) {
        t.g[k] = c->slots[k].d_vmodel;
        t.g_coef[k] = c->h_items[k].g_coef;
    }
    const LinearAdjModel md{c->shape.basis, c->shape.ld, c->shape.rows, c->shape.K, c->shape.part, t};
    launch_linear_adjoint(&md, 1, st);
}

// Upload a linear model (host mean [rows], basis [K][rows]) and build its
// BF16 operand tiles: tile t holds rows 128t..128t+127 of the [rows x Kp]
// basis in the no-swizzle K-major core-matrix layout (8 rows x 8 values per
// 128-byte core matrix).
fr_status upload_model(fr_ctx* c, LinearModel& m, int rows, int K, const float* mean, const float* basis) {
    m.rows = rows;
    m.K = K;
    m.ld = ((rows + 31) / 32) * 32;
    TRY(dalloc(c, &m.mean, m.ld));
    TRY(dalloc(c, &m.basis, (size_t)std::max(K, 1) * m.ld));
    std::vector<float> pad((size_t)m.ld, 0.0f);
    std::copy(mean, mean + (size_t)rows, pad.begin());
    CK(c, cudaMemcpy(m.mean, pad.data(), sizeof(float) * m.ld, cudaMemcpyHostToDevice));
    for (int k = 0; k < K; ++k) {
        std::fill(pad.begin(), pad.end(), 0.0f);
        std::copy(basis + (size_t)k * rows, basis + (size_t)(k + 1) * rows, pad.begin());
        CK(c, cudaMemcpy(m.basis + (size_t)k * m.ld, pad.data(), sizeof(float) * m.ld, cudaMemcpyHostToDevice));
    }
    if (K == 0) return FR_OK;
    TRY(dalloc(c, &m.part, (size_t)FR_MAX_BATCH * K * linear_adj_chunks(rows)));
    m.Kp = ((K + 15) / 16) * 16;
    const int n_tiles = (rows + 127) / 128;
    std::vector<uint16_t> bt((size_t)n_tiles * 128 * m.Kp, 0);
    auto bf16 = [](float f) {
        uint32_t u;
        std::memcpy(&u, &f, 4);
        u += 0x7FFFu + ((u >> 16) & 1u);
        return (uint16_t)(u >> 16);
    };
    for (int t = 0; t < n_tiles; ++t)
        for (int rr = 0; rr < 128; ++rr) {
            const int i = t * 128 + rr;
            if (i >= rows) break;
            const int g = rr >> 3, r = rr & 7;
            for (int k = 0; k < K; ++k) {
                const int cc = k >> 3, kk = k & 7;
                const size_t off = (size_t)t * 128 * m.Kp + ((size_t)(g * (m.Kp / 8) + cc) * 128 + r * 16 + kk * 2) / 2;
                bt[off] = bf16(basis[(size_t)k * rows + i]);
            }
        }
    TRY(dalloc(c, &m.tiles, bt.size()));
    CK(c, cudaMemcpy(m.tiles, bt.data(), sizeof(uint16_t) * bt.size(), cudaMemcpyHostToDevice));
    return FR_OK;
}

// stage lights -> morph -> pose -> face normals + Morton keys -> vertex normals -> BVH
void build_geometry(fr_ctx* c, int n, cudaStream_t st) {
    bool any_stage = false;
    for (int k = 0; k < n; ++k) any_stage |= c->h_items[k].S.stage != nullptr;
    if (any_stage) launch_stage_lights(c->d_items, n, c->NL, st);
    morph(c, n, st);
    launch_pose(c->d_items, n, c->N, st);
    launch_faces(c->d_items, n, c->faces, c->T, st);
    launch_vertex_normals(c->d_items, n, c->vf_off, c->vf_idx, c->N, st);
    launch_lbvh(c->d_items, n, c->faces, c->T, c->status, (c->cfg.flags & FR_FLAG_LBVH) != 0, st);
}

fr_status forward_pass(fr_ctx* c, int n, cudaStream_t st) {
    for (int k = 0; k < n; ++k) {
        const DevItem& it = c->h_items[k];
        // a pixel's samples span two blocks only at spp = 256: their two partial
        // sums are added onto zero (exact in either order)
        if (it.S.spp > 128) CK(c, cudaMemsetAsync(it.image, 0, sizeof(float) * 3 * (size_t)it.S.W * it.S.H, st));
    }
    launch_forward(c->d_items, map_of(c, n, false), c->env_size > 0, 0, false, st);
    return FR_OK;
}

// The part of the reverse pass for items [0, n) that needs only their built
// geometry (not the forward's image or records): the accumulators zeroed, the
// silhouette classification, the order of the primary-edge samples and the
// specular-boundary candidates.
void adjoint_prep(fr_ctx* c, int n, cudaStream_t st) {
    launch_zero_accumulators(c->d_items, n, c->N, c->cfg.tex_size, st);
    bool need_edges = false;
    long max_edge = 0;
    for (int k = 0; k < n; ++k) {
        const DevScene& s = c->h_items[k].S;
        need_edges |= !(s.flags & FR_FLAG_NO_PRIMARY_EDGE) || !(s.flags & FR_FLAG_NO_SHADOW_EDGE);
        if (!(s.flags & FR_FLAG_NO_PRIMARY_EDGE)) max_edge = std::max(max_edge, (long)s.W * s.H * s.edge_spp);
    }
    if (need_edges) launch_classify(c->d_items, n, c->E, c->NL, c->T, st);
    launch_edge_order(c->d_items, n, max_edge, st);
    launch_spec_candidates(c->d_items, n, c->T, spec_map(c, n), st);
}

// The rest of the reverse pass, after adjoint_prep and the loss.  The boundary
// terms (primary edges, the specular lobe's cutoff) and the interior term
// (with the shadow-boundary term) only add into the fixed-point accumulators
// with integer atomics, whose sums do not depend on their order, and read
// nothing the others write: the boundary terms run on the side stream while
// the interior term runs on `st`, and `st` waits for them before the chain.
fr_status adjoint_main(fr_ctx* c, int n, cudaStream_t st) {
    mark(c, 4, st);
    CK(c, cudaEventRecord(c->fork_ev, st));
    CK(c, cudaStreamWaitEvent(c->side, c->fork_ev, 0));
    launch_edge_primary(c->d_items, map_of(c, n, true), c->env_size > 0, c->side);
    launch_edge_specular(c->d_items, spec_map(c, n), c->env_size > 0, c->side);
    CK(c, cudaEventRecord(c->join_ev, c->side));
    bool all_full = true, any_retrace = false, any_stage = false;
    long cap = 0, n_tiles = 1;
    for (int k = 0; k < n; ++k) {
        const DevItem& it = c->h_items[k];
        all_full &= it.rec_full != 0;
        any_retrace |= it.rec_tri == nullptr;
        any_stage |= it.S.stage != nullptr;
        if (it.rec_tri) cap = it.rec_cap;
    }
    const bool env = c->env_size > 0;
    if (all_full || any_retrace) {
        // records of the whole image from this step's forward, or (some item
        // asked for it) re-tracing in the adjoint itself
        launch_adjoint(c->d_items, map_of(c, n, false), c->NL, all_full, any_stage, env, 0, st);
    } else {
        // recomputed records: per tile of `cap` camera samples, from the last
        // tile to the first, a records-only forward pass over the items whose
        // forward did not keep that tile's records (it kept each image's last
        // tile, the first this order meets), then the recorded adjoint over the
        // same tile of every item
        for (int k = 0; k < n; ++k) {
            const DevScene& s = c->h_items[k].S;
            n_tiles = std::max(n_tiles, ((long)s.W * s.H * s.spp + cap - 1) / cap);
        }
        for (long t = n_tiles - 1; t >= 0; --t) {
            const long q0 = t * cap;
            launch_forward(c->d_items,
                           tile_map(c, n, q0, cap, [q0](const DevItem& it) { return !it.rec_full && it.rec_from != q0; }),
                           env, q0, true, st);
            launch_adjoint(c->d_items, tile_map(c, n, q0, cap, [](const DevItem&) { return true; }), c->NL, true,
                           any_stage, env, q0, st);
        }
    }
    mark(c, 5, st);
    // the texture gradients are complete once the interior term is (the
    // boundary terms add none): they are flushed on the side stream, after the
    // boundary terms there, while `st` runs the vertex chain
    CK(c, cudaEventRecord(c->fork_ev, st));
    CK(c, cudaStreamWaitEvent(c->side, c->fork_ev, 0));
    launch_tex_flush(c->d_items, n, c->cfg.tex_size, c->side);
    CK(c, cudaEventRecord(c->tail_ev, c->side));
    CK(c, cudaStreamWaitEvent(st, c->join_ev, 0));
    mark(c, 6, st);
    launch_normals_adjoint(c->d_items, n, c->faces, c->vf_off, c->vf_idx, c->N, st);
    launch_pose_adjoint(c->d_items, n, c->N, st);
    launch_pose_finish(c->d_items, n, c->NL, c->N, st);
    morph_adjoint(c, n, st);
    CK(c, cudaStreamWaitEvent(st, c->tail_ev, 0));
    mark(c, 7, st);
    return FR_OK;
}

// reverse pass for items [0, n) whose geometry is built (adjoint_prep on `st`)
fr_status adjoint_pass(fr_ctx* c, int n, cudaStream_t st) {
    adjoint_prep(c, n, st);
    return adjoint_main(c, n, st);
}

// Fork adjoint_prep onto the context's side stream after the work already on
// `st` (the built geometry); join_prep makes `st` wait for it.  Between the two
// the caller's stream runs the forward and the loss, which share no buffer
// with adjoint_prep.  Under stream capture the fork and join are part of the
// captured graph.
fr_status fork_prep(fr_ctx* c, int n, cudaStream_t st) {
    CK(c, cudaEventRecord(c->fork_ev, st));
    CK(c, cudaStreamWaitEvent(c->side, c->fork_ev, 0));
    adjoint_prep(c, n, c->side);
    CK(c, cudaEventRecord(c->join_ev, c->side));
    return FR_OK;
}

fr_status join_prep(fr_ctx* c, cudaStream_t st) {
    CK(c, cudaStreamWaitEvent(st, c->join_ev, 0));
    return FR_OK;
}

LossTable loss_table(fr_ctx* c, int n, const float* const* targets, double* const* losses, bool adjoint) {
    LossTable t;
    t.n = n;
    t.max_px3 = 0;
    for (int k = 0; k < n; ++k) {
        const DevItem& it = c->h_items[k];
        const Slot& sl = c->slots[k];
        t.it[k] = LossItem{it.S.H, it.S.W, it.image, targets[k], losses[k], sl.sign, sl.loss_part, nullptr,
                           adjoint ? sl.adj_image : nullptr};
        t.max_px3 = std::max(t.max_px3, it.S.H * it.S.W * 3);
    }
    return t;
}

fr_status alloc_slot(fr_ctx* c, Slot& sl) {
    const int N = c->N, T = c->T;
    TRY(dalloc(c, &sl.v_model, c->ld));
    TRY(dalloc(c, &sl.d_vmodel, c->ld));
    TRY(dalloc(c, &sl.v_cam, N));
    TRY(dalloc(c, &sl.vn, N));
    TRY(dalloc(c, &sl.n_face, T));
    const int n_tiles = (T + 255) / 256;
    TRY(dalloc(c, &sl.B.keys, T));
    TRY(dalloc(c, &sl.B.keys_alt, T));
    TRY(dalloc(c, &sl.B.vals, T));
    TRY(dalloc(c, &sl.B.vals_alt, T));
    // radix histogram [256][n_tiles]; the silhouette compaction reuses it for
    // [1 + 64 lists][E / 1024 chunks] counts
    TRY(dalloc(c, &sl.B.hist, std::max(256 * (size_t)n_tiles, (size_t)(1 + FR_MAX_LIGHTS) * ((c->E + 1023) / 1024))));
    TRY(dalloc(c, &sl.B.hist_base, 256));
    TRY(dalloc(c, &sl.B.child, 2 * (size_t)std::max(T - 1, 1)));
    TRY(dalloc(c, &sl.B.parent_int, std::max(T - 1, 1)));
    TRY(dalloc(c, &sl.B.parent_leaf, T));
    TRY(dalloc(c, &sl.B.flag, std::max(T - 1, 1)));
    TRY(dalloc(c, &sl.B.box_int, 2 * (size_t)std::max(T - 1, 1)));
    TRY(dalloc(c, &sl.B.box_leaf, 2 * (size_t)T));
    TRY(dalloc(c, &sl.B.aabb, 6));
    TRY(dalloc(c, &sl.nodes, std::max(T - 1, 1)));
    TRY(dalloc(c, &sl.tris, 3 * (size_t)T));
    TRY(dalloc(c, &sl.slot_of, T));
    // [1 + 64 lists][E] edge flags, then [64 lights][T] per-face facing classes
    TRY(dalloc(c, &sl.sil_flags, (size_t)(1 + FR_MAX_LIGHTS) * c->E + (size_t)FR_MAX_LIGHTS * T));
    TRY(dalloc(c, &sl.lists, (size_t)(1 + FR_MAX_LIGHTS) * c->E));
    TRY(dalloc(c, &sl.counts, 1 + FR_MAX_LIGHTS));
    TRY(dalloc(c, &sl.d_v, 3 * (size_t)N));
    TRY(dalloc(c, &sl.d_n, 3 * (size_t)N));
    TRY(dalloc(c, &sl.tex, 7 * (size_t)c->cfg.tex_size * c->cfg.tex_size));
    TRY(dalloc(c, &sl.dm, 3 * (size_t)N));
    TRY(dalloc(c, &sl.small, FR_SMALL));
    TRY(dalloc(c, &sl.lights, FR_MAX_LIGHTS));
    TRY(dalloc(c, &sl.pose_part, 12 * (size_t)((N + 255) / 256)));
    // processing order of the primary-edge samples (the context's edge_spp, at least 1)
    sl.edge_cap = (long)c->cfg.width * c->cfg.height * std::max(c->cfg.edge_spp, 1);
    TRY(dalloc(c, &sl.edge_perm, (size_t)sl.edge_cap));
    TRY(dalloc(c, &sl.spec_list, (size_t)T));
    TRY(dalloc(c, &sl.spec_box, (size_t)T));
    TRY(dalloc(c, &sl.spec_hist, (size_t)(T + 1023) / 1024 + 1));
    TRY(dalloc(c, &sl.spec_count, 1));
    TRY(dalloc(c, &sl.spec_flag, (size_t)T));
    // hit records (triangle + two visibility words per camera sample): the whole
    // image when it fits FR_RECORDS_BUDGET, else equal tiles of it that do, in
    // whole pixels and whole 128-thread blocks (a multiple of max(128, spp))
    const long samples = (long)c->cfg.width * c->cfg.height * c->cfg.spp;
    const long per = (long)(sizeof(int32_t) + 2 * sizeof(uint64_t));
    const long unit = std::max(128, c->cfg.spp);
    const long n_rec = (samples * per + (long)FR_RECORDS_BUDGET - 1) / (long)FR_RECORDS_BUDGET;
    sl.rec_cap = ((samples + n_rec - 1) / n_rec + unit - 1) / unit * unit;
    TRY(dalloc(c, &sl.rec_tri, (size_t)sl.rec_cap));
    TRY(dalloc(c, &sl.rec_vis, 2 * (size_t)sl.rec_cap));
    return FR_OK;
}

fr_status check_image_args(fr_ctx* c, int W, int H, int spp, int edge_spp) {
    if (W < 1 || H < 1 || (long)W * H > (long)c->cfg.width * c->cfg.height)
        return fail(c, FR_EINVAL, "item image larger than the context's width x height");
    if (!is_pow2(spp) || spp > FR_MAX_SPP) return fail(c, FR_EINVAL, "spp must be a power of two <= 256");
    if (edge_spp < 0 || edge_spp > 64) return fail(c, FR_EINVAL, "edge_spp out of range");
    if ((long)(W + H) * std::max(edge_spp, 1) > 65535)
        return fail(c, FR_EINVAL, "more than 65535 scanlines for the specular-boundary term");
    if ((long)W * H * spp > (1L << 31) - 1024) return fail(c, FR_EINVAL, "too many samples per item");
    return FR_OK;
}

ItemArgs single(fr_ctx* c, const fr_params* p, const fr_grads* g, float* image, const float* adj, uint32_t iteration,
                uint32_t face) {
    ItemArgs a;
    a.W = c->cfg.width; a.H = c->cfg.height; a.spp = c->cfg.spp; a.edge_spp = c->cfg.edge_spp;
    a.flags = c->cfg.flags; a.iteration = iteration; a.face = face;
    a.p = p; a.g = g; a.image = image; a.adj = adj; a.tri_rec = nullptr; a.mask_rec = nullptr;
    a.records = false;
    return a;
}

}  // namespace

void ctx_info(const fr_ctx* c, CtxInfo& o) {
    o = CtxInfo{};
    if (!c) return;
    o.width = c->cfg.width;
    o.height = c->cfg.height;
    o.spp = c->cfg.spp;
    o.tex = c->cfg.tex_size;
    o.K = c->K;
    o.NL = c->NL;
    o.max_batch = c->max_batch;
    o.n_landmarks = c->n_landmarks;
    o.flags = c->cfg.flags;
    o.ready = c->have_mesh && c->have_lights;
    o.have_albedo = c->have_albedo;
    o.k_diffuse = c->have_albedo ? c->albedo[0].K : 0;
    o.k_specular = c->have_albedo ? c->albedo[1].K : 0;
    o.have_stage = c->use_stage;
    o.env_size = c->env_size;
    o.light_da = c->light_d_h;
    o.light_da.insert(o.light_da.end(), c->light_a_h.begin(), c->light_a_h.end());
}

extern "C" {

fr_status fr_create(fr_ctx** out, const fr_config* cfg) {
    if (!out || !cfg) return fail(nullptr, FR_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->width < 1 || cfg->width > 8192 || cfg->height < 1 || cfg->height > 8192)
        return fail(nullptr, FR_EINVAL, "image size out of range");
    if (!is_pow2(cfg->spp) || cfg->spp > FR_MAX_SPP)
        return fail(nullptr, FR_EINVAL, "spp must be a power of two <= 256");
    if (cfg->tex_size < 1 || cfg->tex_size > 8192) return fail(nullptr, FR_EINVAL, "tex_size out of range");
    if (cfg->edge_spp < 0 || cfg->edge_spp > 64) return fail(nullptr, FR_EINVAL, "edge_spp out of range");
    if ((long)cfg->width * cfg->height * cfg->spp > (1L << 31) - 1024)
        return fail(nullptr, FR_EINVAL, "too many samples per call");
    if (cfg->max_batch < 0 || cfg->max_batch > FR_MAX_BATCH) return fail(nullptr, FR_EINVAL, "max_batch out of range");
    fr_ctx* c = new fr_ctx();
    c->cfg = *cfg;
    c->max_batch = std::max(1, cfg->max_batch);
    c->slots.resize(c->max_batch);
    c->h_items.resize(FR_MAX_BATCH);
    const size_t px = (size_t)cfg->width * cfg->height * 3;
    bool ok = dalloc(c, &c->status, 1) == FR_OK && cudaMemset(c->status, 0, sizeof(int)) == cudaSuccess &&
              dalloc(c, &c->counters, 9) == FR_OK &&
              cudaMemset(c->counters, 0, 9 * sizeof(unsigned long long)) == cudaSuccess &&
              dalloc(c, &c->d_items, FR_MAX_BATCH) == FR_OK;
    for (int k = 0; ok && k < c->max_batch; ++k)
        ok = dalloc(c, &c->slots[k].sign, px) == FR_OK && dalloc(c, &c->slots[k].adj_image, px) == FR_OK &&
             dalloc(c, &c->slots[k].loss_part, FR_LOSS_PARTS) == FR_OK;
    if (!ok) {
        g_err = c->err;
        free_all(c);
        delete c;
        return FR_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->join_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->tail_ev, cudaEventDisableTiming) != cudaSuccess) {
        const fr_status st = fail(nullptr, FR_ECUDA, "side stream or events could not be created");
        destroy_side(c);
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return FR_OK;
}

fr_status fr_set_mesh(fr_ctx* c, const fr_mesh* m) {
    if (!c || !m || !m->mean || !m->faces || !m->uv || (m->n_basis > 0 && !m->basis))
        return fail(c, FR_EINVAL, "null argument");
    if (c->have_mesh) return fail(c, FR_EINVAL, "mesh already set on this context");
    const int N = m->n_vertices, T = m->n_triangles, K = m->n_basis;
    if (N < 3 || T < 1 || K < 0 || K > FR_MAX_BASIS) return fail(c, FR_EINVAL, "mesh sizes out of range");
    // topology: vertex -> faces CSR in face order; undirected edges sorted by (a, b)
    std::vector<int> deg(N + 1, 0);
    for (int f = 0; f < T; ++f)
        for (int k = 0; k < 3; ++k) {
            const int v = m->faces[3 * f + k];
            if (v < 0 || v >= N) return fail(c, FR_EINVAL, "face index out of range");
            deg[v + 1]++;
        }
    for (int i = 0; i < N; ++i) deg[i + 1] += deg[i];
    std::vector<int> vf(3 * (size_t)T), fill(deg.begin(), deg.end() - 1);
    for (int f = 0; f < T; ++f)
        for (int k = 0; k < 3; ++k) vf[fill[m->faces[3 * f + k]]++] = f;
    struct HE { int a, b, f; };
    std::vector<HE> he;
    he.reserve(3 * (size_t)T);
    for (int f = 0; f < T; ++f)
        for (int k = 0; k < 3; ++k) {
            const int u = m->faces[3 * f + k], w = m->faces[3 * f + (k + 1) % 3];
            if (u == w) return fail(c, FR_EINVAL, "degenerate face");
            he.push_back({std::min(u, w), std::max(u, w), f});
        }
    std::sort(he.begin(), he.end(), [](const HE& x, const HE& y) {
        return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.f < y.f);
    });
    std::vector<int4> edges;
    for (size_t i = 0; i < he.size();) {
        size_t j = i;
        while (j < he.size() && he[j].a == he[i].a && he[j].b == he[i].b) ++j;
        if (j - i > 2) return fail(c, FR_EINVAL, "non-manifold edge");
        edges.push_back(make_int4(he[i].a, he[i].b, he[i].f, j - i == 2 ? he[i + 1].f : -1));
        i = j;
    }
    c->N = N; c->T = T; c->K = K; c->E = (int)edges.size();
    TRY(upload_model(c, c->shape, 3 * N, K, m->mean, m->basis));
    c->ld = c->shape.ld;
    {
        BvhTopology topo;
        build_bvh_topology(m->mean, m->faces, T, topo);
        TRY(dalloc(c, &c->topo_child, topo.child.size()));
        TRY(dalloc(c, &c->topo_parent_int, topo.parent_int.size()));
        TRY(dalloc(c, &c->topo_parent_leaf, topo.parent_leaf.size()));
        TRY(dalloc(c, &c->topo_vals, topo.vals.size()));
        CK(c, cudaMemcpy(c->topo_child, topo.child.data(), sizeof(int) * topo.child.size(), cudaMemcpyHostToDevice));
        CK(c, cudaMemcpy(c->topo_parent_int, topo.parent_int.data(), sizeof(int) * topo.parent_int.size(),
                         cudaMemcpyHostToDevice));
        CK(c, cudaMemcpy(c->topo_parent_leaf, topo.parent_leaf.data(), sizeof(int) * topo.parent_leaf.size(),
                         cudaMemcpyHostToDevice));
        CK(c, cudaMemcpy(c->topo_vals, topo.vals.data(), sizeof(int) * topo.vals.size(), cudaMemcpyHostToDevice));
    }
    TRY(dalloc(c, &c->faces, T));
    TRY(dalloc(c, &c->uv, N));
    TRY(dalloc(c, &c->vf_off, N + 1));
    TRY(dalloc(c, &c->vf_idx, 3 * (size_t)T));
    TRY(dalloc(c, &c->edges, c->E));
    std::vector<int4> f4(T);
    for (int f = 0; f < T; ++f) f4[f] = make_int4(m->faces[3 * f], m->faces[3 * f + 1], m->faces[3 * f + 2], 0);
    CK(c, cudaMemcpy(c->faces, f4.data(), sizeof(int4) * T, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->uv, m->uv, sizeof(float2) * N, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->vf_off, deg.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->vf_idx, vf.data(), sizeof(int) * 3 * (size_t)T, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->edges, edges.data(), sizeof(int4) * c->E, cudaMemcpyHostToDevice));
    for (Slot& sl : c->slots) TRY(alloc_slot(c, sl));
    c->have_mesh = true;
    return FR_OK;
}

fr_status fr_set_albedo(fr_ctx* c, const fr_albedo_model* am) {
    if (!c || !am) return fail(c, FR_EINVAL, "null argument");
    if (c->have_albedo) return fail(c, FR_EINVAL, "albedo model already set");
    const int rows = 3 * c->cfg.tex_size * c->cfg.tex_size;
    const int ks[2] = {am->k_diffuse, am->k_specular};
    const float* means[2] = {am->mean_diffuse, am->mean_specular};
    const float* bases[2] = {am->basis_diffuse, am->basis_specular};
    for (int q = 0; q < 2; ++q) {
        if (ks[q] < 0 || ks[q] > FR_MAX_BASIS) return fail(c, FR_EINVAL, "albedo basis size out of range");
        if (!means[q] || (ks[q] > 0 && !bases[q])) return fail(c, FR_EINVAL, "null albedo mean or basis");
    }
    for (int q = 0; q < 2; ++q) TRY(upload_model(c, c->albedo[q], rows, ks[q], means[q], bases[q]));
    c->have_albedo = true;
    return FR_OK;
}

fr_status fr_set_landmarks(fr_ctx* c, int32_t n, const int32_t* idx) {
    if (!c || !idx) return fail(c, FR_EINVAL, "null argument");
    if (!c->have_mesh) return fail(c, FR_EINVAL, "mesh must be set first");
    if (n < 1 || n > 256) return fail(c, FR_EINVAL, "1 <= n_landmarks <= 256");
    for (int l = 0; l < n; ++l)
        if (idx[l] < 0 || idx[l] >= c->N) return fail(c, FR_EINVAL, "landmark vertex out of range");
    if (!c->landmarks) TRY(dalloc(c, &c->landmarks, 256));
    CK(c, cudaMemcpy(c->landmarks, idx, sizeof(int) * n, cudaMemcpyHostToDevice));
    c->n_landmarks = n;
    return FR_OK;
}

fr_status fr_landmark_loss(fr_ctx* c, const fr_params* p, int32_t width, int32_t height, const float* z,
                           float weight, double* loss, fr_grads* g, float* projected, void* stream) {
    if (!c || !p || !z || !loss) return fail(c, FR_EINVAL, "null argument");
    if (c->n_landmarks == 0) return fail(c, FR_EINVAL, "landmarks not set");
    if (c->poisoned) return fail(c, FR_ECUDA, "context unusable after an unsafe device timeout");
    if (!p->rot || !p->trans || !p->focal || (c->K > 0 && !p->coef)) return fail(c, FR_EINVAL, "null parameter");
    if (width < 1 || height < 1) return fail(c, FR_EINVAL, "bad image size");
    LandmarkArgs a;
    a.mean = c->shape.mean;
    a.basis = c->shape.basis;
    a.ld = c->shape.ld;
    a.K = c->K;
    a.idx = c->landmarks;
    a.L = c->n_landmarks;
    a.W = width;
    a.H = height;
    a.coef = p->coef; a.rot = p->rot; a.trans = p->trans; a.focal = p->focal;
    a.z = z;
    a.weight = weight;
    a.loss = loss;
    a.proj = projected;
    a.g_coef = g ? g->coef : nullptr;
    a.g_rot = g ? g->rot : nullptr;
    a.g_trans = g ? g->trans : nullptr;
    a.g_focal = g ? g->focal : nullptr;
    launch_landmarks(a, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

fr_status fr_albedo_morph(fr_ctx* c, int32_t n, const float* const* beta, const float* const* gamma,
                          float* const* diffuse, float* const* specular, void* stream) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    if (c->poisoned) return fail(c, FR_ECUDA, "context unusable after an unsafe device timeout");
    if (!c->have_albedo) return fail(c, FR_EINVAL, "albedo model not set");
    if (n < 1 || n > c->max_batch) return fail(c, FR_EINVAL, "1 <= n <= max_batch faces required");
    const float* const* coefs[2] = {beta, gamma};
    float* const* outs[2] = {diffuse, specular};
    LinearTable tab[2];
    for (int q = 0; q < 2; ++q) {
        if (!outs[q]) continue;
        const LinearModel& m = c->albedo[q];
        if (m.K > 0 && !coefs[q]) return fail(c, FR_EINVAL, "null coefficient array");
        LinearTable& t = tab[q];
        t.n = n;
        for (int k = 0; k < n; ++k) {
            if (!outs[q][k] || !aligned16(outs[q][k])) return fail(c, FR_EINVAL, "null or misaligned texture");
            if (m.K > 0 && !coefs[q][k]) return fail(c, FR_EINVAL, "null coefficients");
            t.coef[k] = m.K > 0 ? coefs[q][k] : nullptr;
            t.out[k] = outs[q][k];
        }
    }
    // on the tensor cores both albedos go in one launch; the FP32 path and
    // models without columns (mean only) go one model at a time
    TcModel tm[2];
    int n_tc = 0;
    for (int q = 0; q < 2; ++q) {
        if (!outs[q]) continue;
        const LinearModel& m = c->albedo[q];
        if ((c->cfg.flags & FR_FLAG_MORPH_BF16) && m.K > 0)
            tm[n_tc++] = TcModel{m.tiles, m.Kp, m.K, m.mean, m.rows, tab[q]};
        else
            linear_forward(c, m, tab[q], S_(stream));
    }
    if (n_tc > 0) launch_linear_tc(tm, n_tc, c->status, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_albedo_adjoint(fr_ctx* c, int32_t n, const float* const* g_diffuse, const float* const* g_specular,
                            float* const* g_beta, float* const* g_gamma, void* stream) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    if (c->poisoned) return fail(c, FR_ECUDA, "context unusable after an unsafe device timeout");
    if (!c->have_albedo) return fail(c, FR_EINVAL, "albedo model not set");
    if (n < 1 || n > c->max_batch) return fail(c, FR_EINVAL, "1 <= n <= max_batch faces required");
    const float* const* gs[2] = {g_diffuse, g_specular};
    float* const* outs[2] = {g_beta, g_gamma};
    LinearAdjModel md[2];
    int n_md = 0;
    for (int q = 0; q < 2; ++q) {                      // both albedos in one launch
        const LinearModel& m = c->albedo[q];
        if (!outs[q] || m.K == 0) continue;
        if (!gs[q]) return fail(c, FR_EINVAL, "null texture-gradient array");
        LinearAdjTable t;
        t.n = n;
        for (int k = 0; k < n; ++k) {
            if (!gs[q][k] || !aligned16(gs[q][k])) return fail(c, FR_EINVAL, "null or misaligned texture gradient");
            t.g[k] = gs[q][k];
            t.g_coef[k] = outs[q][k];
        }
        md[n_md++] = LinearAdjModel{m.basis, m.ld, m.rows, m.K, m.part, t};
    }
    launch_linear_adjoint(md, n_md, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_set_lights(fr_ctx* c, const fr_light_stage* ls) {
    if (!c || !ls || !ls->records || !ls->d || !ls->a) return fail(c, FR_EINVAL, "null argument");
    if (ls->n_lights < 1 || ls->n_lights > FR_MAX_LIGHTS) return fail(c, FR_EINVAL, "1 <= n_lights <= 128");
    std::vector<LightDev> L(ls->n_lights);
    bool any_env = false;
    for (int j = 0; j < ls->n_lights; ++j) {
        const float* r = ls->records + 11 * j;
        LightDev& d = L[j];
        d.type = (int)r[0];
        if (d.type < 0 || d.type > 3) return fail(c, FR_EINVAL, "unknown emitter type");
        if (d.type == FR_LIGHT_ENV) {             // environment block: integer texel ranges
            const int me = ls->env_size;
            if (me < 1 || me > FR_MAX_ENV) return fail(c, FR_EINVAL, "env_size must be 1..64 with environment blocks");
            const int i0 = (int)r[1], i1 = (int)r[2], j0 = (int)r[3], j1 = (int)r[4];
            if ((float)i0 != r[1] || (float)i1 != r[2] || (float)j0 != r[3] || (float)j1 != r[4] || i0 < 0 ||
                i1 <= i0 || i1 > me || j0 < 0 || j1 <= j0 || j1 > me)
                return fail(c, FR_EINVAL, "environment block outside the map");
            d.c = f3((float)i0, (float)i1, (float)j0);
            d.e1 = f3((float)j1, 0.0f, 0.0f);
            d.e2 = d.n = f3(0.0f, 0.0f, 0.0f);
            d.area = (float)((i1 - i0) * (j1 - j0));
            d.scale = 1.0f;
            d.env = me;
            any_env = true;
            continue;
        }
        d.c = f3(r[1], r[2], r[3]);
        d.e1 = f3(r[4], r[5], r[6]);
        d.e2 = f3(r[7], r[8], r[9]);
        const double cx = (double)d.e1.y * d.e2.z - (double)d.e1.z * d.e2.y;
        const double cy = (double)d.e1.z * d.e2.x - (double)d.e1.x * d.e2.z;
        const double cz = (double)d.e1.x * d.e2.y - (double)d.e1.y * d.e2.x;
        const double cl = sqrt(cx * cx + cy * cy + cz * cz);
        if (!(cl > 0.0)) return fail(c, FR_EINVAL, "degenerate emitter");
        if (!(ls->a[j] > 0.0f) || !(ls->d[j] > 0.0f)) return fail(c, FR_EINVAL, "light d and a must be > 0");
        d.n = f3((float)(cx / cl), (float)(cy / cl), (float)(cz / cl));
        if (d.type == 0) d.area = (float)cl;
        else if (d.type == 1) d.area = (float)(0.5 * cl);
        else d.area = (float)(3.14159265358979323846 * ((double)d.e1.x * d.e1.x + (double)d.e1.y * d.e1.y + (double)d.e1.z * d.e1.z));
        d.scale = (float)((double)ls->d[j] * ls->d[j] / ls->a[j]);
        d.env = 0;
    }
    if (any_env && ls->stage) return fail(c, FR_EINVAL, "environment blocks cannot be combined with a light stage");
    if (!c->lights) TRY(dalloc(c, &c->lights, FR_MAX_LIGHTS));
    CK(c, cudaMemcpy(c->lights, L.data(), sizeof(LightDev) * L.size(), cudaMemcpyHostToDevice));
    c->env_size = any_env ? ls->env_size : 0;
    c->use_stage = ls->stage != nullptr;
    if (ls->stage) {
        if (!c->stage) TRY(dalloc(c, &c->stage, 12 * (size_t)FR_MAX_LIGHTS));
        CK(c, cudaMemcpy(c->stage, ls->stage, sizeof(float) * 12 * ls->n_lights, cudaMemcpyHostToDevice));
    }
    c->NL = ls->n_lights;
    c->light_d_h.assign(ls->d, ls->d + ls->n_lights);
    c->light_a_h.assign(ls->a, ls->a + ls->n_lights);
    c->have_lights = true;
    return FR_OK;
}

fr_status fr_forward(fr_ctx* c, const fr_params* p, float* image, uint32_t iteration, uint32_t face_id,
                     void* stream) {
    TRY(check_params(c, p));
    if (!image) return fail(c, FR_EINVAL, "null image");
    const cudaStream_t st = S_(stream);
    c->h_items[0] = make_item(c, 0, single(c, p, nullptr, image, nullptr, iteration, face_id));
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    TRY(forward_pass(c, 1, st));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_backward(fr_ctx* c, const fr_params* p, const float* adj_image, fr_grads* g, uint32_t iteration,
                      uint32_t face_id, void* stream) {
    TRY(check_params(c, p));
    if (!adj_image || !g) return fail(c, FR_EINVAL, "null argument");
    const cudaStream_t st = S_(stream);
    c->h_items[0] = make_item(c, 0, single(c, p, g, nullptr, adj_image, iteration, face_id));
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    TRY(adjoint_pass(c, 1, st));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_loss(fr_ctx* c, const float* image, const float* target, double* loss, float* adj_image,
                  float* blurred, void* stream) {
    if (!c || !image || !target || !loss) return fail(c, FR_EINVAL, "null argument");
    if (c->poisoned) return fail(c, FR_ECUDA, "context unusable after an unsafe device timeout");
    launch_loss(c->cfg.height, c->cfg.width, image, target, loss, c->slots[0].sign, c->slots[0].loss_part, blurred,
                adj_image, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_render(fr_ctx* c, const fr_params* p, const float* target, float* image, double* loss, fr_grads* g,
                    uint32_t iteration, uint32_t face_id, void* stream) {
    TRY(check_params(c, p));
    if (!image || !target || !loss) return fail(c, FR_EINVAL, "null argument");
    const cudaStream_t st = S_(stream);
    mark(c, 0, st);
    ItemArgs a = single(c, p, g, image, nullptr, iteration, face_id);
    a.records = g != nullptr;
    c->h_items[0] = make_item(c, 0, a);
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    mark(c, 1, st);
    if (g) TRY(fork_prep(c, 1, st));
    TRY(forward_pass(c, 1, st));
    mark(c, 2, st);
    const float* tg[1] = {target};
    double* ls[1] = {loss};
    launch_loss(loss_table(c, 1, tg, ls, g != nullptr), st);
    mark(c, 3, st);
    if (g) {
        TRY(join_prep(c, st));
        TRY(adjoint_main(c, 1, st));
    }
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_render_batch(fr_ctx* c, const fr_item* items, int32_t n, void* stream) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    if (!items || n < 1 || n > c->max_batch) return fail(c, FR_EINVAL, "1 <= n <= max_batch items required");
    const cudaStream_t st = S_(stream);
    bool any_grad = false;
    const float* tg[FR_MAX_BATCH];
    double* ls[FR_MAX_BATCH];
    for (int k = 0; k < n; ++k) {
        const fr_item& x = items[k];
        TRY(check_params(c, &x.params));
        TRY(check_image_args(c, x.width, x.height, x.spp, x.edge_spp));
        if (!x.image || !x.target || !x.loss) return fail(c, FR_EINVAL, "null image, target or loss");
        ItemArgs a;
        a.W = x.width; a.H = x.height; a.spp = x.spp; a.edge_spp = x.edge_spp;
        a.flags = x.flags; a.iteration = x.iteration; a.face = x.face_id;
        a.p = &x.params; a.g = x.grads; a.image = x.image; a.adj = nullptr; a.tri_rec = nullptr;
        a.mask_rec = nullptr;
        a.records = true;
        c->h_items[k] = make_item(c, k, a);
        tg[k] = x.target;
        ls[k] = x.loss;
        any_grad |= x.grads != nullptr;
    }
    mark(c, 0, st);
    TRY(upload(c, n, st));
    build_geometry(c, n, st);
    mark(c, 1, st);
    if (any_grad) TRY(fork_prep(c, n, st));
    TRY(forward_pass(c, n, st));
    mark(c, 2, st);
    launch_loss(loss_table(c, n, tg, ls, any_grad), st);
    mark(c, 3, st);
    if (any_grad) {
        // items without gradients run the reverse pass on a zero adjoint; their
        // parameter outputs are null, so nothing is written for them
        for (int k = 0; k < n; ++k)
            if (!items[k].grads)
                CK(c, cudaMemsetAsync(c->slots[k].adj_image, 0,
                                      sizeof(float) * 3 * (size_t)items[k].width * items[k].height, st));
        TRY(join_prep(c, st));
        TRY(adjoint_main(c, n, st));
    }
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_set_flags(fr_ctx* c, uint32_t flags) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    c->cfg.flags = flags;
    return FR_OK;
}

fr_status fr_debug_wait_timeout(fr_ctx* c, uint32_t polls, void* stream) {
    if (!c || polls < 1 || polls > (1u << 22)) return fail(c, FR_EINVAL, "1 <= polls <= 2^22");
    launch_wait_probe(polls, c->status, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_record_tile(fr_ctx* c, int64_t samples) {
    if (!c || samples < 0) return fail(c, FR_EINVAL, "bad argument");
    if (samples == 0) {
        c->rec_tile = 0;
        return FR_OK;
    }
    const long unit = std::max(128, c->cfg.spp);
    c->rec_tile = std::max(unit, (long)samples / unit * unit);
    return FR_OK;
}

fr_status fr_sync_status(fr_ctx* c, void* stream) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    CK(c, cudaStreamSynchronize(S_(stream)));
    int s = 0;
    CK(c, cudaMemcpy(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(c, cudaMemset(c->status, 0, sizeof(int)));
    if (s & FR_STATUS_TIMEOUT_UNSAFE) {
        c->poisoned = true;
        return fail(c, FR_ETIMEOUT, "bounded wait gave up and copies or MMAs may still be in flight: "
                                    "the context is unusable");
    }
    if (s & FR_STATUS_STACK_OVERFLOW) return fail(c, FR_EOVERFLOW, "traversal stack overflow");
    if (s & FR_STATUS_TIMEOUT) return fail(c, FR_ETIMEOUT, "bounded wait gave up");
    if (s & FR_STATUS_BAD_BVH) return fail(c, FR_EOVERFLOW, "invalid BVH (construction check failed)");
    return FR_OK;
}

const char* fr_last_error(const fr_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

void fr_destroy(fr_ctx* c) {
    if (!c) return;
    cudaDeviceSynchronize();
    for (cudaEvent_t& e : c->ev)
        if (e) cudaEventDestroy(e);
    destroy_side(c);
    free_all(c);
    delete c;
}

fr_status fr_philox(uint32_t k0, uint32_t k1, const uint32_t* counters, int32_t n, uint32_t* out, void* stream) {
    if (!counters || !out || n < 0) return fail(nullptr, FR_EINVAL, "bad argument");
    launch_philox(k0, k1, counters, n, out, S_(stream));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FR_OK : fail(nullptr, FR_ECUDA, cudaGetErrorString(e));
}

fr_status fr_debug_geometry(fr_ctx* c, const fr_params* p, float* v_cam, float* n_vert, void* stream) {
    TRY(check_params(c, p));
    const cudaStream_t st = S_(stream);
    c->h_items[0] = make_item(c, 0, single(c, p, nullptr, nullptr, nullptr, 0, 0));
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    if (v_cam)
        CK(c, cudaMemcpy2DAsync(v_cam, 3 * sizeof(float), c->slots[0].v_cam, sizeof(float4), 3 * sizeof(float), c->N,
                                cudaMemcpyDeviceToDevice, st));
    if (n_vert)
        CK(c, cudaMemcpy2DAsync(n_vert, 3 * sizeof(float), c->slots[0].vn, sizeof(float4), 3 * sizeof(float), c->N,
                                cudaMemcpyDeviceToDevice, st));
    return FR_OK;
}

fr_status fr_debug_trace(fr_ctx* c, const fr_params* p, const float* org, const float* dir, int32_t n,
                         int32_t* tri, float* t, void* stream) {
    TRY(check_params(c, p));
    if (!org || !dir || !tri || !t || n < 0) return fail(c, FR_EINVAL, "bad argument");
    const cudaStream_t st = S_(stream);
    c->h_items[0] = make_item(c, 0, single(c, p, nullptr, nullptr, nullptr, 0, 0));
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    launch_trace_rays(c->d_items, org, dir, n, tri, t, st);
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_records(fr_ctx* c, const fr_params* p, float* image, int32_t* tri_rec, uint64_t* mask_rec,
                           uint32_t iteration, uint32_t face_id, void* stream) {
    TRY(check_params(c, p));
    if (!image) return fail(c, FR_EINVAL, "null image");
    const cudaStream_t st = S_(stream);
    ItemArgs a = single(c, p, nullptr, image, nullptr, iteration, face_id);
    a.tri_rec = tri_rec;
    a.mask_rec = mask_rec;
    c->h_items[0] = make_item(c, 0, a);
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    TRY(forward_pass(c, 1, st));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_silhouettes(fr_ctx* c, const fr_params* p, int32_t* prim, int32_t* n_prim, int32_t* per_light,
                               int32_t* counts, void* stream) {
    TRY(check_params(c, p));
    const cudaStream_t st = S_(stream);
    c->h_items[0] = make_item(c, 0, single(c, p, nullptr, nullptr, nullptr, 0, 0));
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    launch_classify(c->d_items, 1, c->E, c->NL, c->T, st);
    const Slot& sl = c->slots[0];
    if (prim) CK(c, cudaMemcpyAsync(prim, sl.lists, sizeof(int) * c->E, cudaMemcpyDeviceToDevice, st));
    if (n_prim) CK(c, cudaMemcpyAsync(n_prim, sl.counts, sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (per_light)
        CK(c, cudaMemcpyAsync(per_light, sl.lists + c->E, sizeof(int) * (size_t)c->NL * c->E, cudaMemcpyDeviceToDevice, st));
    if (counts) CK(c, cudaMemcpyAsync(counts, sl.counts + 1, sizeof(int) * c->NL, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_bvh(fr_ctx* c, const fr_params* p, int32_t* out, void* stream) {
    TRY(check_params(c, p));
    if (!out) return fail(c, FR_EINVAL, "null out");
    const cudaStream_t st = S_(stream);
    c->h_items[0] = make_item(c, 0, single(c, p, nullptr, nullptr, nullptr, 0, 0));
    TRY(upload(c, 1, st));
    build_geometry(c, 1, st);
    launch_bvh_check(c->d_items, c->T, out, st);
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_morph(fr_ctx* c, const fr_params* params, int32_t n, float* out, void* stream) {
    if (!c || !params || !out || n < 1 || n > c->max_batch) return fail(c, FR_EINVAL, "bad argument");
    if (c->poisoned) return fail(c, FR_ECUDA, "context unusable after an unsafe device timeout");
    const cudaStream_t st = S_(stream);
    for (int k = 0; k < n; ++k) {
        TRY(check_params(c, &params[k]));
        c->h_items[k] = make_item(c, k, single(c, &params[k], nullptr, nullptr, nullptr, 0, 0));
    }
    TRY(upload(c, n, st));
    morph(c, n, st);
    for (int k = 0; k < n; ++k)
        CK(c, cudaMemcpyAsync(out + (size_t)k * 3 * c->N, c->slots[k].v_model, sizeof(float) * 3 * c->N,
                              cudaMemcpyDeviceToDevice, st));
    CK(c, cudaGetLastError());
    return FR_OK;
}

int32_t fr_num_edges(const fr_ctx* c) { return c ? c->E : 0; }

fr_status fr_counters(fr_ctx* c, uint64_t* out, int32_t reset, void* stream) {
    if (!c || !out) return fail(c, FR_EINVAL, "null argument");
    CK(c, cudaStreamSynchronize(S_(stream)));
    unsigned long long h[9];
    CK(c, cudaMemcpy(h, c->counters, sizeof(h), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 9; ++k) out[k] = h[k];
    if (reset) CK(c, cudaMemset(c->counters, 0, sizeof(h)));
    return FR_OK;
}

fr_status fr_set_timing(fr_ctx* c, int32_t on) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    if (on && !c->ev[0])
        for (cudaEvent_t& e : c->ev) CK(c, cudaEventCreate(&e));
    c->timing = on != 0;
    return FR_OK;
}

fr_status fr_get_timing(fr_ctx* c, float* out) {
    if (!c || !out) return fail(c, FR_EINVAL, "null argument");
    if (!c->ev[0]) return fail(c, FR_EINVAL, "timing was never enabled");
    CK(c, cudaEventSynchronize(c->ev[7]));
    for (int k = 0; k < 7; ++k) CK(c, cudaEventElapsedTime(&out[k], c->ev[k], c->ev[k + 1]));
    CK(c, cudaEventElapsedTime(&out[7], c->ev[0], c->ev[7]));
    return FR_OK;
}

uint64_t fr_kernel_launches(void) { return g_launches.load(); }

}  // extern "C"
