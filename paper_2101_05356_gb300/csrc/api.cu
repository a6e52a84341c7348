// C-ABI of the facert library: context and scratch ownership, argument checks
// and the orchestration of the hot path (include/facert.h documents each call).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/facert.h"
#include "common.cuh"
#include "kernels.h"

struct fr_ctx {
    fr_config cfg{};
    int N = 0, T = 0, K = 0, NL = 0, E = 0, ld = 0;
    bool have_mesh = false, have_lights = false;
    std::string err;
    // mesh and lights
    float* mean = nullptr;
    float* basis = nullptr;
    int4* faces = nullptr;
    float2* uv = nullptr;
    int* vf_off = nullptr;
    int* vf_idx = nullptr;
    int4* edges = nullptr;
    LightDev* lights = nullptr;
    // per-call geometry
    float* v_model = nullptr;
    float4* v_cam = nullptr;
    float4* vn = nullptr;
    float4* n_face = nullptr;
    BvhScratch B{};
    BvhNode* nodes = nullptr;
    float4* tris = nullptr;
    // edges
    uint8_t* sil_flags = nullptr;
    int* lists = nullptr;
    int* counts = nullptr;
    // adjoint
    float* d_v = nullptr;
    float* d_n = nullptr;
    float* dm = nullptr;
    float* d_vmodel = nullptr;
    double* small = nullptr;
    double* acc12 = nullptr;
    // loss
    float* sign = nullptr;
    float* adj_image = nullptr;
    int* status = nullptr;
    unsigned long long* counters = nullptr;   // [kernel][rays, nodes, triangle tests]
    // per-stage CUDA-event timing
    bool timing = false;
    cudaEvent_t ev[9] = {};
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

#define TRY(x)                         \
    do {                               \
        fr_status s_ = (x);            \
        if (s_ != FR_OK) return s_;    \
    } while (0)

cudaStream_t S_(void* s) { return static_cast<cudaStream_t>(s); }

// stage marks: 0 start, 1 after build, 2 after forward, 3 after loss,
// 4 after classify, 5 after adjoint, 6 after edge_primary, 7 after chain
void mark(fr_ctx* c, int k, cudaStream_t st) {
    if (c->timing) cudaEventRecord(c->ev[k], st);
}

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

fr_status check_params(fr_ctx* c, const fr_params* p) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    if (!c->have_mesh || !c->have_lights) return fail(c, FR_EINVAL, "mesh and lights must be set first");
    if (!p || !p->rot || !p->trans || !p->focal || !p->light_i || !p->diffuse || !p->specular || !p->roughness ||
        (c->K > 0 && !p->coef))
        return fail(c, FR_EINVAL, "null parameter pointer");
    return FR_OK;
}

DevScene scene_of(const fr_ctx* c) {
    DevScene s;
    s.N = c->N; s.T = c->T; s.K = c->K; s.NL = c->NL; s.E = c->E;
    s.W = c->cfg.width; s.H = c->cfg.height; s.spp = c->cfg.spp; s.M = c->cfg.tex_size;
    s.edge_spp = c->cfg.edge_spp;
    s.flags = c->cfg.flags; s.seed = c->cfg.seed;
    s.v = c->v_cam; s.vn = c->vn; s.uv = c->uv; s.faces = c->faces; s.nodes = c->nodes; s.tris = c->tris;
    s.lights = c->lights; s.status = c->status; s.counters = c->counters;
    return s;
}

DevParams params_of(const fr_params* p) {
    return DevParams{p->coef, p->rot, p->trans, p->focal, p->light_i, p->diffuse, p->specular, p->roughness};
}

EdgeLists lists_of(const fr_ctx* c) {
    EdgeLists L;
    L.edges = c->edges;
    L.prim_list = c->lists;
    L.prim_count = c->counts;
    L.light_list = c->lists + c->E;
    L.light_count = c->counts + 1;
    return L;
}

// morph -> pose -> face normals + Morton keys -> vertex normals -> LBVH
fr_status build_geometry(fr_ctx* c, const fr_params* p, cudaStream_t st) {
    if (c->K > 0) launch_morph(c->mean, c->basis, c->ld, c->K, p->coef, c->v_model, st);
    else CK(c, cudaMemcpyAsync(c->v_model, c->mean, sizeof(float) * c->ld, cudaMemcpyDeviceToDevice, st));
    launch_pose(c->v_model, c->N, p->rot, p->trans, c->v_cam, c->B.aabb, st);
    launch_faces(c->v_cam, c->faces, c->T, c->B.aabb, c->n_face, c->B.keys, c->B.vals, st);
    launch_vertex_normals(c->n_face, c->vf_off, c->vf_idx, c->N, c->vn, st);
    launch_lbvh(c->v_cam, c->faces, c->T, c->B, c->nodes, c->tris, c->status, st);
    CK(c, cudaGetLastError());
    return FR_OK;
}

// reverse pass given geometry already built for p
fr_status adjoint_pass(fr_ctx* c, const fr_params* p, const float* adj_image, fr_grads* g, uint32_t iteration,
                       uint32_t face, cudaStream_t st) {
    const DevScene S = scene_of(c);
    const DevParams P = params_of(p);
    const EdgeLists EL = lists_of(c);
    CK(c, cudaMemsetAsync(c->d_v, 0, sizeof(float) * 3 * (size_t)c->N, st));
    CK(c, cudaMemsetAsync(c->d_n, 0, sizeof(float) * 3 * (size_t)c->N, st));
    CK(c, cudaMemsetAsync(c->small, 0, sizeof(double) * (1 + 3 * FR_MAX_LIGHTS), st));
    CK(c, cudaMemsetAsync(c->acc12, 0, sizeof(double) * 12, st));
    const bool need_edges = !(c->cfg.flags & FR_FLAG_NO_PRIMARY_EDGE) || !(c->cfg.flags & FR_FLAG_NO_SHADOW_EDGE);
    if (need_edges) launch_classify(S, EL, c->sil_flags, st);
    mark(c, 4, st);
    DevGrads G;
    G.d_v = c->d_v;
    G.d_n = c->d_n;
    G.diffuse = g->diffuse;
    G.specular = g->specular;
    G.roughness = g->roughness;
    G.small = c->small;
    launch_adjoint(S, P, G, EL, adj_image, iteration, face, st);
    mark(c, 5, st);
    if (!(c->cfg.flags & FR_FLAG_NO_PRIMARY_EDGE) && c->cfg.edge_spp > 0)
        launch_edge_primary(S, P, G, EL, adj_image, iteration, face, st);
    mark(c, 6, st);
    launch_normals_adjoint(c->v_cam, c->vn, c->d_n, c->faces, c->vf_off, c->vf_idx, c->N, c->dm, c->d_v, st);
    launch_pose_adjoint(c->v_model, c->N, c->ld, p->rot, p->trans, c->d_v, c->d_vmodel, c->acc12, st);
    launch_pose_finish(p->rot, c->acc12, c->small, c->NL, g->rot, g->trans, g->focal, g->light_i, st);
    if (g->coef) launch_morph_adjoint(c->basis, c->ld, c->K, 3 * c->N, c->d_vmodel, g->coef, st);
    mark(c, 7, st);
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status alloc_scratch(fr_ctx* c) {
    const int N = c->N, T = c->T;
    TRY(dalloc(c, &c->v_model, c->ld));
    TRY(dalloc(c, &c->d_vmodel, c->ld));
    TRY(dalloc(c, &c->v_cam, N));
    TRY(dalloc(c, &c->vn, N));
    TRY(dalloc(c, &c->n_face, T));
    const int n_tiles = (T + 255) / 256;
    TRY(dalloc(c, &c->B.keys, T));
    TRY(dalloc(c, &c->B.keys_alt, T));
    TRY(dalloc(c, &c->B.vals, T));
    TRY(dalloc(c, &c->B.vals_alt, T));
    TRY(dalloc(c, &c->B.hist, 256 * (size_t)n_tiles));
    TRY(dalloc(c, &c->B.child, 2 * (size_t)std::max(T - 1, 1)));
    TRY(dalloc(c, &c->B.parent_int, std::max(T - 1, 1)));
    TRY(dalloc(c, &c->B.parent_leaf, T));
    TRY(dalloc(c, &c->B.flag, std::max(T - 1, 1)));
    TRY(dalloc(c, &c->B.box_int, 2 * (size_t)std::max(T - 1, 1)));
    TRY(dalloc(c, &c->B.box_leaf, 2 * (size_t)T));
    TRY(dalloc(c, &c->B.aabb, 6));
    TRY(dalloc(c, &c->nodes, std::max(T - 1, 1)));
    TRY(dalloc(c, &c->tris, 3 * (size_t)T));
    TRY(dalloc(c, &c->sil_flags, (size_t)(1 + FR_MAX_LIGHTS) * c->E));
    TRY(dalloc(c, &c->lists, (size_t)(1 + FR_MAX_LIGHTS) * c->E));
    TRY(dalloc(c, &c->counts, 1 + FR_MAX_LIGHTS));
    TRY(dalloc(c, &c->d_v, 3 * (size_t)N));
    TRY(dalloc(c, &c->d_n, 3 * (size_t)N));
    TRY(dalloc(c, &c->dm, 3 * (size_t)N));
    TRY(dalloc(c, &c->small, 1 + 3 * FR_MAX_LIGHTS));
    TRY(dalloc(c, &c->acc12, 12));
    return FR_OK;
}

}  // namespace

extern "C" {

fr_status fr_create(fr_ctx** out, const fr_config* cfg) {
    if (!out || !cfg) return fail(nullptr, FR_EINVAL, "null argument");
    *out = nullptr;
    if (cfg->width < 1 || cfg->width > 8192 || cfg->height < 1 || cfg->height > 8192)
        return fail(nullptr, FR_EINVAL, "image size out of range");
    if (!is_pow2(cfg->spp) || cfg->spp > 1024) return fail(nullptr, FR_EINVAL, "spp must be a power of two <= 1024");
    if (cfg->tex_size < 1 || cfg->tex_size > 8192) return fail(nullptr, FR_EINVAL, "tex_size out of range");
    if (cfg->edge_spp < 0 || cfg->edge_spp > 64) return fail(nullptr, FR_EINVAL, "edge_spp out of range");
    if ((long)cfg->width * cfg->height * cfg->spp > (1L << 31) - 1024)
        return fail(nullptr, FR_EINVAL, "too many samples per call");
    fr_ctx* c = new fr_ctx();
    c->cfg = *cfg;
    if (dalloc(c, &c->status, 1) != FR_OK || cudaMemset(c->status, 0, sizeof(int)) != cudaSuccess ||
        dalloc(c, &c->counters, 9) != FR_OK ||
        cudaMemset(c->counters, 0, 9 * sizeof(unsigned long long)) != cudaSuccess ||
        dalloc(c, &c->sign, (size_t)cfg->width * cfg->height * 3) != FR_OK ||
        dalloc(c, &c->adj_image, (size_t)cfg->width * cfg->height * 3) != FR_OK) {
        g_err = c->err;
        free_all(c);
        delete c;
        return FR_ENOMEM;
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
    c->ld = ((3 * N + 31) / 32) * 32;
    TRY(dalloc(c, &c->mean, c->ld));
    TRY(dalloc(c, &c->basis, (size_t)std::max(K, 1) * c->ld));
    TRY(dalloc(c, &c->faces, T));
    TRY(dalloc(c, &c->uv, N));
    TRY(dalloc(c, &c->vf_off, N + 1));
    TRY(dalloc(c, &c->vf_idx, 3 * (size_t)T));
    TRY(dalloc(c, &c->edges, c->E));
    std::vector<float> pad((size_t)c->ld, 0.0f);
    std::copy(m->mean, m->mean + 3 * (size_t)N, pad.begin());
    CK(c, cudaMemcpy(c->mean, pad.data(), sizeof(float) * c->ld, cudaMemcpyHostToDevice));
    for (int k = 0; k < K; ++k) {
        std::fill(pad.begin(), pad.end(), 0.0f);
        std::copy(m->basis + (size_t)k * 3 * N, m->basis + (size_t)(k + 1) * 3 * N, pad.begin());
        CK(c, cudaMemcpy(c->basis + (size_t)k * c->ld, pad.data(), sizeof(float) * c->ld, cudaMemcpyHostToDevice));
    }
    std::vector<int4> f4(T);
    for (int f = 0; f < T; ++f) f4[f] = make_int4(m->faces[3 * f], m->faces[3 * f + 1], m->faces[3 * f + 2], 0);
    CK(c, cudaMemcpy(c->faces, f4.data(), sizeof(int4) * T, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->uv, m->uv, sizeof(float2) * N, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->vf_off, deg.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->vf_idx, vf.data(), sizeof(int) * 3 * (size_t)T, cudaMemcpyHostToDevice));
    CK(c, cudaMemcpy(c->edges, edges.data(), sizeof(int4) * c->E, cudaMemcpyHostToDevice));
    TRY(alloc_scratch(c));
    c->have_mesh = true;
    return FR_OK;
}

fr_status fr_set_lights(fr_ctx* c, const fr_light_stage* ls) {
    if (!c || !ls || !ls->records || !ls->d || !ls->a) return fail(c, FR_EINVAL, "null argument");
    if (ls->n_lights < 1 || ls->n_lights > FR_MAX_LIGHTS) return fail(c, FR_EINVAL, "1 <= n_lights <= 64");
    std::vector<LightDev> L(ls->n_lights);
    for (int j = 0; j < ls->n_lights; ++j) {
        const float* r = ls->records + 11 * j;
        LightDev& d = L[j];
        d.type = (int)r[0];
        if (d.type < 0 || d.type > 2) return fail(c, FR_EINVAL, "unknown emitter type");
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
        d.pad = 0;
    }
    if (!c->lights) TRY(dalloc(c, &c->lights, FR_MAX_LIGHTS));
    CK(c, cudaMemcpy(c->lights, L.data(), sizeof(LightDev) * L.size(), cudaMemcpyHostToDevice));
    c->NL = ls->n_lights;
    c->have_lights = true;
    return FR_OK;
}

fr_status fr_forward(fr_ctx* c, const fr_params* p, float* image, uint32_t iteration, uint32_t face_id,
                     void* stream) {
    TRY(check_params(c, p));
    if (!image) return fail(c, FR_EINVAL, "null image");
    TRY(build_geometry(c, p, S_(stream)));
    launch_forward(scene_of(c), params_of(p), image, nullptr, nullptr, iteration, face_id, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_backward(fr_ctx* c, const fr_params* p, const float* adj_image, fr_grads* g, uint32_t iteration,
                      uint32_t face_id, void* stream) {
    TRY(check_params(c, p));
    if (!adj_image || !g) return fail(c, FR_EINVAL, "null argument");
    TRY(build_geometry(c, p, S_(stream)));
    return adjoint_pass(c, p, adj_image, g, iteration, face_id, S_(stream));
}

fr_status fr_loss(fr_ctx* c, const float* image, const float* target, double* loss, float* adj_image,
                  float* blurred, void* stream) {
    if (!c || !image || !target || !loss) return fail(c, FR_EINVAL, "null argument");
    launch_loss(c->cfg.height, c->cfg.width, image, target, loss, c->sign, blurred, adj_image, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_render(fr_ctx* c, const fr_params* p, const float* target, float* image, double* loss, fr_grads* g,
                    uint32_t iteration, uint32_t face_id, void* stream) {
    TRY(check_params(c, p));
    if (!image || !target || !loss) return fail(c, FR_EINVAL, "null argument");
    const cudaStream_t st = S_(stream);
    mark(c, 0, st);
    TRY(build_geometry(c, p, st));
    mark(c, 1, st);
    launch_forward(scene_of(c), params_of(p), image, nullptr, nullptr, iteration, face_id, st);
    mark(c, 2, st);
    launch_loss(c->cfg.height, c->cfg.width, image, target, loss, c->sign, nullptr, g ? c->adj_image : nullptr, st);
    mark(c, 3, st);
    CK(c, cudaGetLastError());
    if (g) return adjoint_pass(c, p, c->adj_image, g, iteration, face_id, st);
    return FR_OK;
}

fr_status fr_set_flags(fr_ctx* c, uint32_t flags) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    c->cfg.flags = flags;
    return FR_OK;
}

fr_status fr_sync_status(fr_ctx* c, void* stream) {
    if (!c) return fail(nullptr, FR_EINVAL, "null context");
    CK(c, cudaStreamSynchronize(S_(stream)));
    int s = 0;
    CK(c, cudaMemcpy(&s, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(c, cudaMemset(c->status, 0, sizeof(int)));
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
    TRY(build_geometry(c, p, S_(stream)));
    if (v_cam)
        CK(c, cudaMemcpy2DAsync(v_cam, 3 * sizeof(float), c->v_cam, sizeof(float4), 3 * sizeof(float), c->N,
                                cudaMemcpyDeviceToDevice, S_(stream)));
    if (n_vert)
        CK(c, cudaMemcpy2DAsync(n_vert, 3 * sizeof(float), c->vn, sizeof(float4), 3 * sizeof(float), c->N,
                                cudaMemcpyDeviceToDevice, S_(stream)));
    return FR_OK;
}

fr_status fr_debug_trace(fr_ctx* c, const fr_params* p, const float* org, const float* dir, int32_t n,
                         int32_t* tri, float* t, void* stream) {
    TRY(check_params(c, p));
    if (!org || !dir || !tri || !t || n < 0) return fail(c, FR_EINVAL, "bad argument");
    TRY(build_geometry(c, p, S_(stream)));
    launch_trace_rays(scene_of(c), org, dir, n, tri, t, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_records(fr_ctx* c, const fr_params* p, float* image, int32_t* tri_rec, uint64_t* mask_rec,
                           uint32_t iteration, uint32_t face_id, void* stream) {
    TRY(check_params(c, p));
    if (!image) return fail(c, FR_EINVAL, "null image");
    TRY(build_geometry(c, p, S_(stream)));
    launch_forward(scene_of(c), params_of(p), image, tri_rec, mask_rec, iteration, face_id, S_(stream));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_silhouettes(fr_ctx* c, const fr_params* p, int32_t* prim, int32_t* n_prim, int32_t* per_light,
                               int32_t* counts, void* stream) {
    TRY(check_params(c, p));
    TRY(build_geometry(c, p, S_(stream)));
    const EdgeLists EL = lists_of(c);
    launch_classify(scene_of(c), EL, c->sil_flags, S_(stream));
    const cudaStream_t st = S_(stream);
    if (prim) CK(c, cudaMemcpyAsync(prim, c->lists, sizeof(int) * c->E, cudaMemcpyDeviceToDevice, st));
    if (n_prim) CK(c, cudaMemcpyAsync(n_prim, c->counts, sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (per_light)
        CK(c, cudaMemcpyAsync(per_light, c->lists + c->E, sizeof(int) * (size_t)c->NL * c->E, cudaMemcpyDeviceToDevice, st));
    if (counts) CK(c, cudaMemcpyAsync(counts, c->counts + 1, sizeof(int) * c->NL, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaGetLastError());
    return FR_OK;
}

fr_status fr_debug_bvh(fr_ctx* c, const fr_params* p, int32_t* out, void* stream) {
    TRY(check_params(c, p));
    if (!out) return fail(c, FR_EINVAL, "null out");
    TRY(build_geometry(c, p, S_(stream)));
    launch_bvh_check(c->nodes, c->B, c->T, out, S_(stream));
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
