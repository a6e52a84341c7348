// Forward render, adjoint (interior + shadow-boundary terms), primary-edge
// boundary term and silhouette classification (Sec. 4: the Monte Carlo
// estimator F with shadow rays, differentiated with edge sampling).
//
// One thread per camera sample (pixel, sample).  Shadow rays of a warp are
// compacted through a 64-entry ring in shared memory so that every traversal
// launched runs 32 lanes wide; the visibility outcome lands in a per-lane
// bitmask and each lane then sums its own visible lights in light order, so the
// result does not depend on the compaction order.
#include "common.cuh"
#include "kernels.h"
#include "shade.cuh"
#include "trace.cuh"

namespace {

constexpr int RT_THREADS = 128;
constexpr int RT_WARPS = RT_THREADS / 32;

// Traversal stack placement: a per-thread array in local memory (L1-cached,
// default) or a [FR_STACK][RT_THREADS] shared-memory array.  Measured on GB300
// (paper-scale face): local stacks let 8 forward / 6 adjoint blocks reside per
// SM and run the forward 1.5x and the adjoint 1.2x faster than shared stacks at
// 3 blocks per SM.
#ifndef FR_STACK_LOCAL
#define FR_STACK_LOCAL 1
#endif
// minimum resident blocks per SM requested from the compiler (register cap).
// Measured on GB300 (paper-scale face): the forward is fastest at 10 blocks
// (3.11 ms; 8: 3.28 ms, 12: 3.47 ms), the primary-edge kernel at 8, the
// adjoint reading hit records at 5 (0.601 ms; 6: 0.618 ms, 8: 0.637 ms) and
// the re-tracing adjoint at 8 (4.20 ms; 6: 4.38 ms, 5: 4.65 ms).
#ifndef FR_FWD_MIN_BLOCKS
#define FR_FWD_MIN_BLOCKS 10
#endif
#ifndef FR_EDGE_MIN_BLOCKS
#define FR_EDGE_MIN_BLOCKS 8
#endif
#ifndef FR_ADJ_REC_MIN_BLOCKS
#define FR_ADJ_REC_MIN_BLOCKS 5
#endif
#ifndef FR_ADJ_MIN_BLOCKS
#define FR_ADJ_MIN_BLOCKS 8
#endif
constexpr unsigned FULL = 0xffffffffu;
constexpr float SHADOW_EPS = 1e-4f;     // shadow segment trimmed to (eps, 1 - eps)

struct WarpQueue {
    float4 job[64][2];                  // (y.xyz, z.x) (z.y, z.z, skip slot, owner | light << 8 | distant << 16)
    unsigned long long vis[32];
};

struct RtShared {
#if !FR_STACK_LOCAL
    int stack[FR_STACK * RT_THREADS];
#endif
    WarpQueue wq[RT_WARPS];
};

// Per-warp focal / light partials of the adjoint kernels live in dynamic
// shared memory: RT_WARPS rows of n values.  Each warp writes each of its
// values once (an FP32 warp sum), so they are kept in FP32 and turned to FP64
// only by the block sum: the same doubles as converting each at once, without
// the narrow FP64 pipe in the per-light loop.
extern __shared__ float acc_dyn[];

#if FR_STACK_LOCAL
#define FR_STACK_DECL int lstack_[FR_STACK];
#define my_stack(sh) (Stack{lstack_, 1})
#else
#define FR_STACK_DECL
FR_D Stack my_stack(RtShared& sh) { return Stack{&sh.stack[threadIdx.x], RT_THREADS}; }
#endif

struct SampleState {
    bool hit;
    bool lit;          // shaded: the hit triangle faces the camera (and, with the view
                       // cutoff flag, n_s . o > 0); otherwise it reflects nothing
    int tri;
    int slot;          // the hit triangle's leaf slot (skipped by its shadow rays)
    float b1, b2;
    float3 d;          // camera ray direction (not normalised)
    float3 y, ns, o;
    float2 uv;
    Material m;
    Tap tap;
};

// Primary ray through screen point (sx, sy) and the shading state at its hit.
// rec >= -1 is this ray's recorded hit triangle (-1: miss) and replaces the
// traversal; rec = REC_TRACE traces.
// CAN_TRACE = false compiles the traversal out (callers that always have a
// record).
constexpr int REC_TRACE = -2;

// The material fetch of a shading state (bilinear taps of the diffuse,
// specular and roughness textures at the hit's uv).
FR_D void sample_material(const DevScene& S, const DevParams& P, SampleState& ss) {
    if (!ss.hit) return;
    ss.tap = make_tap(S.M, ss.uv.x, ss.uv.y);
    ss.m.c = f3(tap_fetch(P.diffuse, 3, 0, ss.tap, S.M, nullptr, nullptr),
                tap_fetch(P.diffuse, 3, 1, ss.tap, S.M, nullptr, nullptr),
                tap_fetch(P.diffuse, 3, 2, ss.tap, S.M, nullptr, nullptr));
    ss.m.s = f3(tap_fetch(P.specular, 3, 0, ss.tap, S.M, nullptr, nullptr),
                tap_fetch(P.specular, 3, 1, ss.tap, S.M, nullptr, nullptr),
                tap_fetch(P.specular, 3, 2, ss.tap, S.M, nullptr, nullptr));
    ss.m.r = tap_fetch(P.roughness, 1, 0, ss.tap, S.M, nullptr, nullptr);
}

// MATERIAL = false leaves the material to a later sample_material call (the
// forward fetches it after the shadow traversal, so it is not live across it).
// `given` (non-null) imposes the hit instead (its triangle, slot and barycentrics).
template <bool CAN_TRACE = true, bool MATERIAL = true>
FR_D void primary_state(const DevScene& S, const DevParams& P, bool active, float sx, float sy,
                        Stack st, SampleState& ss, RayStats& rs, int rec = REC_TRACE, const Hit* given = nullptr) {
    ss.hit = false;
    ss.lit = false;
    ss.tri = ss.slot = -1;
    if (!active) return;
    const float f = __ldg(P.focal);
    ss.d = f3((sx - 0.5f * S.W) / f, -(sy - 0.5f * S.H) / f, -1.0f);
    const RayPre r = ray_setup(f3(0.0f, 0.0f, 0.0f), ss.d);
    const Hit h = given ? *given
                        : (CAN_TRACE && rec == REC_TRACE) ? trace_closest(S, r, 0.0f, INFINITY, st, rs)
                                                          : hit_record(S, r, rec);
    if (h.tri < 0) return;
    ss.hit = true;
    ss.tri = h.tri;
    ss.slot = h.slot;
    ss.b1 = h.b1;
    ss.b2 = h.b2;
    const int4 fc = __ldg(&S.faces[h.tri]);
    const float b0 = 1.0f - h.b1 - h.b2;
    const float3 v0 = xyz(__ldg(&S.v[fc.x])), v1 = xyz(__ldg(&S.v[fc.y])), v2 = xyz(__ldg(&S.v[fc.z]));
    const float3 n0 = xyz(__ldg(&S.vn[fc.x])), n1 = xyz(__ldg(&S.vn[fc.y])), n2 = xyz(__ldg(&S.vn[fc.z]));
    ss.y = v0 * b0 + v1 * h.b1 + v2 * h.b2;
    const float3 m = n0 * b0 + n1 * h.b1 + n2 * h.b2;
    ss.ns = m * rsqrtf(dot(m, m));
    ss.o = -ss.d * rsqrtf(dot(ss.d, ss.d));
    // one-sided surfaces: seen from behind, a triangle reflects nothing (that
    // change happens at geometric silhouettes, which the primary-edge term samples)
    ss.lit = dot(cross(v1 - v0, v2 - v0), ss.o) > 0.0f &&
             (!(S.flags & FR_FLAG_VIEW_CUTOFF_D) || dot(ss.ns, ss.o) > 0.0f);
    const float2 t0 = __ldg(&S.uv[fc.x]), t1 = __ldg(&S.uv[fc.y]), t2 = __ldg(&S.uv[fc.z]);
    ss.uv = make_float2(b0 * t0.x + h.b1 * t1.x + h.b2 * t2.x, b0 * t0.y + h.b1 * t1.y + h.b2 * t2.y);
    if (MATERIAL) sample_material(S, P, ss);
}

// Light-sample dims of a sampler, cached per Philox block (warp-uniform).
struct DimCache {
    int b = -1;
    uint4 w;
    FR_D float2 pair(const Sampler& s, int d) {
        const int bb = d >> 2;
        if (bb != b) { w = s.block(bb); b = bb; }
        return (d & 2) ? make_float2(u24(w.z), u24(w.w)) : make_float2(u24(w.x), u24(w.y));
    }
};

FR_D bool light_visible_geometry(const LightDev& L, float3 z, const SampleState& ss) {
    const float3 lv = z - ss.y;
    return dot(ss.ns, lv) > 0.0f && -dot(L.n, lv) > 0.0f;
}

// Trace the queued jobs [head, head + n) of this warp's ring (lane k takes job k).
// ENV: the launch may hold environment blocks (lights at infinity); otherwise
// their code is compiled out.
template <bool ENV>
FR_D void drain(const DevScene& S, WarpQueue& q, int head, int n, Stack st, RayStats& rs) {
    const int lane = threadIdx.x & 31;
    if (lane < n) {
        const float4 a = q.job[(head + lane) & 63][0], b = q.job[(head + lane) & 63][1];
        const float3 y = f3(a.x, a.y, a.z), z = f3(a.w, b.x, b.y);
        const int skip = __float_as_int(b.z), tag = __float_as_int(b.w);
        // a segment y -> z to an area emitter, or a ray along the direction z
        // to a light at infinity
        const bool distant = ENV && ((tag >> 16) & 1);
        const RayPre r = ray_setup(y, distant ? z : z - y);
        if (!trace_any(S, r, SHADOW_EPS, distant ? INFINITY : 1.0f - SHADOW_EPS, skip, st, rs))
            atomicOr(&q.vis[tag & 31], 1ull << ((tag >> 8) & 63));
    }
    __syncwarp();
}

// Warp-cooperative shadow visibility for the lights [j0, j0 + 64): bit j - j0
// is set when the shadow ray to this lane's light-j sample is traced and
// unoccluded.  All 32 lanes must call this together.
template <bool ENV>
FR_D uint64_t shadow_mask(const DevScene& S, const SampleState& ss, const Sampler& smp, int dim0,
                          WarpQueue& q, Stack st, RayStats& rs, int j0) {
    const int lane = threadIdx.x & 31;
    q.vis[lane] = 0ull;
    __syncwarp();
    const bool want = ss.hit && ss.lit && !(S.flags & FR_FLAG_FLAT_D);
    int head = 0, count = 0;
    DimCache dc;
    const int j1 = min(S.NL, j0 + 64);
    for (int j = j0; j < j1; ++j) {
        bool need = false;
        float3 z = f3(0.0f, 0.0f, 0.0f);
        const bool distant = ENV && S.lights[j].type == FR_LIGHT_ENV_D;      // warp-uniform
        if (want) {
            const LightDev& L = S.lights[j];
            const float2 u = dc.pair(smp, dim0 + 2 * j);
            if (distant) {                       // z = the direction of the sample
                z = env_sample(L, u.x, u.y).w;
                need = dot(ss.ns, z) > 0.0f;
            } else {
                z = light_point(L, u.x, u.y);
                need = light_visible_geometry(L, z, ss);
            }
        }
        const unsigned ballot = __ballot_sync(FULL, need);
        if (need) {
            const int slot = (head + count + __popc(ballot & ((1u << lane) - 1u))) & 63;
            q.job[slot][0] = make_float4(ss.y.x, ss.y.y, ss.y.z, z.x);
            q.job[slot][1] = make_float4(z.y, z.z, __int_as_float(ss.slot),
                                         __int_as_float(lane | ((j - j0) << 8) | ((int)distant << 16)));
        }
        count += __popc(ballot);
        __syncwarp();
        if (count >= 32) {
            drain<ENV>(S, q, head, 32, st, rs);
            head = (head + 32) & 63;
            count -= 32;
        }
    }
    if (count > 0) drain<ENV>(S, q, head, count, st, rs);
    return q.vis[lane];
}

// Unoccluded contribution of light j at z (without the 1/pdf area factor):
// h = f_r cos_s cos_l / |z - y|^2 (RGB).  With ADJ, the upstream gradient gh
// (dE/dh per channel) flows into g (n, o, c, s, r) and into gy.
template <bool ADJ>
FR_D float3 light_h(uint32_t flags, const LightDev& L, float3 z, const SampleState& ss, float3 gh,
                    ShadeAdj* g, float3* gy, float3* gz = nullptr) {
    const float3 lv = z - ss.y;
    const float d2 = dot(lv, lv);
    const float inv_len = rsqrtf(d2);
    const float inv_d2 = inv_len * inv_len;
    const float3 l = lv * inv_len;
    const float cos_s = dot(ss.ns, l), cos_l = -dot(L.n, l);
    if (!(cos_s > 0.0f) || !(cos_l > 0.0f) || !ss.lit) return f3(0.0f, 0.0f, 0.0f);
    const float geo = cos_s * cos_l * inv_d2;
    float3 f;
    if (ADJ) {
        const float3 gf = f3(gh.x * geo, gh.y * geo, gh.z * geo);
        const float3 keep_l = g->l;
        g->l = f3(0.0f, 0.0f, 0.0f);
        f = brdf<true>(flags, ss.ns, l, ss.o, ss.m, gf, g);
        const float ggeo = gh.x * f.x + gh.y * f.y + gh.z * f.z;
        const float gcs = ggeo * cos_l * inv_d2, gcl = ggeo * cos_s * inv_d2, gd2 = -ggeo * geo * inv_d2;
        g->n += l * gcs;
        const float3 gl = g->l + ss.ns * gcs - L.n * gcl;
        g->l = keep_l;
        const float3 glv = (gl - l * dot(l, gl)) * inv_len + lv * (2.0f * gd2);
        *gy -= glv;
        if (gz) *gz = glv;                     // lv = z - y
    } else {
        f = brdf<false>(flags, ss.ns, l, ss.o, ss.m, f3(0, 0, 0), nullptr);
    }
    return f * geo;
}

// Unoccluded contribution of a light at infinity in direction l (without the
// 1/pdf weight): h = f_r cos_s.  l does not depend on the parameters; with ADJ
// the upstream gradient gh flows into g's n, o, c, s and r.
template <bool ADJ>
FR_D float3 light_h_env(uint32_t flags, float3 l, const SampleState& ss, float3 gh, ShadeAdj* g) {
    const float cos_s = dot(ss.ns, l);
    if (!(cos_s > 0.0f) || !ss.lit) return f3(0.0f, 0.0f, 0.0f);
    float3 f;
    if (ADJ) {
        const float3 keep_l = g->l;
        f = brdf<true>(flags, ss.ns, l, ss.o, ss.m, gh * cos_s, g);
        g->l = keep_l;
        g->n += l * (gh.x * f.x + gh.y * f.y + gh.z * f.z);
    } else {
        f = brdf<false>(flags, ss.ns, l, ss.o, ss.m, f3(0, 0, 0), nullptr);
    }
    return f * cos_s;
}

FR_D float3 env_radiance(const DevParams& P, int texel) {
    return f3(__ldg(&P.env[3 * texel]), __ldg(&P.env[3 * texel + 1]), __ldg(&P.env[3 * texel + 2]));
}

// Light j's frame in the virtual light stage and the velocities of an emitter
// point z (held at its emitter coordinates) with respect to (d, a, p0, p1):
// dz/dd = (z - C) / d, dz/da = (z - P) / (2 a), dz/dp0 = d (V0 - V2),
// dz/dp1 = d (V1 - V2) (P = C + d (p0 V0 + p1 V1 + p2 V2), Sec. 3.3).
struct StageFrame {
    float3 C, P, dA, dB;    // stage centre, light centre, V0 - V2, V1 - V2
    float d, a;
};

FR_D StageFrame stage_frame(const DevScene& S, const DevParams& P, int j) {
    const float* g = S.stage + 12 * j;
    StageFrame F;
    F.C = f3(g[0], g[1], g[2]);
    const float3 A = f3(g[3], g[4], g[5]), B = f3(g[6], g[7], g[8]), V = f3(g[9], g[10], g[11]);
    F.d = P.light_d[j];
    F.a = P.light_a[j];
    const float p0 = P.light_p[2 * j], p1 = P.light_p[2 * j + 1];
    F.P = F.C + (A * p0 + B * p1 + V * (1.0f - p0 - p1)) * F.d;
    F.dA = A - V;
    F.dB = B - V;
    return F;
}

FR_D float3 intensity(const DevScene& S, const DevParams& P, int j) {
    const float sc = S.lights[j].scale;
    return f3(sc * __ldg(&P.light_i[3 * j]), sc * __ldg(&P.light_i[3 * j + 1]), sc * __ldg(&P.light_i[3 * j + 2]));
}

// Radiance of this lane's sample given its state and visibility mask.
template <bool ENV>
FR_D float3 radiance_from(const DevScene& S, const DevParams& P, const SampleState& ss, uint64_t vis,
                          const Sampler& smp, int dim0, int j0) {
    float3 Lo = f3(0.0f, 0.0f, 0.0f);
    if (!ss.hit) return Lo;
    if (S.flags & FR_FLAG_FLAT_D) return j0 == 0 ? ss.m.c : Lo;
    DimCache dc;
    const int j1 = min(S.NL, j0 + 64);
    for (int j = j0; j < j1; ++j) {
        if (!((vis >> (j - j0)) & 1ull)) continue;
        const LightDev& L = S.lights[j];
        const float2 u = dc.pair(smp, dim0 + 2 * j);
        if (ENV && L.type == FR_LIGHT_ENV_D) {
            const EnvDir ed = env_sample(L, u.x, u.y);
            const float3 h = light_h_env<false>(S.flags, ed.w, ss, f3(0, 0, 0), nullptr);
            const float3 E = env_radiance(P, ed.texel);
            Lo += f3(h.x * E.x, h.y * E.y, h.z * E.z) * ed.weight;
            continue;
        }
        const float3 z = light_point(L, u.x, u.y);
        const float3 h = light_h<false>(S.flags, L, z, ss, f3(0, 0, 0), nullptr, nullptr);
        const float3 I = intensity(S, P, j);
        Lo += f3(h.x * I.x, h.y * I.y, h.z * I.z) * L.area;
    }
    return Lo;
}

// Warp-cooperative visibility at screen point (sx, sy): the camera ray's hit
// (without the material) and both shadow-visibility words.
template <bool ENV>
FR_D void visibility_at(const DevScene& S, const DevParams& P, bool active, float sx, float sy,
                        const Sampler& smp, int dim0, RtShared& sh, Stack stk, SampleState& ss, uint64_t* vis,
                        RayStats& rs) {
    primary_state<true, false>(S, P, active, sx, sy, stk, ss, rs);
    vis[0] = vis[1] = 0ull;
    for (int j0 = 0; j0 < max(S.NL, 1); j0 += 64)            // lights in chunks of 64 (warp-uniform)
        vis[j0 >> 6] = shadow_mask<ENV>(S, ss, smp, dim0, sh.wq[threadIdx.x >> 5], stk, rs, j0);
}

// Radiance of a sample whose visibility is known: the material, then the lights.
template <bool ENV>
FR_D float3 shade_visible(const DevScene& S, const DevParams& P, const Sampler& smp, int dim0, SampleState& ss,
                          const uint64_t* vis) {
    sample_material(S, P, ss);
    float3 Lo = f3(0.0f, 0.0f, 0.0f);
    for (int j0 = 0; j0 < max(S.NL, 1); j0 += 64) Lo += radiance_from<ENV>(S, P, ss, vis[j0 >> 6], smp, dim0, j0);
    return Lo;
}

// Full warp-cooperative radiance evaluation at screen point (sx, sy):
// visibility first, then the material and the radiance, so that the material
// is not live across the shadow traversal.
template <bool ENV>
FR_D float3 radiance_at(const DevScene& S, const DevParams& P, bool active, float sx, float sy,
                        const Sampler& smp, int dim0, RtShared& sh, Stack stk, SampleState& ss, uint64_t* vis,
                        RayStats& rs) {
    visibility_at<ENV>(S, P, active, sx, sy, smp, dim0, sh, stk, ss, vis, rs);
    return shade_visible<ENV>(S, P, smp, dim0, ss, vis);
}

FR_D float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// sum over aligned groups of `width` lanes (width a power of two <= 32)
FR_D float group_sum(float v, int width) {
    for (int o = width >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Visibility words a hit record holds: one for up to 64 lights, else two.
FR_D int vis_words(const DevScene& S) { return S.NL > 64 ? 2 : 1; }

FR_D void store_vis(const DevScene& S, uint64_t* rec_vis, long i, const uint64_t* vis) {
    if (S.NL > 64) reinterpret_cast<ulonglong2*>(rec_vis)[i] = make_ulonglong2(vis[0], vis[1]);
    else rec_vis[i] = vis[0];
}

// Camera samples [q0, q0 + the block map's count) of each item.  records_only
// (a tile of the adjoint's recomputed records): trace the camera ray and the
// shadow rays, write the hit records of the tile at q - q0, and shade
// nothing.  Otherwise: the forward render, writing the records of samples
// q >= it.rec_from at q - it.rec_from (the whole image when it fits the
// record buffer, else its last tile; it.rec_from < 0: none).
template <bool ENV>
__global__ void __launch_bounds__(RT_THREADS, FR_FWD_MIN_BLOCKS) k_forward(const DevItem* items, BlockMap map,
                                                                           long q0, int records_only) {
    __shared__ RtShared sh;
    FR_STACK_DECL
    const int item = item_of_block(map);
    const DevItem& it = items[item];
    const DevScene& S = it.S;
    const DevParams& P = it.P;
    float* image = it.image;
    int32_t* tri_rec = it.tri_rec;
    uint64_t* mask_rec = it.mask_rec;
    const uint32_t iteration = it.iteration, face = it.face;
    const long total = (long)S.W * S.H * S.spp;
    const long ql = (long)(blockIdx.x - map.block0[item]) * RT_THREADS + threadIdx.x;
    const long q = q0 + ql;
    const bool valid = q < total;
    const int pixel = valid ? (int)(q / S.spp) : 0;
    const int s = valid ? (int)(q % S.spp) : 0;
    const Sampler smp{make_uint2(S.seed, FR_STREAM_PRIMARY), (uint32_t)pixel, (uint32_t)s, iteration, face};
    const float2 jit = smp.pair(0);
    SampleState ss;
    uint64_t vis[2];
    RayStats rs;
    visibility_at<ENV>(S, P, valid, (float)(pixel % S.W) + jit.x, (float)(pixel / S.W) + jit.y, smp, 2, sh,
                       my_stack(sh), ss, vis, rs);
    if (records_only) {                                 // launch-uniform
        flush_stats(S.counters + 3, rs);                // the adjoint's rays
        if (valid) {
            it.rec_tri[ql] = ss.tri;
            if (ss.hit) store_vis(S, it.rec_vis, ql, vis);
        }
        return;
    }
    const float3 Lo = shade_visible<ENV>(S, P, smp, 2, ss, vis);
    flush_stats(S.counters + 0, rs);
    if (valid && tri_rec) tri_rec[q] = ss.tri;
    if (valid && mask_rec) {
        mask_rec[2 * q] = vis[0];
        mask_rec[2 * q + 1] = vis[1];
    }
    // (a sample that misses the face has no visibility to record: nothing reads it)
    if (valid && it.rec_from >= 0 && q >= it.rec_from) {
        it.rec_tri[q - it.rec_from] = ss.tri;
        if (ss.hit) store_vis(S, it.rec_vis, q - it.rec_from, vis);
    }
    // per-pixel mean: lanes of one pixel summed in a fixed tree order; above
    // 32 spp the warps of one pixel (within this block) add their sums in warp
    // order, and at 256 spp the two blocks of a pixel add their partials onto
    // the zeroed image (two addends onto zero: exact in either order), so the
    // image does not depend on scheduling
    const int width = S.spp < 32 ? S.spp : 32;
    const float rx = group_sum(Lo.x, width), ry = group_sum(Lo.y, width), rz = group_sum(Lo.z, width);
    const float inv = 1.0f / (float)S.spp;
    if (S.spp <= 32) {
        if (valid && (s % width) == 0) {
            float* px = image + 3 * (size_t)pixel;
            px[0] = rx * inv; px[1] = ry * inv; px[2] = rz * inv;
        }
    } else {                                            // block-uniform (one item per block)
        __shared__ float wsum[RT_WARPS][3];
        const int warp = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            wsum[warp][0] = rx; wsum[warp][1] = ry; wsum[warp][2] = rz;
        }
        __syncthreads();
        const int wpp = min(S.spp >> 5, RT_WARPS);     // warps of this pixel in this block
        if (valid && (threadIdx.x & (32 * wpp - 1)) == 0) {
            float a = 0.0f, b = 0.0f, c = 0.0f;
            for (int k = warp; k < warp + wpp; ++k) {
                a += wsum[k][0]; b += wsum[k][1]; c += wsum[k][2];
            }
            float* px = image + 3 * (size_t)pixel;
            if (S.spp <= RT_THREADS) {
                px[0] = a * inv; px[1] = b * inv; px[2] = c * inv;
            } else {
                atomicAdd(&px[0], a * inv); atomicAdd(&px[1], b * inv); atomicAdd(&px[2], c * inv);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
FR_D void block_acc_init(int n) {
    for (int i = threadIdx.x; i < RT_WARPS * n; i += RT_THREADS) acc_dyn[i] = 0.0f;
    __syncthreads();
}

// per-warp partials [from, from + count) of rows of n_acc, summed in warp
// order, then one fixed-point add per value into out[0, count)
FR_D void block_acc_flush(int n_acc, int from, int count, fix64* out) {
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += RT_THREADS) {
        double s = 0.0;
        for (int w = 0; w < RT_WARPS; ++w) s += (double)acc_dyn[w * n_acc + from + i];
        if (s != 0.0) atomicAdd(&out[i], (fix64)to_fix_d(s));
    }
}

FR_D void add_vec(fix64* base, int vertex, float3 g, bool on) {
    if (!on) return;
    fix_add(&base[3 * vertex + 0], g.x);
    fix_add(&base[3 * vertex + 1], g.y);
    fix_add(&base[3 * vertex + 2], g.z);
}

// Warp-aggregated scatter of a per-vertex 3-vector (lanes hitting the same
// vertex combine first).
FR_D void scatter_vertex(fix64* base, int vertex, float3 g, bool on) {
    const unsigned act = __ballot_sync(FULL, on);
    if (!on) return;
    fix64* const a[3] = {&base[3 * vertex + 0], &base[3 * vertex + 1], &base[3 * vertex + 2]};
    const float v[3] = {g.x, g.y, g.z};
    warp_agg_add_n<3>(a, v, (uint32_t)vertex, act);
}

// Is edge E (first vertex A) a silhouette seen from y?  Boundary edges always
// are; an interior edge is when y lies strictly on different sides of its two
// faces' planes (FP64).
FR_D bool silhouette_from(const DevScene& S, int4 E, float3 A, float3 y) {
    if (E.w < 0) return true;
    const int4 ff[2] = {S.faces[E.z], S.faces[E.w]};
    const double yx = (double)y.x - A.x, yy = (double)y.y - A.y, yz = (double)y.z - A.z;
    int sg[2];
    for (int k = 0; k < 2; ++k) {
        const float4 p0 = S.v[ff[k].x], p1 = S.v[ff[k].y], p2 = S.v[ff[k].z];
        const double e1x = (double)p1.x - p0.x, e1y = (double)p1.y - p0.y, e1z = (double)p1.z - p0.z;
        const double e2x = (double)p2.x - p0.x, e2y = (double)p2.y - p0.y, e2z = (double)p2.z - p0.z;
        const double nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
        const double dd = nx * yx + ny * yy + nz * yz;
        sg[k] = (dd > 0.0) - (dd < 0.0);
    }
    return sg[0] != sg[1];
}

// Shadow-boundary sample for a light at infinity: the boundary lies on the
// sphere of directions, w(t) = (p(t) - y) / |p(t) - y| for the edge point
// p(t) = A + t (B - A).  Its normal velocity is m . (dp - dy) / |p - y| with m
// the curve's unit normal tangent to the sphere, and arc length |dw/dt| dt.
FR_D void shadow_edge_env(const DevScene& S, const DevParams& P, const LightDev& L, const SampleState& ss, int4 E,
                          float3 A, float3 B, float t, int Sj, float3 w, float3& gy, fix64* d_v, Stack st,
                          RayStats& rs) {
    const float3 e = B - A;
    const float3 q = A + e * t - ss.y;
    const float r2 = dot(q, q);
    if (!(r2 > 0.0f)) return;
    const float inv_r = 1.0f / sqrtf(r2);
    const float3 wv = q * inv_r;
    int row, col;
    env_texel_of(wv, L.env, row, col);
    if (!env_block_has(L, row, col)) return;
    if (!silhouette_from(S, E, A, ss.y)) return;
    const float3 h = light_h_env<false>(S.flags, wv, ss, f3(0, 0, 0), nullptr);
    if (h.x == 0.0f && h.y == 0.0f && h.z == 0.0f) return;
    const float3 tan = (e - wv * dot(wv, e)) * inv_r;     // dw/dt
    const float tl = length(tan);
    if (!(tl > 0.0f)) return;
    const float3 m = cross(wv, tan) * (1.0f / tl);
    float3 wp = wv + m * SHADOW_EPS, wm = wv - m * SHADOW_EPS;
    wp = wp * (1.0f / length(wp));
    wm = wm * (1.0f / length(wm));
    const bool vp = !trace_any(S, ray_setup(ss.y, wp), SHADOW_EPS, INFINITY, ss.slot, st, rs);
    const bool vm = !trace_any(S, ray_setup(ss.y, wm), SHADOW_EPS, INFINITY, ss.slot, st, rs);
    const float dV = (float)vp - (float)vm;
    if (dV == 0.0f) return;
    const float3 Le = env_radiance(P, row * L.env + col);
    const float C = -dV * (float)S.NL * (float)Sj * tl * (w.x * h.x * Le.x + w.y * h.y * Le.y + w.z * h.z * Le.z);
    const float3 gp = m * (C * inv_r);
    gy -= gp;
    add_vec(d_v, E.x, gp * (1.0f - t), true);
    add_vec(d_v, E.y, gp * t, true);
}

// One shadow-boundary edge sample at this lane's shading point (edge sampling
// for visibility of the emitter, Sec. 4).  Adds C * dz/dy . m to gy and
// scatters the edge-vertex terms.  Returns nothing; inactive lanes do nothing.
template <bool ENV>
FR_D void shadow_edge(const DevScene& S, const DevParams& P, const EdgeLists& EL, const SampleState& ss,
                      const Sampler& sm2, float3 w, float3& gy, fix64* d_v, fix64* small, Stack st, RayStats& rs) {
    const uint4 blk = sm2.block(0);
    const float u0 = u24(blk.x), u1 = u24(blk.y), u2 = u24(blk.z);
    const int j = min((int)(u0 * (float)S.NL), S.NL - 1);
    const int Sj = EL.light_count[j];
    if (Sj == 0) return;
    const int eid = EL.light_list[(size_t)j * S.E + min((int)(u1 * (float)Sj), Sj - 1)];
    const int4 E = EL.edges[eid];
    const int4 fc = S.faces[ss.tri];
    const bool ha = (E.x == fc.x || E.x == fc.y || E.x == fc.z);
    const bool hb = (E.y == fc.x || E.y == fc.y || E.y == fc.z);
    if (ha && hb) return;
    const float3 A = xyz(S.v[E.x]), B = xyz(S.v[E.y]);
    // the emitter-plane projection first: it rejects almost every sample in
    // FP32, before the FP64 silhouette test (all conditions must hold, so the
    // order does not change which samples count)
    const LightDev& L = S.lights[j];
    const float t = u2;
    if (ENV && L.type == FR_LIGHT_ENV_D) {
        shadow_edge_env(S, P, L, ss, E, A, B, t, Sj, w, gy, d_v, st, rs);
        return;
    }
    const float3 e = B - A;
    const float3 pe = A + e * t;
    const float3 q = pe - ss.y;
    const float den = dot(q, L.n);
    const float num = dot(L.c - ss.y, L.n);
    if (den == 0.0f) return;
    const float sc = num / den;
    if (!(sc > 1.0f)) return;
    const float3 z = ss.y + q * sc;
    if (!inside_emitter(L, z)) return;
    if (!silhouette_from(S, E, A, ss.y)) return;
    const float3 h = light_h<false>(S.flags, L, z, ss, f3(0, 0, 0), nullptr, nullptr);
    if (h.x == 0.0f && h.y == 0.0f && h.z == 0.0f) return;
    const float3 tan = (e - q * (dot(e, L.n) / den)) * sc;
    const float tl = length(tan);
    if (!(tl > 0.0f)) return;
    const float3 m = cross(L.n, tan) * (1.0f / tl);
    const float3 zp = z + m * SHADOW_EPS, zm = z - m * SHADOW_EPS;
    const bool vp = !trace_any(S, ray_setup(ss.y, zp - ss.y), SHADOW_EPS, 1.0f - SHADOW_EPS, ss.slot, st, rs);
    const bool vm = !trace_any(S, ray_setup(ss.y, zm - ss.y), SHADOW_EPS, 1.0f - SHADOW_EPS, ss.slot, st, rs);
    const float dV = (float)vp - (float)vm;
    if (dV == 0.0f) return;
    const float3 I = intensity(S, P, j);
    const float scale = -dV * (float)S.NL * (float)Sj * tl;
    const float C = scale * (w.x * h.x * I.x + w.y * h.y * I.y + w.z * h.z * I.z);
    const float mq = dot(m, q);
    const float3 g_y = m * (1.0f - sc) + L.n * (mq * (sc - 1.0f) / den);
    const float3 g_p = m * sc - L.n * (mq * sc / den);
    gy += g_y * C;
    add_vec(d_v, E.x, g_p * (C * (1.0f - t)), true);
    add_vec(d_v, E.y, g_p * (C * t), true);
    if (S.stage) {
        // a stage light moves under the boundary: the boundary's normal velocity
        // relative to the emitter's own points (the plane moves only with d)
        const StageFrame F = stage_frame(S, P, j);
        const float vd = mq * dot(L.n, L.c - F.C) / (F.d * den) - dot(m, z - F.C) / F.d;
        const float va = -dot(m, z - F.P) / (2.0f * F.a);
        const float vp0 = -F.d * dot(m, F.dA), vp1 = -F.d * dot(m, F.dB);
        fix64* g = small + FR_GEO_OFF + 4 * j;
        fix_add(&g[0], C * vd);
        fix_add(&g[1], C * va);
        fix_add(&g[2], C * vp0);
        fix_add(&g[3], C * vp1);
    }
}

// Camera samples [q0, q0 + the block map's count) of each item.  RECORDED:
// every item of the launch has the hit records of these samples in its record
// buffer at q - q0 (written by the forward of the same step, or by the
// records-only forward pass of this tile), so the camera and shadow
// traversals are compiled out (a smaller kernel); otherwise each item re-traces
// unless its forward recorded the whole image (q0 = 0).
// Chain rule from a camera sample's shading state back to its hit triangle's
// vertices and vertex normals and to the camera ray direction d: given the
// gradients w.r.t. the shading normal ns = m / |m| (m = sum b_k n_k), the view
// direction o = -d / |d|, the hit point y = sum b_k v_k and the barycentrics
// (gb, e.g. from texture coordinates), with the barycentrics of the ray from
// the camera centre along d (Moller-Trumbore form).
struct HitChain {
    float3 gv[3], gn[3], gd;
};

FR_D HitChain hit_chain(float3 v0, float3 v1, float3 v2, float3 n0, float3 n1, float3 n2, float3 d, float3 g_ns,
                        float3 g_o, float3 gy, float gb0, float gb1, float gb2) {
    HitChain h;
    // intersection quantities (ray origin at the camera)
    const float3 e1 = v1 - v0, e2 = v2 - v0, sv = -v0;
    const float3 pv = cross(d, e2), qv = cross(sv, e1);
    const float det = dot(e1, pv), inv_det = __fdividef(1.0f, det);
    const float b1 = dot(sv, pv) * inv_det, b2 = dot(d, qv) * inv_det, b0 = 1.0f - b1 - b2;
    // shading normal ns = m / |m|
    const float3 mm = n0 * b0 + n1 * b1 + n2 * b2;
    const float inv_m = rsqrtf(dot(mm, mm));
    const float3 nsh = mm * inv_m;
    const float3 gm = (g_ns - nsh * dot(nsh, g_ns)) * inv_m;
    h.gn[0] = gm * b0; h.gn[1] = gm * b1; h.gn[2] = gm * b2;
    gb0 += dot(n0, gm); gb1 += dot(n1, gm); gb2 += dot(n2, gm);
    // y = sum b_k v_k
    float3 gv0 = gy * b0, gv1 = gy * b1, gv2 = gy * b2;
    gb0 += dot(v0, gy); gb1 += dot(v1, gy); gb2 += dot(v2, gy);
    // view direction o = -d / |d|
    const float inv_d = rsqrtf(dot(d, d));
    const float3 od = -d * inv_d;
    float3 gd = -(g_o - od * dot(od, g_o)) * inv_d;
    // barycentrics from the intersection
    const float G1 = gb1 - gb0, G2 = gb2 - gb0;
    const float gsp = G1 * inv_det, gdq = G2 * inv_det, gdet = -(G1 * b1 + G2 * b2) * inv_det;
    float3 gs = pv * gsp;
    float3 gp = sv * gsp + e1 * gdet;
    gd += qv * gdq;
    const float3 gq = d * gdq;
    float3 ge1 = pv * gdet;
    gs += cross(e1, gq);
    ge1 += cross(gq, sv);
    gd += cross(e2, gp);
    const float3 ge2 = cross(gp, d);
    h.gv[0] = gv0 + (-gs - ge1 - ge2);
    h.gv[1] = gv1 + ge1;
    h.gv[2] = gv2 + ge2;
    h.gd = gd;
    return h;
}

template <bool RECORDED, bool ENV>
__global__ void __launch_bounds__(RT_THREADS, RECORDED ? FR_ADJ_REC_MIN_BLOCKS : FR_ADJ_MIN_BLOCKS)
    k_adjoint(const DevItem* items, BlockMap map, long q0) {
    __shared__ RtShared sh;
    FR_STACK_DECL
    const int item = item_of_block(map);
    const DevItem& it = items[item];
    const DevScene& S = it.S;
    const DevParams& P = it.P;
    const DevGrads& G = it.G;
    const EdgeLists& EL = it.EL;
    const float* adj_image = it.adj;
    const uint32_t iteration = it.iteration, face = it.face;
    const bool stage = S.stage != nullptr;                      // lights built from (d, a, p)
    const int n_acc = 1 + 3 * S.NL + (stage ? 4 * S.NL : 0);
    block_acc_init(n_acc);
    const long total = (long)S.W * S.H * S.spp;
    const long ql = (long)(blockIdx.x - map.block0[item]) * RT_THREADS + threadIdx.x;   // record index
    const long qi = q0 + ql;
    bool valid = qi < total;
    const int pixel = valid ? (int)(qi / S.spp) : 0;
    const int s = valid ? (int)(qi % S.spp) : 0;
    float3 w = f3(0.0f, 0.0f, 0.0f);
    if (valid) {
        const float inv = 1.0f / (float)S.spp;
        w = f3(adj_image[3 * (size_t)pixel] * inv, adj_image[3 * (size_t)pixel + 1] * inv,
               adj_image[3 * (size_t)pixel + 2] * inv);
        if (w.x == 0.0f && w.y == 0.0f && w.z == 0.0f) valid = false;
    }
    const Sampler smp{make_uint2(S.seed, FR_STREAM_PRIMARY), (uint32_t)pixel, (uint32_t)s, iteration, face};
    const float2 jit = smp.pair(0);
    const float sx = (float)(pixel % S.W) + jit.x, sy = (float)(pixel / S.W) + jit.y;
    SampleState ss;
    RayStats rs;
    // the forward of a fused step may have recorded this sample's hit and
    // shadow visibility; otherwise both are re-traced with the same counters
    const bool recorded = RECORDED || it.rec_full;             // block-uniform
    primary_state<!RECORDED, false>(S, P, valid, sx, sy, my_stack(sh), ss, rs,
                                    recorded ? (valid ? it.rec_tri[ql] : -1) : REC_TRACE);
    // the visibility words of every 64-light chunk (recorded, or re-traced with
    // the forward's counters) before the material fetch, so that the material
    // is not live across the shadow traversal
    uint64_t vis_w[2] = {0ull, 0ull};
    if (!(S.flags & FR_FLAG_FLAT_D)) {
        for (int j0 = 0; j0 < S.NL; j0 += 64) {                // warp-uniform
            if (recorded)
                vis_w[j0 >> 6] = (valid && ss.hit) ? it.rec_vis[vis_words(S) * ql + (j0 >> 6)] : 0ull;
            else
                vis_w[j0 >> 6] = shadow_mask<ENV>(S, ss, smp, 2, sh.wq[threadIdx.x >> 5], my_stack(sh), rs, j0);
        }
    }
    sample_material(S, P, ss);
    const bool interior = !(S.flags & FR_FLAG_NO_INTERIOR_D);
    ShadeAdj g;
    g.n = g.l = g.o = g.c = g.s = f3(0.0f, 0.0f, 0.0f);
    g.r = 0.0f;
    float3 gy = f3(0.0f, 0.0f, 0.0f);
    if (S.flags & FR_FLAG_FLAT_D) {
        if (ss.hit && interior) g.c = w;
    } else {
        DimCache dc;
        uint64_t vis = 0ull;
        for (int j = 0; j < S.NL; ++j) {                       // warp-uniform loop
            if ((j & 63) == 0) vis = vis_w[j >> 6];            // lights in chunks of 64
            if (ENV && S.lights[j].type == FR_LIGHT_ENV_D) {    // warp-uniform
                // a light at infinity: the radiance gradient goes to the sampled texel
                float3 ge = f3(0.0f, 0.0f, 0.0f);
                int texel = 0;
                if (interior && ss.hit && ((vis >> (j & 63)) & 1ull)) {
                    const float2 u = dc.pair(smp, 2 + 2 * j);
                    const EnvDir ed = env_sample(S.lights[j], u.x, u.y);
                    const float3 E = env_radiance(P, ed.texel);
                    const float3 h = light_h_env<true>(S.flags, ed.w, ss, f3(w.x * E.x, w.y * E.y, w.z * E.z) * ed.weight, &g);
                    ge = f3(w.x * h.x, w.y * h.y, w.z * h.z) * ed.weight;
                    texel = ed.texel;
                }
                const bool add = ge.x != 0.0f || ge.y != 0.0f || ge.z != 0.0f;
                const unsigned act = __ballot_sync(FULL, add);
                if (add) {
                    fix64* const a[3] = {&G.small[FR_ENV_OFF + 3 * texel], &G.small[FR_ENV_OFF + 3 * texel + 1],
                                         &G.small[FR_ENV_OFF + 3 * texel + 2]};
                    const float v[3] = {ge.x, ge.y, ge.z};
                    warp_agg_add_n<3>(a, v, (uint32_t)texel, act);
                }
                continue;
            }
            float3 gI = f3(0.0f, 0.0f, 0.0f);
            float gl4[4] = {0.0f, 0.0f, 0.0f, 0.0f};            // d, a, p0, p1 of light j
            if (interior && ss.hit && ((vis >> (j & 63)) & 1ull)) {
                const LightDev& L = S.lights[j];
                const float2 u = dc.pair(smp, 2 + 2 * j);
                const float3 z = light_point(L, u.x, u.y);
                const float3 I = intensity(S, P, j);
                const float3 gh = f3(w.x * I.x, w.y * I.y, w.z * I.z) * L.area;
                float3 gz = f3(0.0f, 0.0f, 0.0f);
                const float3 h = light_h<true>(S.flags, L, z, ss, gh, &g, &gy, stage ? &gz : nullptr);
                gI = f3(w.x * h.x, w.y * h.y, w.z * h.z) * (L.area * L.scale);
                if (stage) {
                    // the sample point moves with the light; area * d^2/a = F d^4
                    const StageFrame F = stage_frame(S, P, j);
                    const float gIi = gI.x * __ldg(&P.light_i[3 * j]) + gI.y * __ldg(&P.light_i[3 * j + 1]) +
                                      gI.z * __ldg(&P.light_i[3 * j + 2]);
                    gl4[0] = (dot(gz, z - F.C) + 4.0f * gIi) / F.d;
                    gl4[1] = dot(gz, z - F.P) / (2.0f * F.a);
                    gl4[2] = F.d * dot(gz, F.dA);
                    gl4[3] = F.d * dot(gz, F.dB);
                }
            }
            // a light no lane of the warp saw adds exact zeros: skip its reductions
            const bool any = __any_sync(0xffffffffu, gI.x != 0.0f || gI.y != 0.0f || gI.z != 0.0f ||
                                                         gl4[0] != 0.0f || gl4[1] != 0.0f || gl4[2] != 0.0f ||
                                                         gl4[3] != 0.0f);
            if (any) {
                const float sx_ = warp_sum(gI.x), sy_ = warp_sum(gI.y), sz_ = warp_sum(gI.z);
                if ((threadIdx.x & 31) == 0) {
                    float* wa = acc_dyn + (threadIdx.x >> 5) * n_acc;
                    wa[1 + 3 * j] = sx_;
                    wa[1 + 3 * j + 1] = sy_;
                    wa[1 + 3 * j + 2] = sz_;
                }
                if (stage) {                                   // block-uniform
                    float sg[4];
                    for (int q = 0; q < 4; ++q) sg[q] = warp_sum(gl4[q]);
                    if ((threadIdx.x & 31) == 0) {
                        float* wa = acc_dyn + (threadIdx.x >> 5) * n_acc + 1 + 3 * S.NL + 4 * j;
                        for (int q = 0; q < 4; ++q) wa[q] = sg[q];
                    }
                }
            }
        }
        if (!(S.flags & FR_FLAG_NO_SHADOW_EDGE_D) && ss.hit && ss.lit) {
            const Sampler sm2{make_uint2(S.seed, FR_STREAM_EDGE_SHADOW), (uint32_t)pixel, (uint32_t)s, iteration, face};
            shadow_edge<ENV>(S, P, EL, ss, sm2, w, gy, G.d_v, G.small, my_stack(sh), rs);
        }
    }
    // ---- chain rule back to the hit triangle, its normals and the camera ----
    const bool on = ss.hit;
    int4 fc = make_int4(0, 0, 0, 0);
    float gfocal = 0.0f;
    float3 gv0 = f3(0, 0, 0), gv1 = f3(0, 0, 0), gv2 = f3(0, 0, 0);
    float3 gn0 = f3(0, 0, 0), gn1 = f3(0, 0, 0), gn2 = f3(0, 0, 0);
    float gtex[7] = {0, 0, 0, 0, 0, 0, 0};
    if (on) {
        fc = S.faces[ss.tri];
        const float3 v0 = xyz(S.v[fc.x]), v1 = xyz(S.v[fc.y]), v2 = xyz(S.v[fc.z]);
        const float3 n0 = xyz(S.vn[fc.x]), n1 = xyz(S.vn[fc.y]), n2 = xyz(S.vn[fc.z]);
        const float2 t0 = S.uv[fc.x], t1 = S.uv[fc.y], t2 = S.uv[fc.z];
        // textures: value gradients and d/d(uv)
        float gu = 0.0f, gvv = 0.0f;
        for (int ch = 0; ch < 3; ++ch) {
            float du, dv;
            tap_fetch(P.diffuse, 3, ch, ss.tap, S.M, &du, &dv);
            const float gc = comp(g.c, ch);
            gu += gc * du; gvv += gc * dv;
            tap_fetch(P.specular, 3, ch, ss.tap, S.M, &du, &dv);
            const float gs = comp(g.s, ch);
            gu += gs * du; gvv += gs * dv;
            gtex[ch] = gc;
            gtex[3 + ch] = gs;
        }
        {
            float du, dv;
            tap_fetch(P.roughness, 1, 0, ss.tap, S.M, &du, &dv);
            gu += g.r * du; gvv += g.r * dv;
            gtex[6] = g.r;
        }
        const float gb0 = gu * t0.x + gvv * t0.y, gb1 = gu * t1.x + gvv * t1.y, gb2 = gu * t2.x + gvv * t2.y;
        const HitChain hc = hit_chain(v0, v1, v2, n0, n1, n2, ss.d, g.n, g.o, gy, gb0, gb1, gb2);
        gv0 = hc.gv[0]; gv1 = hc.gv[1]; gv2 = hc.gv[2];
        gn0 = hc.gn[0]; gn1 = hc.gn[1]; gn2 = hc.gn[2];
        // d = ((sx - W/2)/f, -(sy - H/2)/f, -1)
        const float f = P.focal[0];
        gfocal = -(hc.gd.x * ss.d.x + hc.gd.y * ss.d.y) / f;
    }
    // vertex position and normal gradients, warp-aggregated by vertex
    {
        const unsigned act = __ballot_sync(FULL, on);
        if (on) {
            const int vx[3] = {fc.x, fc.y, fc.z};
            const float3 gvv[3] = {gv0, gv1, gv2}, gnn[3] = {gn0, gn1, gn2};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                fix64* const a[6] = {&G.d_v[3 * vx[k]], &G.d_v[3 * vx[k] + 1], &G.d_v[3 * vx[k] + 2],
                                     &G.d_n[3 * vx[k]], &G.d_n[3 * vx[k] + 1], &G.d_n[3 * vx[k] + 2]};
                const float v[6] = {gvv[k].x, gvv[k].y, gvv[k].z, gnn[k].x, gnn[k].y, gnn[k].z};
                warp_agg_add_n<6>(a, v, (uint32_t)vx[k], act);
            }
        }
    }
    // bilinear texture scatter (4 taps), warp-aggregated by texel: the 3 diffuse,
    // 3 specular and 1 roughness channels of a tap together
    const bool tex_on = on && interior;
    const size_t M2 = (size_t)S.M * S.M;
    const int taps[4] = {ss.tap.i00, ss.tap.i10, ss.tap.i01, ss.tap.i11};
    const float tw[4] = {(1.0f - ss.tap.fx) * (1.0f - ss.tap.fy), ss.tap.fx * (1.0f - ss.tap.fy),
                         (1.0f - ss.tap.fx) * ss.tap.fy, ss.tap.fx * ss.tap.fy};
    {
        const unsigned act = __ballot_sync(FULL, tex_on);
        if (tex_on) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const size_t t3 = 3 * (size_t)taps[k];
                fix64* const a[7] = {&G.tex[t3], &G.tex[t3 + 1], &G.tex[t3 + 2], &G.tex[3 * M2 + t3],
                                     &G.tex[3 * M2 + t3 + 1], &G.tex[3 * M2 + t3 + 2], &G.tex[6 * M2 + taps[k]]};
                const float v[7] = {gtex[0] * tw[k], gtex[1] * tw[k], gtex[2] * tw[k], gtex[3] * tw[k],
                                    gtex[4] * tw[k], gtex[5] * tw[k], gtex[6] * tw[k]};
                warp_agg_add_n<7>(a, v, (uint32_t)taps[k], act);
            }
        }
    }
    const float gf_w = warp_sum(gfocal);
    if ((threadIdx.x & 31) == 0) acc_dyn[(threadIdx.x >> 5) * n_acc] = gf_w;
    flush_stats(S.counters + 3, rs);
    block_acc_flush(n_acc, 0, 1 + 3 * S.NL, G.small);
    if (stage) block_acc_flush(n_acc, 1 + 3 * S.NL, 4 * S.NL, G.small + FR_GEO_OFF);
}

// ---------------------------------------------------------------------------
// processing order of the primary-edge samples
// ---------------------------------------------------------------------------
// Each primary-edge sample picks a random silhouette edge, so consecutive
// samples land far apart and a warp's camera and shadow rays diverge.  Within
// each chunk of EDGE_CHUNK consecutive samples this kernel sorts the samples
// by the image position their edge point projects to, in Morton order
// (samples that cannot contribute last), with a bitonic sort; k_edge_primary
// then processes them in that order.  The set of samples, and so the estimate, is unchanged;
// the order is a deterministic function of the inputs.
constexpr int EDGE_CHUNK = 4096;                   // 12 bits of in-chunk index
constexpr int EDGE_SORT_THREADS = 1024;

// Bitonic compare-exchange seen from element i (partner i ^ j) of the
// sequence stage (k, j): the lower index of an ascending pair keeps the
// smaller key, as does the upper index of a descending pair.
__device__ __forceinline__ uint32_t bitonic_pick(uint32_t mine, uint32_t other, int i, int j, int k) {
    const bool keep_min = ((i & j) == 0) == ((i & k) == 0);
    return keep_min ? min(mine, other) : max(mine, other);
}

// Thread t holds keys 4t .. 4t + 3 in registers: the stages with j <= 2 run
// inside the thread, those with 4 <= j <= 64 between the lanes of a warp
// (partner lane t ^ j / 4), and only those with j >= 128 go through shared
// memory (15 of the 78 stages for 4096 keys).  The keys are distinct, so the
// result is the one sorted order.
__global__ void __launch_bounds__(EDGE_SORT_THREADS) k_edge_order(const DevItem* items) {
    static_assert(EDGE_CHUNK == 4 * EDGE_SORT_THREADS, "four keys per thread");
    __shared__ uint4 key4[EDGE_SORT_THREADS];
    uint32_t* key = reinterpret_cast<uint32_t*>(key4);
    const DevItem& it = items[blockIdx.y];
    const DevScene& S = it.S;
    const long n_edge = (S.flags & FR_FLAG_NO_PRIMARY_EDGE_D) ? 0 : (long)S.W * S.H * S.edge_spp;
    const long base = (long)blockIdx.x * EDGE_CHUNK;
    if (base >= n_edge || !it.edge_perm) return;         // block-uniform
    const int Sn = *it.EL.prim_count;
    const float f = it.P.focal[0];
    const int t = threadIdx.x;
    uint32_t r[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int q = 4 * t + m;
        const long e = base + q;
        uint32_t k20 = 0xFFFFFu;                           // no contribution possible: last
        if (e < n_edge && Sn > 0) {
            const Sampler smp{make_uint2(S.seed, FR_STREAM_EDGE_PRIMARY), (uint32_t)e, 0u, it.iteration, it.face};
            const uint4 blk = smp.block(0);
            const int4 E = it.EL.edges[it.EL.prim_list[min((int)(u24(blk.x) * (float)Sn), Sn - 1)]];
            const float3 A = xyz(S.v[E.x]), B = xyz(S.v[E.y]);
            const float3 p = A + (B - A) * u24(blk.y);
            if (p.z < 0.0f) {
                const float X = 0.5f * S.W + f * p.x / -p.z, Y = 0.5f * S.H - f * p.y / -p.z;
                if (X >= 0.0f && X < (float)S.W && Y >= 0.0f && Y < (float)S.H) {
                    // Morton order of the point on a 1024 x 1024 grid over the image, 20
                    // bits (row-major pixel order puts the left and right silhouettes of a
                    // row side by side: measured 6% slower in k_edge_primary)
                    const uint32_t gx = min(1023u, (uint32_t)(X * (1024.0f / (float)S.W)));
                    const uint32_t gy = min(1023u, (uint32_t)(Y * (1024.0f / (float)S.H)));
                    uint32_t m = 0;
                    for (int bit = 0; bit < 10; ++bit)
                        m |= (((gx >> bit) & 1u) << (2 * bit)) | (((gy >> bit) & 1u) << (2 * bit + 1));
                    k20 = min(m, 0xFFFFEu);
                }
            }
        }
        r[m] = (k20 << 12) | (uint32_t)q;                  // the index makes keys distinct
    }
    for (int k = 2; k <= EDGE_CHUNK; k <<= 1) {            // bitonic sort, ascending
        int j = k >> 1;
        if (j >= 128) {                                    // across warps: shared memory
            key4[t] = make_uint4(r[0], r[1], r[2], r[3]);
            __syncthreads();
            for (; j >= 128; j >>= 1) {
                for (int i = t; i < EDGE_CHUNK; i += EDGE_SORT_THREADS) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const uint32_t a = key[i], b = key[ixj];
                        if ((a > b) == ((i & k) == 0)) {
                            key[i] = b;
                            key[ixj] = a;
                        }
                    }
                }
                __syncthreads();
            }
            const uint4 v = key4[t];
            r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
            __syncthreads();                               // before key4 is written again
        }
        for (; j >= 4; j >>= 1) {                          // within the warp
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const uint32_t o = __shfl_xor_sync(FULL, r[m], j >> 2);
                r[m] = bitonic_pick(r[m], o, 4 * t + m, j, k);
            }
        }
        // within the thread: j = 2 (when k >= 4), then j = 1
        if (k >= 4) {
            const uint32_t n0 = bitonic_pick(r[0], r[2], 4 * t, 2, k), n1 = bitonic_pick(r[1], r[3], 4 * t + 1, 2, k);
            const uint32_t n2 = bitonic_pick(r[2], r[0], 4 * t + 2, 2, k), n3 = bitonic_pick(r[3], r[1], 4 * t + 3, 2, k);
            r[0] = n0; r[1] = n1; r[2] = n2; r[3] = n3;
        }
        const uint32_t n0 = bitonic_pick(r[0], r[1], 4 * t, 1, k), n1 = bitonic_pick(r[1], r[0], 4 * t + 1, 1, k);
        const uint32_t n2 = bitonic_pick(r[2], r[3], 4 * t + 2, 1, k), n3 = bitonic_pick(r[3], r[2], 4 * t + 3, 1, k);
        r[0] = n0; r[1] = n1; r[2] = n2; r[3] = n3;
    }
    // samples past n_edge carry the largest keys, so positions [0, count) hold
    // exactly this chunk's samples
    const int count = (int)min((long)EDGE_CHUNK, n_edge - base);
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (4 * t + m < count) it.edge_perm[base + 4 * t + m] = (int)(base + (r[m] & (EDGE_CHUNK - 1)));
}

// ---------------------------------------------------------------------------
// primary-visibility boundary term: edge samples in screen space
// ---------------------------------------------------------------------------
template <bool ENV>
__global__ void __launch_bounds__(RT_THREADS, FR_EDGE_MIN_BLOCKS) k_edge_primary(const DevItem* items, BlockMap map) {
    __shared__ RtShared sh;
    FR_STACK_DECL
    const int item = item_of_block(map);
    const DevItem& it = items[item];
    const DevScene& S = it.S;
    const DevParams& P = it.P;
    const DevGrads& G = it.G;
    const EdgeLists& EL = it.EL;
    const float* adj_image = it.adj;
    const uint32_t iteration = it.iteration, face = it.face;
    block_acc_init(1);
    const long n_edge = (long)S.W * S.H * S.edge_spp;
    // two lanes per edge sample: the even one evaluates the radiance on the
    // + side of the edge, the odd one on the - side (twice the warps of one
    // lane doing both in turn; the same samples and the same arithmetic)
    const long t0 = (long)(blockIdx.x - map.block0[item]) * RT_THREADS + threadIdx.x;
    const long e0 = t0 >> 1;
    const int side = (int)(t0 & 1);
    bool active = e0 < n_edge;
    // samples are processed in the order k_edge_order chose (same samples, so
    // the same estimate; nearby samples share a warp)
    const long e = (active && it.edge_perm) ? (long)it.edge_perm[e0] : e0;
    const int Sn = *EL.prim_count;
    if (Sn == 0) active = false;
    const Sampler smp{make_uint2(S.seed, FR_STREAM_EDGE_PRIMARY), (uint32_t)(active ? e : 0), 0u, iteration, face};
    const uint4 blk = smp.block(0);
    int4 E = make_int4(0, 0, 0, 0);
    float3 A = f3(0, 0, 0), B = f3(0, 0, 0), p = f3(0, 0, 0);
    float t = 0.0f, X = 0.0f, Y = 0.0f, mx = 0.0f, my = 0.0f, tl = 0.0f, wz = 1.0f;
    float3 adj = f3(0, 0, 0);
    const float f = P.focal[0];
    if (active) {
        E = EL.edges[EL.prim_list[min((int)(u24(blk.x) * (float)Sn), Sn - 1)]];
        A = xyz(S.v[E.x]);
        B = xyz(S.v[E.y]);
        t = u24(blk.y);
        const float3 ed = B - A;
        p = A + ed * t;
        if (!(p.z < 0.0f)) active = false;
        if (active) {
            wz = -p.z;
            X = 0.5f * S.W + f * p.x / wz;
            Y = 0.5f * S.H - f * p.y / wz;
            if (!(X >= 0.0f && X < (float)S.W && Y >= 0.0f && Y < (float)S.H)) active = false;
        }
        if (active) {
            const int pix = (int)floorf(Y) * S.W + (int)floorf(X);
            adj = f3(adj_image[3 * (size_t)pix], adj_image[3 * (size_t)pix + 1], adj_image[3 * (size_t)pix + 2]);
            if (adj.x == 0.0f && adj.y == 0.0f && adj.z == 0.0f) active = false;
            const float tx = f * (ed.x * wz + p.x * ed.z) / (wz * wz);
            const float ty = -f * (ed.y * wz + p.y * ed.z) / (wz * wz);
            tl = sqrtf(tx * tx + ty * ty);
            if (!(tl > 0.0f)) active = false;
            mx = -ty / tl;
            my = tx / tl;
        }
    }
    const float eps = side ? -1e-3f : 1e-3f;
    SampleState ss;
    uint64_t vis[2];
    RayStats rs;
    const float3 L = radiance_at<ENV>(S, P, active, X + eps * mx, Y + eps * my, smp, 4, sh, my_stack(sh), ss, vis, rs);
    const float3 Lo = f3(__shfl_xor_sync(FULL, L.x, 1), __shfl_xor_sync(FULL, L.y, 1), __shfl_xor_sync(FULL, L.z, 1));
    const float3 Lp = side ? Lo : L, Lm = side ? L : Lo;
    if (side) active = false;                          // the even lane adds the pair's term
    flush_stats(S.counters + 6, rs);
    float gf = 0.0f;
    float3 gA = f3(0, 0, 0), gB = f3(0, 0, 0);
    if (active) {
        const float scale = (float)Sn * tl / (float)n_edge;
        const float Wt = -(adj.x * (Lp.x - Lm.x) + adj.y * (Lp.y - Lm.y) + adj.z * (Lp.z - Lm.z)) * scale;
        const float3 gp = f3(Wt * mx * f / wz, -Wt * my * f / wz, Wt * (mx * f * p.x - my * f * p.y) / (wz * wz));
        gA = gp * (1.0f - t);
        gB = gp * t;
        gf = Wt * (mx * p.x - my * p.y) / wz;
        if (Wt == 0.0f) active = false;
    }
    scatter_vertex(G.d_v, E.x, gA, active);
    scatter_vertex(G.d_v, E.y, gB, active);
    const float gw = warp_sum(gf);
    if ((threadIdx.x & 31) == 0) acc_dyn[threadIdx.x >> 5] = gw;
    block_acc_flush(1, 0, 1, G.small);
}

// ---------------------------------------------------------------------------
// boundary of the specular lobe inside triangles: the curve n_s . o = 0
// ---------------------------------------------------------------------------
// The lobe (App. A, Eq. brdf_spec) needs n_s . o > 0 and does not vanish as
// n_s . o -> 0+, so the image jumps on the curve n_s . o = 0 inside
// front-facing triangles whose interpolated normals turn away from the
// camera.  Edge sampling (Sec. 4) meets that curve along image scanlines:
// per pixel row and per pixel column edge_spp lines at uniform offsets (rows
// first).  The rays of a line fill a plane through the camera centre; it cuts
// a triangle along a chord with linear barycentrics, on which q(b) = m(b) .
// (-p(b)) (m = sum b_i n_i, p = sum b_i v_i; q has the sign of n_s . o) is an
// exact quadratic.  A crossing x contributes adj . (L+ - L-) G_theta |n_x| /
// (|grad G|^2 k) on rows (|n_y| on columns), L+- the one-sided limits of the
// radiance there, G = n_s . o at the fixed screen point, grad G its screen
// gradient: the two families' shares n_x^2 and n_y^2 of the line integral,
// each with a bounded weight.

// Candidate triangles: in front of the camera, facing it, and q not of one
// sign over the triangle.  q's degree-2 Bernstein coefficients over the
// triangle (q_ii = -n_i . v_i at the corners, (q_ij + q_ji) / 2 on the edges)
// bound it, so a triangle whose six coefficients share a strict sign has no
// crossing.  Decided in FP64 (so that it agrees with the FP64 crossings
// below); FP32 first, taken whenever it is farther from zero than a generous
// bound on its error (64 u times the sum of the magnitudes of the products).
__device__ bool spec_candidate64(const float4 (&p)[3], const float4 (&q)[3]) {
    double v[3][3], n[3][3];
    for (int i = 0; i < 3; ++i) {
        v[i][0] = p[i].x; v[i][1] = p[i].y; v[i][2] = p[i].z;
        n[i][0] = q[i].x; n[i][1] = q[i].y; n[i][2] = q[i].z;
    }
    if (!(v[0][2] < 0.0 && v[1][2] < 0.0 && v[2][2] < 0.0)) return false;
    const double e1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
    const double e2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
    const double nf[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    if (!(nf[0] * v[0][0] + nf[1] * v[0][1] + nf[2] * v[0][2] < 0.0)) return false;
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            const double qij = -(n[i][0] * v[j][0] + n[i][1] * v[j][1] + n[i][2] * v[j][2]);
            const double qji = -(n[j][0] * v[i][0] + n[j][1] * v[i][1] + n[j][2] * v[i][2]);
            const double b = 0.5 * (qij + qji);
            lo = fmin(lo, b);
            hi = fmax(hi, b);
        }
    return lo <= 0.0 && hi > 0.0;
}

__device__ bool spec_candidate(const DevScene& S, int f) {
    const int4 t = S.faces[f];
    const float4 p[3] = {S.v[t.x], S.v[t.y], S.v[t.z]};
    const float4 q[3] = {S.vn[t.x], S.vn[t.y], S.vn[t.z]};
    if (!(p[0].z < 0.0f && p[1].z < 0.0f && p[2].z < 0.0f)) return false;
    constexpr float U64 = 64.0f * 5.9604645e-8f;
    const float3 e1 = xyz(p[1]) - xyz(p[0]), e2 = xyz(p[2]) - xyz(p[0]), v0 = xyz(p[0]);
    const float3 nf = cross(e1, e2);
    const float3 na = f3(fabsf(e1.y * e2.z) + fabsf(e1.z * e2.y), fabsf(e1.z * e2.x) + fabsf(e1.x * e2.z),
                         fabsf(e1.x * e2.y) + fabsf(e1.y * e2.x));
    const float fv = dot(nf, v0);
    const float fe = U64 * (na.x * fabsf(v0.x) + na.y * fabsf(v0.y) + na.z * fabsf(v0.z));
    if (fv > fe) return false;                                  // faces away, surely
    if (!(fv < -fe)) return spec_candidate64(p, q);
    float lo = INFINITY, hi = -INFINITY, err = 0.0f;
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            const float3 ni = xyz(q[i]), nj = xyz(q[j]), vi = xyz(p[i]), vj = xyz(p[j]);
            const float b = -0.5f * (dot(ni, vj) + dot(nj, vi));
            const float m = 0.5f * (fabsf(ni.x * vj.x) + fabsf(ni.y * vj.y) + fabsf(ni.z * vj.z) +
                                    fabsf(nj.x * vi.x) + fabsf(nj.y * vi.y) + fabsf(nj.z * vi.z));
            lo = fminf(lo, b);
            hi = fmaxf(hi, b);
            err = fmaxf(err, U64 * m);
        }
    if (lo > err || hi < -err) return false;                    // one strict sign, surely
    if (lo < -err && hi > err) return true;
    return spec_candidate64(p, q);
}

constexpr int SPEC_CHUNK = 1024;

// per-chunk candidate counts; each triangle's flag kept for the scatter
__global__ void __launch_bounds__(SPEC_CHUNK) k_spec_count(const DevItem* items) {
    __shared__ int warp_tot[SPEC_CHUNK / 32];
    const DevItem& it = items[blockIdx.y];
    const DevScene& S = it.S;
    const int f = blockIdx.x * SPEC_CHUNK + threadIdx.x;
    const bool want = !(S.flags & (FR_FLAG_NO_SPECULAR_EDGE_D | FR_FLAG_FLAT_D));
    if ((long)blockIdx.x * SPEC_CHUNK >= S.T) return;          // block-uniform
    const bool on = want && f < S.T && spec_candidate(S, f);
    if (f < S.T) it.spec_flag[f] = on ? 1 : 0;
    const unsigned b = __ballot_sync(FULL, on);
    if ((threadIdx.x & 31) == 0) warp_tot[threadIdx.x >> 5] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < SPEC_CHUNK / 32; ++w) t += warp_tot[w];
        it.spec_hist[blockIdx.x] = t;
    }
}

// exclusive scan of the chunk counts: one warp, each lane a run of chunks
__global__ void k_spec_scan(const DevItem* items) {
    const DevItem& it = items[blockIdx.x];
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    const int n_chunks = (it.S.T + SPEC_CHUNK - 1) / SPEC_CHUNK;
    const int per = (n_chunks + 31) / 32, c0 = lane * per, c1 = min(n_chunks, c0 + per);
    int own = 0;
    for (int c = c0; c < c1; ++c) own += it.spec_hist[c];
    int incl = own;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    int run = incl - own;
    for (int c = c0; c < c1; ++c) {
        const int v = it.spec_hist[c];
        it.spec_hist[c] = run;
        run += v;
    }
    if (lane == 31) *it.spec_count = incl;
}

// ordered candidate list (triangle index order) with each candidate's screen
// bounding box (x0, x1, y0, y1), widened by a hair
__global__ void __launch_bounds__(SPEC_CHUNK) k_spec_scatter(const DevItem* items) {
    __shared__ int warp_off[SPEC_CHUNK / 32];
    const DevItem& it = items[blockIdx.y];
    const DevScene& S = it.S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int f = blockIdx.x * SPEC_CHUNK + threadIdx.x;
    if ((long)blockIdx.x * SPEC_CHUNK >= S.T) return;          // block-uniform
    const bool on = f < S.T && it.spec_flag[f];
    const unsigned b = __ballot_sync(FULL, on);
    if (lane == 0) warp_off[wid] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = it.spec_hist[blockIdx.x];
        for (int w = 0; w < SPEC_CHUNK / 32; ++w) {
            const int v = warp_off[w];
            warp_off[w] = run;
            run += v;
        }
    }
    __syncthreads();
    if (on) {
        const int slot = warp_off[wid] + __popc(b & ((1u << lane) - 1u));
        const int4 t = S.faces[f];
        const float fl = it.P.focal[0];
        float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
        const int id[3] = {t.x, t.y, t.z};
        for (int i = 0; i < 3; ++i) {
            const float4 p = S.v[id[i]];
            const float X = 0.5f * S.W + fl * p.x / -p.z, Y = 0.5f * S.H - fl * p.y / -p.z;
            x0 = fminf(x0, X); x1 = fmaxf(x1, X); y0 = fminf(y0, Y); y1 = fmaxf(y1, Y);
        }
        const float m = 1e-3f + 1e-5f * fmaxf(fabsf(x0) + fabsf(x1), fabsf(y0) + fabsf(y1));
        it.spec_list[slot] = f;
        it.spec_box[slot] = make_float4(x0 - m, x1 + m, y0 - m, y1 + m);
    }
}

// Scanline `scan` of an item: (row?, coordinate c in pixels), c = (i + u) / k.
FR_D bool spec_scanline(const DevScene& S, uint32_t iteration, uint32_t face, int scan, double& c) {
    const int k = max(S.edge_spp, 1);
    const bool row = scan < S.H * k;
    const int idx = row ? scan : scan - S.H * k;
    const Sampler sm{make_uint2(S.seed, FR_STREAM_EDGE_SPECULAR), 0xFFFFFFFFu, (uint32_t)scan, iteration, face};
    c = ((double)idx + (double)u24(sm.block(0).x)) / (double)k;
    return row;
}

// Crossings of the line (row?, c) with the curve inside triangle f, in order
// along the line: screen points (x, y); returns their count (0..2).  FP64.
FR_D int spec_roots(const DevScene& S, int f, bool row, double c, double fl, double2 out[2]) {
    const int4 t = S.faces[f];
    const int id[3] = {t.x, t.y, t.z};
    double v[3][3], n[3][3];
    for (int i = 0; i < 3; ++i) {
        const float4 a = S.v[id[i]], b = S.vn[id[i]];
        v[i][0] = a.x; v[i][1] = a.y; v[i][2] = a.z;
        n[i][0] = b.x; n[i][1] = b.y; n[i][2] = b.z;
    }
    const double nrm[3] = {row ? 0.0 : 1.0, row ? 1.0 : 0.0, row ? -(c - 0.5 * S.H) / fl : (c - 0.5 * S.W) / fl};
    double ph[3];
    for (int i = 0; i < 3; ++i) ph[i] = nrm[0] * v[i][0] + nrm[1] * v[i][1] + nrm[2] * v[i][2];
    double bc[2][3];
    int ne = 0;
    for (int e = 0; e < 3 && ne < 2; ++e) {           // chord ends: edges straddling the plane
        const int i = e, j = e == 2 ? 0 : e + 1;
        if ((ph[i] > 0.0) == (ph[j] > 0.0)) continue;
        const double tt = ph[i] / (ph[i] - ph[j]);
        bc[ne][0] = bc[ne][1] = bc[ne][2] = 0.0;
        bc[ne][i] = 1.0 - tt;
        bc[ne][j] = tt;
        ++ne;
    }
    if (ne != 2) return 0;
    double Q[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Q[i][j] = -(n[i][0] * v[j][0] + n[i][1] * v[j][1] + n[i][2] * v[j][2]);
    const double dl[3] = {bc[1][0] - bc[0][0], bc[1][1] - bc[0][1], bc[1][2] - bc[0][2]};
    double a2 = 0.0, a1 = 0.0, a0 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            a2 += dl[i] * dl[j] * Q[i][j];
            a1 += bc[0][i] * dl[j] * Q[i][j];
            a0 += bc[0][i] * bc[0][j] * Q[i][j];
        }
    double a1b = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) a1b += dl[i] * bc[0][j] * Q[i][j];
    a1 += a1b;
    double sr[2];
    int nr = 0;
    if (a2 == 0.0) {
        if (a1 != 0.0) sr[nr++] = -a0 / a1;
    } else {
        const double disc = a1 * a1 - 4.0 * a2 * a0;
        if (disc > 0.0) {
            const double sq = sqrt(disc);
            const double qq = -0.5 * (a1 + (a1 >= 0.0 ? sq : -sq));
            sr[nr++] = qq / a2;
            sr[nr++] = a0 / qq;
        }
    }
    int m = 0;
    for (int r = 0; r < nr; ++r) {
        if (!(sr[r] >= 0.0 && sr[r] <= 1.0)) continue;
        double p[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 3; ++i) {
            const double b = bc[0][i] + sr[r] * dl[i];
            p[0] += b * v[i][0]; p[1] += b * v[i][1]; p[2] += b * v[i][2];
        }
        out[m++] = row ? make_double2(0.5 * S.W + fl * p[0] / -p[2], c) : make_double2(c, 0.5 * S.H - fl * p[1] / -p[2]);
    }
    if (m == 2 && (row ? out[1].x < out[0].x : out[1].y < out[0].y)) {
        const double2 tmp = out[0];
        out[0] = out[1];
        out[1] = tmp;
    }
    return m;
}

constexpr int SPEC_QUEUE = 128;          // crossings queued per warp (< 32 wait before a chunk adds <= 64)

struct SpecQueue {
    int code[SPEC_QUEUE];                // 2 * triangle + root
    float x[SPEC_QUEUE], y[SPEC_QUEUE];
};

// Evaluate the queued crossings [head, head + n) (n <= 32), one lane each:
// the jump of the cutoff at the crossing x is the difference of the two
// one-sided limits of the radiance of the crossing's own triangle there (the
// same hit, shadow rays and light samples; the view direction tilted to
// n_s . o = +-1e-5), with no part of the continuous change across the curve
// and nothing of a silhouette the curve may run next to; the curve is seen
// only where that triangle is the visible surface (nothing along the camera
// ray is nearer).  All 32 lanes call this together.
template <bool ENV>
FR_D void spec_eval(const DevItem& it, const SpecQueue& q, int head, int n, int scan, bool row, RtShared& sh,
                    Stack stk, RayStats& rs, float& gfocal) {
    const DevScene& S = it.S;
    const DevParams& P = it.P;
    const int lane = threadIdx.x & 31;
    bool active = lane < n;
    const int code = active ? q.code[(head + lane) & (SPEC_QUEUE - 1)] : 0;
    const float X = active ? q.x[(head + lane) & (SPEC_QUEUE - 1)] : 0.0f;
    const float Y = active ? q.y[(head + lane) & (SPEC_QUEUE - 1)] : 0.0f;
    const int tri = code >> 1;
    const float f = P.focal[0];
    float3 adj = f3(0, 0, 0);
    HitChain hc;
    int4 fc = make_int4(0, 0, 0, 0);
    float gx = 0.0f, gy = 0.0f, g2 = 0.0f;
    bool front = false;
    float3 d = f3(0, 0, 0);
    Hit own;                        // the ray on the crossing's own triangle's plane
    own.tri = own.slot = -1;
    own.t = own.b1 = own.b2 = 0.0f;
    if (active) {
        const int pix = (int)floorf(Y) * S.W + (int)floorf(X);
        adj = f3(it.adj[3 * (size_t)pix], it.adj[3 * (size_t)pix + 1], it.adj[3 * (size_t)pix + 2]);
        if (adj.x == 0.0f && adj.y == 0.0f && adj.z == 0.0f) active = false;
    }
    if (active) {
        // G = n_s . o at the crossing and its gradients: d/dns = o, d/do = ns
        fc = S.faces[tri];
        const float3 v0 = xyz(S.v[fc.x]), v1 = xyz(S.v[fc.y]), v2 = xyz(S.v[fc.z]);
        const float3 n0 = xyz(S.vn[fc.x]), n1 = xyz(S.vn[fc.y]), n2 = xyz(S.vn[fc.z]);
        d = f3((X - 0.5f * S.W) / f, -(Y - 0.5f * S.H) / f, -1.0f);
        const float3 e1 = v1 - v0, e2 = v2 - v0, sv = -v0;
        const float3 pv = cross(d, e2), qv = cross(sv, e1);
        const float inv_det = __fdividef(1.0f, dot(e1, pv));
        const float b1 = dot(sv, pv) * inv_det, b2 = dot(d, qv) * inv_det, b0 = 1.0f - b1 - b2;
        const float t_own = dot(e2, qv) * inv_det;                 // along d to the triangle's plane
        own.t = t_own;
        own.b1 = b1;
        own.b2 = b2;
        own.tri = tri;
        own.slot = __ldg(&S.slot_of[tri]);
        const float3 mm = n0 * b0 + n1 * b1 + n2 * b2;
        const float3 ns = mm * rsqrtf(dot(mm, mm));
        const float3 o = -d * rsqrtf(dot(d, d));
        front = dot(cross(e1, e2), o) > 0.0f;
        hc = hit_chain(v0, v1, v2, n0, n1, n2, d, o, ns, f3(0, 0, 0), 0.0f, 0.0f, 0.0f);
        // d = ((X - W/2)/f, -(Y - H/2)/f, -1): dG/dX = gd.x / f, dG/dY = -gd.y / f
        gx = hc.gd.x / f;
        gy = -hc.gd.y / f;
        g2 = gx * gx + gy * gy;
        if (!(g2 > 0.0f)) active = false;
        if (active) {
            // (the traversal's own distance to a grazing triangle is only good to
            // ~1e-4 relative, so the triangle itself never hides the crossing)
            const Hit h = trace_closest(S, ray_setup(f3(0.0f, 0.0f, 0.0f), d), 0.0f, INFINITY, stk, rs);
            if (h.tri >= 0 && h.tri != tri && h.t < t_own * (1.0f - 1e-5f)) active = false;
        }
    }
    const Sampler smp{make_uint2(S.seed, FR_STREAM_EDGE_SPECULAR), (uint32_t)code, (uint32_t)scan, it.iteration,
                      it.face};
    // the crossing's own triangle at x (imposed: on a grazing sliver the
    // watertight test could reject a point of it); its shadow rays are those
    // of the lit side
    SampleState ss;
    primary_state<true, false>(S, P, active, X, Y, stk, ss, rs, REC_TRACE, &own);
    if (ss.hit) ss.lit = front;
    uint64_t vis[2] = {0ull, 0ull};
    for (int j0 = 0; j0 < max(S.NL, 1); j0 += 64)                  // warp-uniform
        vis[j0 >> 6] = shadow_mask<ENV>(S, ss, smp, 4, sh.wq[threadIdx.x >> 5], stk, rs, j0);
    float3 Lp = f3(0.0f, 0.0f, 0.0f), Lm = f3(0.0f, 0.0f, 0.0f);
    if (active && ss.hit) {
        sample_material(S, P, ss);
        const float3 om = ss.o - ss.ns * dot(ss.ns, ss.o);
        SampleState sp = ss, sm = ss;
        const float3 op = om + ss.ns * 1e-5f, on = om - ss.ns * 1e-5f;
        sp.o = op * rsqrtf(dot(op, op));
        sm.o = on * rsqrtf(dot(on, on));
        if (S.flags & FR_FLAG_VIEW_CUTOFF_D) sm.lit = false;        // the cut-everything reading
        for (int j0 = 0; j0 < max(S.NL, 1); j0 += 64) {
            Lp += radiance_from<ENV>(S, P, sp, vis[j0 >> 6], smp, 4, j0);
            Lm += radiance_from<ENV>(S, P, sm, vis[j0 >> 6], smp, 4, j0);
        }
    } else {
        active = false;
    }
    float wg = 0.0f;
    if (active) {
        const float jump = adj.x * (Lp.x - Lm.x) + adj.y * (Lp.y - Lm.y) + adj.z * (Lp.z - Lm.z);
        wg = jump * (row ? fabsf(gx) : fabsf(gy)) / (g2 * (float)max(S.edge_spp, 1));
        if (wg == 0.0f) active = false;
    }
    const unsigned act = __ballot_sync(FULL, active);
    if (active) {
        const int vx[3] = {fc.x, fc.y, fc.z};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            fix64* const a[6] = {&it.G.d_v[3 * vx[k]], &it.G.d_v[3 * vx[k] + 1], &it.G.d_v[3 * vx[k] + 2],
                                 &it.G.d_n[3 * vx[k]], &it.G.d_n[3 * vx[k] + 1], &it.G.d_n[3 * vx[k] + 2]};
            const float v[6] = {wg * hc.gv[k].x, wg * hc.gv[k].y, wg * hc.gv[k].z,
                                wg * hc.gn[k].x, wg * hc.gn[k].y, wg * hc.gn[k].z};
            warp_agg_add_n<6>(a, v, (uint32_t)vx[k], act);
        }
        gfocal += wg * -(hc.gd.x * d.x + hc.gd.y * d.y) / f;
    }
}

// One block per scanline of an item; its warps take the item's candidates in
// chunks of 32 (warp w: chunks w, w + 4, ...), queue the chunk's crossings in
// candidate order and evaluate them 32 at a time.
template <bool ENV>
__global__ void __launch_bounds__(RT_THREADS, 4) k_edge_specular(const DevItem* items, BlockMap map) {
    __shared__ RtShared sh;
    __shared__ SpecQueue sq[RT_WARPS];
    FR_STACK_DECL
    const int item = item_of_block(map);
    const DevItem& it = items[item];
    const DevScene& S = it.S;
    block_acc_init(1);
    const int scan = blockIdx.x - map.block0[item];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double c;
    const bool row = spec_scanline(S, it.iteration, it.face, scan, c);
    const double fl = (double)it.P.focal[0];
    const int n_cand = *it.spec_count;
    SpecQueue& q = sq[warp];
    int head = 0, count = 0;
    RayStats rs;
    float gfocal = 0.0f;
    for (int c0 = warp * 32; c0 < n_cand; c0 += RT_THREADS) {          // warp-uniform
        const int i = c0 + lane;
        int nc = 0;
        double2 xs[2];
        if (i < n_cand) {
            const float4 box = it.spec_box[i];
            const float cf = (float)c;
            if (row ? (cf >= box.z && cf <= box.w) : (cf >= box.x && cf <= box.y))
                nc = spec_roots(S, it.spec_list[i], row, c, fl, xs);
        }
        // keep the crossings inside the image
        int keep = 0;
        float kx[2], ky[2];
        int kc[2];
        for (int r = 0; r < nc; ++r) {
            if (!(xs[r].x >= 0.0 && xs[r].x < S.W && xs[r].y >= 0.0 && xs[r].y < S.H)) continue;
            const float fx = (float)xs[r].x, fy = (float)xs[r].y;
            if (!(fx < (float)S.W && fy < (float)S.H)) continue;      // rounded onto the far edge
            kx[keep] = fx;
            ky[keep] = fy;
            kc[keep] = 2 * it.spec_list[i] + r;
            ++keep;
        }
        // append in candidate order
        int before = keep;
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, before, o);
            if (lane >= o) before += v;
        }
        const int total = __shfl_sync(FULL, before, 31);
        before -= keep;
        for (int r = 0; r < keep; ++r) {
            const int slot = (head + count + before + r) & (SPEC_QUEUE - 1);
            q.code[slot] = kc[r];
            q.x[slot] = kx[r];
            q.y[slot] = ky[r];
        }
        count += total;
        __syncwarp();
        while (count >= 32) {
            spec_eval<ENV>(it, q, head, 32, scan, row, sh, my_stack(sh), rs, gfocal);
            head = (head + 32) & (SPEC_QUEUE - 1);
            count -= 32;
            __syncwarp();
        }
    }
    if (count > 0) {                                                    // warp-uniform
        spec_eval<ENV>(it, q, head, count, scan, row, sh, my_stack(sh), rs, gfocal);
        __syncwarp();
    }
    flush_stats(S.counters + 6, rs);
    const float gw = warp_sum(gfocal);
    if (lane == 0) acc_dyn[warp] = gw;
    block_acc_flush(1, 0, 1, it.G.small);
}

// ---------------------------------------------------------------------------
// silhouettes (FP64 classification) and ordered compaction
// ---------------------------------------------------------------------------
__device__ double3 face_normal_d(const DevScene& S, int f) {
    const int4 t = S.faces[f];
    const float4 p0 = S.v[t.x], p1 = S.v[t.y], p2 = S.v[t.z];
    const double e1x = (double)p1.x - p0.x, e1y = (double)p1.y - p0.y, e1z = (double)p1.z - p0.z;
    const double e2x = (double)p2.x - p0.x, e2y = (double)p2.y - p0.y, e2z = (double)p2.z - p0.z;
    return make_double3(e1y * e2z - e1z * e2y, e1z * e2x - e1x * e2z, e1x * e2y - e1y * e2x);
}

__device__ int sgn_d(double x) { return (x > 0.0) - (x < 0.0); }

// Signed-distance range [lo, hi] of emitter L over the plane of a face with
// (unnormalised) normal n through p0: the distance is linear over the
// emitter, so the range follows from the corners (quad, triangle) or the
// projected radius (disk).
template <class Real>
FR_D void emitter_range(int type, Real base, Real g1, Real g2, Real& lo, Real& hi) {
    if (type == 0) {
        const Real h = (Real)0.5 * fabs(g1) + (Real)0.5 * fabs(g2);
        lo = base - h; hi = base + h;
    } else if (type == 1) {
        lo = base + fmin((Real)0, fmin(g1, g2)); hi = base + fmax((Real)0, fmax(g1, g2));
    } else {
        const Real r = sqrt(g1 * g1 + g2 * g2);
        lo = base - r; hi = base + r;
    }
}

// Range [lo, hi] of n . w over the directions w of environment block L:
// n . w = n_y cos t + sin t A(p), A(p) = n_x sin p + n_z cos p.  A's range
// over the block's azimuths comes from the ends and its extremes at
// p = atan2(n_x, n_z) + k pi; as sin t >= 0 the minimum (maximum) over the
// block is that of n_y cos t + A_min sin t (A_max) over the polar range, a
// sinusoid whose extremes lie at the ends or at atan2(A, n_y) + k pi.
// Real = float for the fast first pass, double for the decision itself.
template <class Real>
__device__ void env_range(const LightDev& L, Real nx, Real ny, Real nz, Real& lo, Real& hi) {
    const Real pi = (Real)3.14159265358979323846, Me = (Real)L.env;
    const Real t0 = pi * (Real)L.c.x / Me, t1 = pi * (Real)L.c.y / Me;
    const Real f0 = 2 * pi * (Real)L.c.z / Me, f1 = 2 * pi * (Real)L.e1.x / Me;
    const Real A0 = nx * sin(f0) + nz * cos(f0), A1 = nx * sin(f1) + nz * cos(f1);
    Real a_lo = fmin(A0, A1), a_hi = fmax(A0, A1);
    const Real pa = atan2(nx, nz);
    for (int k = -2; k <= 3; ++k) {
        const Real p = pa + (Real)k * pi;
        if (p > f0 && p < f1) {
            const Real Ap = nx * sin(p) + nz * cos(p);
            a_lo = fmin(a_lo, Ap);
            a_hi = fmax(a_hi, Ap);
        }
    }
    for (int side = 0; side < 2; ++side) {
        const Real a = side ? a_hi : a_lo;
        const Real g0 = ny * cos(t0) + a * sin(t0), g1 = ny * cos(t1) + a * sin(t1);
        Real r = side ? fmax(g0, g1) : fmin(g0, g1);
        const Real tc = atan2(a, ny);
        for (int k = -1; k <= 2; ++k) {
            const Real t = tc + (Real)k * pi;
            if (t > t0 && t < t1) {
                const Real g = ny * cos(t) + a * sin(t);
                r = side ? fmax(r, g) : fmin(r, g);
            }
        }
        if (side) hi = r; else lo = r;
    }
}

// Facing class of face f over emitter j: 1 = every point of the emitter is in
// front of the face's plane, 2 = every point behind, 3 = mixed, decided in
// FP64.  An FP32 evaluation decides first whenever it is farther from zero
// than a bound on its rounding error (64 u times the sum of the magnitudes
// involved, u = 2^-24, a generous multiple of the few roundings per term), so
// the FP64 work runs only for nearly grazing pairs and every class equals the
// FP64 one.  Thread (face f, group blockIdx.y of CLS_LIGHTS emitters).
constexpr int CLS_LIGHTS = 8;

__global__ void k_face_class(const DevItem* items) {
    const DevItem& it = items[blockIdx.z];
    const DevScene& S = it.S;
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    const int j0 = blockIdx.y * CLS_LIGHTS, j1 = min(S.NL, j0 + CLS_LIGHTS);
    if (f >= S.T || j0 >= j1) return;
    const int4 tv = S.faces[f];
    const float3 q0 = xyz(S.v[tv.x]), q1 = xyz(S.v[tv.y]), q2 = xyz(S.v[tv.z]);
    const float3 a = q1 - q0, b = q2 - q0;
    const float3 nf = cross(a, b);
    const float3 na = f3(fabsf(a.y * b.z) + fabsf(a.z * b.y), fabsf(a.z * b.x) + fabsf(a.x * b.z),
                         fabsf(a.x * b.y) + fabsf(a.y * b.x));    // bounds |n| and its rounding
    // the FP64 plane, computed on first need
    bool have64 = false;
    double3 n = make_double3(0.0, 0.0, 0.0);
    double d = 0.0;
    auto plane64 = [&]() {
        if (have64) return;
        n = face_normal_d(S, f);
        const float4 p0 = S.v[tv.x];
        d = n.x * p0.x + n.y * p0.y + n.z * p0.z;
        have64 = true;
    };
    for (int j = j0; j < j1; ++j) {
        const LightDev& L = S.lights[j];
        if (L.type == FR_LIGHT_ENV_D) {        // a point at infinity along w is in front iff n . w > 0
            // FP32 first: it decides whenever it is farther from zero than a
            // generous bound on its error (64 u times the bound on |n|); else FP64
            float lo32, hi32;
            env_range<float>(L, nf.x, nf.y, nf.z, lo32, hi32);
            const float err = 64.0f * 5.9604645e-8f * (na.x + na.y + na.z);
            uint8_t cls = 0;
            if (lo32 > err) cls = 1;
            else if (hi32 < -err) cls = 2;
            else if (lo32 < -err && hi32 > err) cls = 3;
            if (!cls) {
                plane64();
                double lo, hi;
                env_range<double>(L, n.x, n.y, n.z, lo, hi);
                cls = lo > 0.0 ? 1 : (hi < 0.0 ? 2 : 3);
            }
            it.sil_flags[(size_t)(1 + FR_MAX_LIGHTS) * S.E + (size_t)j * S.T + f] = cls;
            continue;
        }
        {
            const float3 w = L.c - q0;
            float lo32, hi32;
            emitter_range<float>(L.type, dot(nf, w), dot(nf, L.e1), dot(nf, L.e2), lo32, hi32);
            const float mag = na.x * (fabsf(w.x) + fabsf(L.e1.x) + fabsf(L.e2.x)) +
                              na.y * (fabsf(w.y) + fabsf(L.e1.y) + fabsf(L.e2.y)) +
                              na.z * (fabsf(w.z) + fabsf(L.e1.z) + fabsf(L.e2.z));
            const float err = 64.0f * 5.9604645e-8f * mag;
            uint8_t cls = 0;
            if (lo32 > err) cls = 1;
            else if (hi32 < -err) cls = 2;
            else if (lo32 < -err && hi32 > err) cls = 3;
            if (cls) {
                it.sil_flags[(size_t)(1 + FR_MAX_LIGHTS) * S.E + (size_t)j * S.T + f] = cls;
                continue;
            }
        }
        plane64();
        const double base = n.x * L.c.x + n.y * L.c.y + n.z * L.c.z - d;
        const double g1 = n.x * L.e1.x + n.y * L.e1.y + n.z * L.e1.z;
        const double g2 = n.x * L.e2.x + n.y * L.e2.y + n.z * L.e2.z;
        double lo, hi;
        emitter_range<double>(L.type, base, g1, g2, lo, hi);
        it.sil_flags[(size_t)(1 + FR_MAX_LIGHTS) * S.E + (size_t)j * S.T + f] = lo > 0.0 ? 1 : (hi < 0.0 ? 2 : 3);
    }
}

// Ordered compaction of the flagged edge ids of every list, in three parallel
// passes: flags and per-chunk counts, per-list exclusive scan of the counts,
// scatter.
constexpr int CMP_CHUNK = 1024;
constexpr int CLS_LISTS = 8;

// flags[list][E]: list 0 = primary silhouettes (w.r.t. the camera centre,
// FP64 per edge), list 1 + j = conservative shadow candidates of light j
// (edges whose two faces are not both entirely in front of or both entirely
// behind emitter j).  Block (chunk of CMP_CHUNK edges, group blockIdx.y of
// CLS_LISTS lists) also writes each list's count of flagged edges in the
// chunk to hist[list][chunk] (the radix-sort histogram is free here).
__global__ void __launch_bounds__(CMP_CHUNK) k_classify(const DevItem* items, int n_chunks) {
    __shared__ int warp_cnt[CLS_LISTS][CMP_CHUNK / 32];
    const DevItem& it = items[blockIdx.z];
    const DevScene& S = it.S;
    const int l0 = blockIdx.y * CLS_LISTS, l1 = min(1 + S.NL, l0 + CLS_LISTS);
    if (l0 >= l1) return;                                // the whole block
    uint8_t* flags = it.sil_flags;
    const uint8_t* cls = flags + (size_t)(1 + FR_MAX_LIGHTS) * S.E;
    const int e = blockIdx.x * CMP_CHUNK + threadIdx.x;
    const bool in = e < S.E;
    const int4 E = in ? it.EL.edges[e] : make_int4(0, 0, 0, 0);
    for (int l = l0; l < l1; ++l) {
        bool on = false;
        if (in) {
            if (E.w < 0) {
                on = true;                               // a boundary edge is in every list
            } else if (l == 0) {
                const float4 pa = S.v[E.x];
                const double ax = pa.x, ay = pa.y, az = pa.z;
                const double3 n1 = face_normal_d(S, E.z), n2 = face_normal_d(S, E.w);
                on = sgn_d(-(n1.x * ax + n1.y * ay + n1.z * az)) != sgn_d(-(n2.x * ax + n2.y * ay + n2.z * az));
            } else {
                const size_t j = (size_t)(l - 1) * S.T;
                const uint8_t c1 = cls[j + E.z], c2 = cls[j + E.w];
                on = !((c1 == 1 && c2 == 1) || (c1 == 2 && c2 == 2));
            }
            flags[(size_t)l * S.E + e] = on;
        }
        const unsigned bal = __ballot_sync(FULL, on);
        if ((threadIdx.x & 31) == 0) warp_cnt[l - l0][threadIdx.x >> 5] = __popc(bal);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < l1 - l0) {                                   // warp w: list l0 + w, its 32 warp counts
        int v = warp_cnt[w][lane];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) it.B.hist[(l0 + w) * n_chunks + blockIdx.x] = v;
    }
}

// Exclusive scan of each list's chunk counts in place, one warp per list (32
// chunks a round, carried), and the list's total.
__global__ void k_compact_scan(const DevItem* items, int n_lists, int n_chunks) {
    const DevItem& it = items[blockIdx.x];
    const int lane = threadIdx.x & 31;
    for (int list = threadIdx.x >> 5; list < n_lists; list += blockDim.x >> 5) {
        int* h = it.B.hist + list * n_chunks;
        int carry = 0;
        for (int c0 = 0; c0 < n_chunks; c0 += 32) {
            const int c = c0 + lane;
            const int v = c < n_chunks ? h[c] : 0;
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(FULL, x, o);
                if (lane >= o) x += y;
            }
            if (c < n_chunks) h[c] = carry + x - v;
            carry += __shfl_sync(FULL, x, 31);
        }
        if (lane == 0) it.EL.prim_count[list] = carry;
    }
}

__global__ void __launch_bounds__(CMP_CHUNK) k_compact_scatter(const DevItem* items, int E, int n_chunks) {
    __shared__ int warp_off[CMP_CHUNK / 32];
    const DevItem& it = items[blockIdx.z];
    const int list = blockIdx.y, chunk = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = chunk * CMP_CHUNK + threadIdx.x;
    const bool on = i < E && it.sil_flags[(size_t)list * E + i];
    const unsigned b = __ballot_sync(FULL, on);
    if (lane == 0) warp_off[wid] = __popc(b);
    __syncthreads();
    if (wid == 0) {                                      // exclusive scan of the 32 warp counts
        const int v = warp_off[lane];
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        warp_off[lane] = it.B.hist[list * n_chunks + chunk] + x - v;
    }
    __syncthreads();
    if (on) it.EL.prim_list[(size_t)list * E + warp_off[wid] + __popc(b & ((1u << lane) - 1u))] = i;
}

__global__ void __launch_bounds__(RT_THREADS) k_trace_rays(const DevItem* items, const float* org, const float* dir,
                                                           int n, int32_t* tri, float* tout) {
    const DevScene& S = items[0].S;
    __shared__ int stack[FR_STACK * RT_THREADS];
    const int i = blockIdx.x * RT_THREADS + threadIdx.x;
    if (i >= n) return;
    const RayPre r = ray_setup(f3(org[3 * i], org[3 * i + 1], org[3 * i + 2]), f3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]));
    RayStats rs;
    const Hit h = trace_closest(S, r, 0.0f, INFINITY, Stack{&stack[threadIdx.x], RT_THREADS}, rs);
    tri[i] = h.tri;
    tout[i] = h.tri >= 0 ? h.t : -1.0f;
}

int blocks_for(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int map_blocks(const BlockMap& m) { return m.block0[m.n]; }

// Shared-memory carveout of the ray kernels in percent (-1: the driver's
// choice).  L1 holds the BVH nodes, triangles and local traversal stacks, so a
// large carveout starves it.
#ifndef FR_CARVEOUT
#define FR_CARVEOUT -1
#endif
template <bool ENV>
void set_carveout() {
    static bool done = false;
    if (done || FR_CARVEOUT < 0) return;
    cudaFuncSetAttribute(k_forward<ENV>, cudaFuncAttributePreferredSharedMemoryCarveout, FR_CARVEOUT);
    cudaFuncSetAttribute(k_adjoint<false, ENV>, cudaFuncAttributePreferredSharedMemoryCarveout, FR_CARVEOUT);
    cudaFuncSetAttribute(k_adjoint<true, ENV>, cudaFuncAttributePreferredSharedMemoryCarveout, FR_CARVEOUT);
    cudaFuncSetAttribute(k_edge_primary<ENV>, cudaFuncAttributePreferredSharedMemoryCarveout, FR_CARVEOUT);
    done = true;
}

// env: some item of the launch has environment blocks (the kernels compiled
// with their code); otherwise the light-stage-only instantiation runs.
void launch_forward(const DevItem* items, const BlockMap& map, bool env, long q0, bool records_only,
                    cudaStream_t st) {
    if (map_blocks(map) == 0) return;
    if (env) {
        set_carveout<true>();
        k_forward<true><<<map_blocks(map), RT_THREADS, 0, st>>>(items, map, q0, records_only ? 1 : 0);
    } else {
        set_carveout<false>();
        k_forward<false><<<map_blocks(map), RT_THREADS, 0, st>>>(items, map, q0, records_only ? 1 : 0);
    }
    fr_count_launches(1);
}

void launch_adjoint(const DevItem* items, const BlockMap& map, int NL, bool all_recorded, bool any_stage, bool env,
                    long q0, cudaStream_t st) {
    if (map_blocks(map) == 0) return;
    const size_t acc_bytes = sizeof(float) * RT_WARPS * (1 + (any_stage ? 7 : 3) * (size_t)NL);
    if (env) {
        if (all_recorded)
            k_adjoint<true, true><<<map_blocks(map), RT_THREADS, acc_bytes, st>>>(items, map, q0);
        else
            k_adjoint<false, true><<<map_blocks(map), RT_THREADS, acc_bytes, st>>>(items, map, q0);
    } else {
        if (all_recorded)
            k_adjoint<true, false><<<map_blocks(map), RT_THREADS, acc_bytes, st>>>(items, map, q0);
        else
            k_adjoint<false, false><<<map_blocks(map), RT_THREADS, acc_bytes, st>>>(items, map, q0);
    }
    fr_count_launches(1);
}

void launch_edge_order(const DevItem* items, int n, long max_edge, cudaStream_t st) {
    if (n <= 0 || max_edge <= 0) return;
    k_edge_order<<<dim3((unsigned)((max_edge + EDGE_CHUNK - 1) / EDGE_CHUNK), n), EDGE_SORT_THREADS, 0, st>>>(items);
    fr_count_launches(1);
}

void launch_edge_primary(const DevItem* items, const BlockMap& map, bool env, cudaStream_t st) {
    if (map_blocks(map) == 0) return;
    if (env)
        k_edge_primary<true><<<map_blocks(map), RT_THREADS, sizeof(float) * RT_WARPS, st>>>(items, map);
    else
        k_edge_primary<false><<<map_blocks(map), RT_THREADS, sizeof(float) * RT_WARPS, st>>>(items, map);
    fr_count_launches(1);
}

// Candidates of the specular-boundary term (ordered list per item); they need
// only the posed geometry and the camera.  `map` is the boundary kernel's.
void launch_spec_candidates(const DevItem* items, int n, int T, const BlockMap& map, cudaStream_t st) {
    if (n <= 0 || map_blocks(map) == 0) return;
    const int n_chunks = blocks_for(T, SPEC_CHUNK);
    k_spec_count<<<dim3(n_chunks, n), SPEC_CHUNK, 0, st>>>(items);
    k_spec_scan<<<n, 32, 0, st>>>(items);
    k_spec_scatter<<<dim3(n_chunks, n), SPEC_CHUNK, 0, st>>>(items);
    fr_count_launches(3);
}

// The specular-boundary term over the candidates: one block per scanline of
// each item (`map`).
void launch_edge_specular(const DevItem* items, const BlockMap& map, bool env, cudaStream_t st) {
    if (map_blocks(map) == 0) return;
    if (env)
        k_edge_specular<true><<<map_blocks(map), RT_THREADS, sizeof(float) * RT_WARPS, st>>>(items, map);
    else
        k_edge_specular<false><<<map_blocks(map), RT_THREADS, sizeof(float) * RT_WARPS, st>>>(items, map);
    fr_count_launches(1);
}

void launch_classify(const DevItem* items, int n, int E, int NL, int T, cudaStream_t st) {
    if (NL > 0) {
        k_face_class<<<dim3(blocks_for(T, 256), blocks_for(NL, CLS_LIGHTS), n), 256, 0, st>>>(items);
        fr_count_launches(1);
    }
    const int n_chunks = blocks_for(E, CMP_CHUNK);
    k_classify<<<dim3(n_chunks, blocks_for(1 + NL, CLS_LISTS), n), CMP_CHUNK, 0, st>>>(items, n_chunks);
    k_compact_scan<<<n, 32 * std::min(32, 1 + NL), 0, st>>>(items, 1 + NL, n_chunks);
    k_compact_scatter<<<dim3(n_chunks, 1 + NL, n), CMP_CHUNK, 0, st>>>(items, E, n_chunks);
    fr_count_launches(3);
}

void launch_trace_rays(const DevItem* items, const float* org, const float* dir, int n, int32_t* tri, float* t,
                       cudaStream_t st) {
    if (n <= 0) return;
    k_trace_rays<<<blocks_for(n, RT_THREADS), RT_THREADS, 0, st>>>(items, org, dir, n, tri, t);
    fr_count_launches(1);
}
