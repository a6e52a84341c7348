// Shared device definitions of the facert CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define FR_HD __host__ __device__ __forceinline__
#define FR_D __device__ __forceinline__

// device status word bits (read by fr_sync_status)
#define FR_STATUS_STACK_OVERFLOW 1
#define FR_STATUS_TIMEOUT 2
#define FR_STATUS_BAD_BVH 4
// a bounded wait gave up and so did the second wait for the CTA's own copies or
// MMAs in flight: a late write may still land, so the context is unusable
#define FR_STATUS_TIMEOUT_UNSAFE 8

constexpr int FR_MAX_LIGHTS = 128;
constexpr int FR_MAX_ENV_D = 64;       // environment map side (FR_MAX_ENV of the C interface)
constexpr int FR_MAX_BASIS = 256;
constexpr int FR_STACK = 64;           // traversal stack entries per thread
constexpr int FR_MAX_SPP = 256;        // camera samples per pixel
constexpr float FR_PI = 3.14159265358979323846f;

// ---------------------------------------------------------------------------
// small vector algebra
// ---------------------------------------------------------------------------
FR_HD float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
FR_HD float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
FR_HD float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
FR_HD float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
FR_HD float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
FR_HD float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
FR_HD float3& operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
FR_HD float3& operator-=(float3& a, float3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
FR_HD float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
FR_HD float3 cross(float3 a, float3 b) {
    return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
FR_HD float length(float3 a) { return sqrtf(dot(a, a)); }
FR_HD float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }
FR_HD float comp(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32 -> 64-bit multiplies, key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
FR_D uint4 philox4x32_10(uint2 key, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { key.x += 0x9E3779B9u; key.y += 0xBB67AE85u; }
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ key.x, lo1, hi0 ^ c.w ^ key.y, lo0);
    }
    return c;
}

// 24-bit uniform in [0, 1): (x >> 8) * 2^-24, exact in float.
FR_D float u24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

// Sample stream: key (seed, tag), counter (index, (sample << 16) | block,
// iteration, face).  Dimension d lives in word d % 4 of block d / 4.
enum { FR_STREAM_PRIMARY = 0, FR_STREAM_EDGE_PRIMARY = 1, FR_STREAM_EDGE_SHADOW = 2, FR_STREAM_EDGE_SPECULAR = 3 };

struct Sampler {
    uint2 key;
    uint32_t index, sample, iteration, face;
    FR_D uint4 block(int b) const {
        return philox4x32_10(key, make_uint4(index, (sample << 16) | (uint32_t)b, iteration, face));
    }
    // two consecutive dims starting at an even dim d (same block)
    FR_D float2 pair(int d) const {
        uint4 w = block(d >> 2);
        return (d & 2) ? make_float2(u24(w.z), u24(w.w)) : make_float2(u24(w.x), u24(w.y));
    }
};

// ---------------------------------------------------------------------------
// device-side scene description (plain pointers, passed by value to kernels)
// ---------------------------------------------------------------------------
// Area emitters (types 0-2) use c, e1, e2, n, area and scale.  An environment
// block (type 3, lights at infinity, Sec. 7) keeps its texel rows [i0, i1) and
// columns [j0, j1) as small integers in c = (i0, i1, j0) and e1.x = j1, the
// map's side in `env`; area = texels in the block, scale = 1.
struct LightDev {
    float3 c, e1, e2, n;   // n: unit normal of the emitting side
    float area, scale;     // scale = d^2 / a  (Eq. lightIntensity)
    int type, env;
};

// Binary BVH node holding both children's boxes (64 B, four 16-B loads).
struct __align__(16) BvhNode {
    float4 a;   // lo0.x lo0.y lo0.z hi0.x
    float4 b;   // hi0.y hi0.z lo1.x lo1.y
    float4 c;   // lo1.z hi1.x hi1.y hi1.z
    int4 d;     // child0, child1 (>= 0 internal, < 0 leaf ~slot), pad, pad
};

struct DevScene {
    int N, T, K, NL, E, W, H, spp, M, edge_spp;
    uint32_t flags, seed;
    const float4* v;        // camera-space vertices [N]
    const float4* vn;       // unit vertex normals [N]
    const float2* uv;       // [N]
    const int4* faces;      // [T]
    const BvhNode* nodes;   // [max(T - 1, 1)]
    const float4* tris;     // [3T] triangles in BVH leaf order; tris[3s].w = id bits
    const int* slot_of;     // [T] leaf slot of each triangle (inverse of the leaf order)
    const LightDev* lights; // [NL]
    const float* stage;     // [NL][12] virtual light stage frame (centre, unit face V0 V1 V2);
                            // non-null when the lights are built from (d, a, p) parameters
    int env_size;           // side of the environment map (0: no environment blocks)
    int* status;
    unsigned long long* counters;   // [3][3]: per kernel (forward, adjoint, primary edges) rays, nodes, triangle tests
};

// Per-thread traversal work, flushed once per warp at the end of a kernel.
struct RayStats {
    uint32_t rays = 0, nodes = 0, tris = 0;
};

FR_D void flush_stats(unsigned long long* counters, const RayStats& rs) {
    unsigned long long v[3] = {rs.rays, rs.nodes, rs.tris};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    if ((threadIdx.x & 31) == 0 && v[0]) {
        atomicAdd(&counters[0], v[0]);
        atomicAdd(&counters[1], v[1]);
        atomicAdd(&counters[2], v[2]);
    }
}

struct DevParams {
    const float *coef, *rot, *trans, *focal, *light_i, *diffuse, *specular, *roughness;
    const float *light_d, *light_a, *light_p;   // light stage geometry [NL], [NL], [NL][2]
    const float* env;                           // environment radiance [env][env][3]
};

// Fixed-point accumulator layout of G.small: focal, then 3 per light
// (intensity), then from FR_GEO_OFF 4 per light (d, a, p0, p1), then from
// FR_ENV_OFF 3 per environment texel.
constexpr int FR_GEO_OFF = 1 + 3 * FR_MAX_LIGHTS;
constexpr int FR_ENV_OFF = FR_GEO_OFF + 4 * FR_MAX_LIGHTS;
constexpr int FR_SMALL = FR_ENV_OFF + 3 * FR_MAX_ENV_D * FR_MAX_ENV_D;

// Gradient sums are kept in 64-bit fixed point (resolution 2^-32, range
// +-2^31): integer addition is associative, so a sum does not depend on the
// order in which atomics land, and every result is bitwise reproducible
// whatever else shares the launch.
typedef unsigned long long fix64;
constexpr double FR_FIX_SCALE = 4294967296.0;
// round(v * 2^32) to nearest, ties to even: scaling by a power of two is
// exact in FP32 for |v| < 2^31, so converting the FP32 product gives the same
// integer as the FP64 product without using the (narrow) FP64 pipe; measured
// 6% faster adjoint than the FP64 conversion.  Larger |v| saturates.
FR_D long long to_fix(float v) { return __float2ll_rn(v * 4294967296.0f); }
FR_D long long to_fix_d(double v) { return __double2ll_rn(v * FR_FIX_SCALE); }
FR_D double from_fix(fix64 v) { return (double)(long long)v * (1.0 / FR_FIX_SCALE); }
FR_D void fix_add(fix64* a, float v) {
    if (v != 0.0f) atomicAdd(a, (fix64)to_fix(v));
}

struct DevGrads {
    fix64* d_v;            // [N][3] dE/dv' (camera space)
    fix64* d_n;            // [N][3] dE/dn (unit vertex normals)
    fix64* tex;            // [3 M^2] diffuse, [3 M^2] specular, [M^2] roughness
    float *diffuse, *specular, *roughness;   // caller texture gradients (may be null)
    fix64* small;          // [1 + 3 N_L]: focal, then light intensities
};

struct BvhScratch {
    uint32_t *keys, *keys_alt;
    int *vals, *vals_alt;
    int* hist;           // [256][n_tiles]
    int* hist_base;      // [256] digit bases
    int* child;          // [2 (T - 1)] child codes of internal nodes
    int* parent_int;     // [T - 1]
    int* parent_leaf;    // [T]
    int* flag;           // [T - 1]
    float4* box_int;     // [2 (T - 1)] lo, hi
    float4* box_leaf;    // [2 T]
    unsigned* aabb;      // [6] ordered-int scene bounds
};

struct EdgeLists {
    const int4* edges;   // [E] (a, b, f1, f2), a < b, f2 = -1 on the boundary (shared)
    int* prim_list;      // [E]   ordered primary silhouettes (compacted list 0)
    int* prim_count;     // [1]
    int* light_list;     // [NL][E] ordered shadow candidates (lists 1..NL)
    int* light_count;    // [NL]
};

constexpr int FR_MAX_BATCH = 64;

// Everything one face of a batched call needs: its slot's geometry and scratch,
// its image configuration, its parameters and where its results go.  The table
// of items lives in device memory; every kernel of a call reads its item from it
// (geometry kernels by blockIdx.y, ray kernels through a BlockMap).
struct DevItem {
    DevScene S;             // slot geometry (read side) + W, H, spp, edge_spp, flags, seed
    DevParams P;
    DevGrads G;             // d_v, d_n (slot), texture gradients (caller), small (slot)
    EdgeLists EL;
    BvhScratch B;
    BvhNode* nodes;         // slot BVH (write side of S.nodes)
    float4* tris;           // slot triangles (write side of S.tris)
    int* slot_of;           // write side of S.slot_of
    float4* v_cam;          // write side of S.v
    float4* vn;             // write side of S.vn
    float* v_model;
    float* d_vmodel;
    float4* n_face;
    float* dm;
    double* pose_part;      // [ceil(N / 256)][12] per-block pose-gradient partials
    uint8_t* sil_flags;
    float* image;
    const float* adj;       // image-space adjoint read by the ray kernels
    int32_t* tri_rec;
    uint64_t* mask_rec;
    int32_t* rec_tri;       // hit records [rec_cap] (null: the adjoint re-traces every sample)
    uint64_t* rec_vis;      // [rec_cap][1 or 2] visibility words, lights 0..63 (and 64..127 when there
                            // are more than 64), written for samples that hit
    long rec_cap;           // camera samples the record buffer holds (a tile of the image)
    int rec_full;           // this call's forward writes the records of the whole image (it fits)
    long rec_from;          // the forward writes the records of samples >= rec_from (0 with rec_full,
                            // else the first sample of the image's last tile; -1: none)
    int* edge_perm;         // processing order of the primary-edge samples (null: index order)
    int* spec_list;         // candidate triangles of the specular-boundary term [T] (ordered)
    float4* spec_box;       // their screen boxes (x0, x1, y0, y1) [T]
    int* spec_hist;         // per-chunk candidate counts, then offsets [ceil(T / 1024)]
    int* spec_count;        // [1]
    uint8_t* spec_flag;     // each triangle a candidate? [T]
    float *g_coef, *g_rot, *g_trans, *g_focal, *g_light;   // caller gradient outputs (may be null)
    float *g_light_d, *g_light_a, *g_light_p;            // light stage geometry gradients (may be null)
    float* g_env;                                         // environment radiance gradient (may be null)
    LightDev* lights_w;     // write side of S.lights when built from stage parameters
    uint32_t iteration, face;
};

// Blocks [block0[k], block0[k+1]) of a ray launch belong to item k.
struct BlockMap {
    int n;
    int block0[FR_MAX_BATCH + 1];
};

FR_D int item_of_block(const BlockMap& m) {
    int k = 0;
    while (k + 1 < m.n && (int)blockIdx.x >= m.block0[k + 1]) ++k;
    return k;
}

FR_D void set_status(int* status, int bit) { atomicOr(status, bit); }

// Warp-aggregated fixed-point add of N values that share one key (the
// channels of one texel, the coordinates of one vertex): one match over the
// warp, then each value summed over the lanes sharing the key in lane order,
// and the sums added to addr[n] by the first of those lanes.
template <int N>
FR_D void warp_agg_add_n(fix64* const (&addr)[N], const float (&val)[N], uint32_t key, uint32_t active) {
    const uint32_t peers = __match_any_sync(active, key);
    const int lane = threadIdx.x & 31;
    float sum[N];
#pragma unroll
    for (int n = 0; n < N; ++n) sum[n] = 0.0f;
    uint32_t m = peers;
    while (m) {
        const int src = __ffs(m) - 1;
#pragma unroll
        for (int n = 0; n < N; ++n) sum[n] += __shfl_sync(peers, val[n], src);
        m &= m - 1;
    }
    if (lane == __ffs(peers) - 1) {
#pragma unroll
        for (int n = 0; n < N; ++n) fix_add(addr[n], sum[n]);
    }
}

