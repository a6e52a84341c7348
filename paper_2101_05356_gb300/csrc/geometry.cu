// Pose (Gamma(v) = R^-1 (v - T), Sec. 3.1), face/vertex normals, Morton keys,
// and the reverse of each step (normals, pose with FP64 reductions); the morph
// and its transpose are in linear.cu.  Every kernel is batched over the items
// of a call through blockIdx.y.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace {

// R = Rz(t2) Ry(t1) Rx(t0), row-major
FR_D void euler_R(const float* rot, float R[9]) {
    float sx, cx, sy, cy, sz, cz;
    sincosf(rot[0], &sx, &cx);
    sincosf(rot[1], &sy, &cy);
    sincosf(rot[2], &sz, &cz);
    R[0] = cz * cy; R[1] = cz * sy * sx - sz * cx; R[2] = cz * sy * cx + sz * sx;
    R[3] = sz * cy; R[4] = sz * sy * sx + cz * cx; R[5] = sz * sy * cx - cz * sx;
    R[6] = -sy;     R[7] = cy * sx;                R[8] = cy * cx;
}

// Items per k_set_items launch: 32 x 632-byte items stay under the 32 KB
// kernel-parameter limit.
constexpr int ITEMS_PER_LAUNCH = 32;

struct ItemsParam {
    int n;
    DevItem it[ITEMS_PER_LAUNCH];
};

__global__ void k_set_items(ItemsParam p, DevItem* out) {
    const int words = (int)(sizeof(DevItem) / sizeof(int));
    for (int k = 0; k < p.n; ++k) {
        const int* src = reinterpret_cast<const int*>(&p.it[k]);
        int* dst = reinterpret_cast<int*>(&out[k]);
        for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
    }
}

// per-item fixed-point accumulators of the adjoint: dE/dv', dE/dn, texture
// gradients, focal and light partials
__global__ void k_zero_acc(const DevItem* items, int N, int M) {
    const DevItem& it = items[blockIdx.y];
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 3L * N) { it.G.d_v[i] = 0ull; it.G.d_n[i] = 0ull; }
    if (i < 7L * M * M) it.G.tex[i] = 0ull;
    if (blockIdx.x == 0) {
        const int n_small = FR_ENV_OFF + 3 * it.S.env_size * it.S.env_size;
        for (int k = threadIdx.x; k < n_small; k += blockDim.x) it.G.small[k] = 0ull;
    }
}

// add the fixed-point texture gradients into the caller's float gradients
__global__ void k_tex_flush(const DevItem* items, int M) {
    const DevItem& it = items[blockIdx.y];
    const long M2 = (long)M * M;
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 7 * M2) return;
    const float g = (float)from_fix(it.G.tex[i]);
    if (i < 3 * M2) { if (it.G.diffuse) it.G.diffuse[i] += g; }
    else if (i < 6 * M2) { if (it.G.specular) it.G.specular[i - 3 * M2] += g; }
    else if (it.G.roughness) it.G.roughness[i - 6 * M2] += g;
}

FR_D unsigned ordered(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
FR_D float unordered(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__global__ void k_aabb_reset(const DevItem* items) {
    unsigned* aabb = items[blockIdx.x].B.aabb;
    if (threadIdx.x < 3) aabb[threadIdx.x] = 0xffffffffu;
    else if (threadIdx.x < 6) aabb[threadIdx.x] = 0u;
}

__global__ void __launch_bounds__(256) k_pose(const DevItem* items, int N) {
    __shared__ float R[9], T[3];
    __shared__ unsigned bmin[3], bmax[3];
    const DevItem& it = items[blockIdx.y];
    if (threadIdx.x == 0) {
        euler_R(it.P.rot, R);
        T[0] = it.P.trans[0]; T[1] = it.P.trans[1]; T[2] = it.P.trans[2];
        for (int k = 0; k < 3; ++k) { bmin[k] = 0xffffffffu; bmax[k] = 0u; }
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const float* vm = it.v_model;
        const float wx = vm[3 * i] - T[0], wy = vm[3 * i + 1] - T[1], wz = vm[3 * i + 2] - T[2];
        // v' = R^T w
        const float x = R[0] * wx + R[3] * wy + R[6] * wz;
        const float y = R[1] * wx + R[4] * wy + R[7] * wz;
        const float z = R[2] * wx + R[5] * wy + R[8] * wz;
        it.v_cam[i] = make_float4(x, y, z, 0.0f);
        atomicMin(&bmin[0], ordered(x)); atomicMin(&bmin[1], ordered(y)); atomicMin(&bmin[2], ordered(z));
        atomicMax(&bmax[0], ordered(x)); atomicMax(&bmax[1], ordered(y)); atomicMax(&bmax[2], ordered(z));
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        atomicMin(&it.B.aabb[threadIdx.x], bmin[threadIdx.x]);
        atomicMax(&it.B.aabb[3 + threadIdx.x], bmax[threadIdx.x]);
    }
}

FR_D uint32_t spread10(uint32_t x) {
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000FFu;
    x = (x | (x << 8)) & 0x0300F00Fu;
    x = (x | (x << 4)) & 0x030C30C3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__global__ void __launch_bounds__(256) k_faces(const DevItem* items, const int4* __restrict__ faces, int T) {
    const DevItem& it = items[blockIdx.y];
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= T) return;
    const int4 t = faces[f];
    const float4* v = it.v_cam;
    const float3 a = xyz(v[t.x]), b = xyz(v[t.y]), c = xyz(v[t.z]);
    const float3 n = cross(b - a, c - a);
    it.n_face[f] = make_float4(n.x, n.y, n.z, 0.0f);
    const unsigned* aabb = it.B.aabb;
    const float3 lo = f3(unordered(aabb[0]), unordered(aabb[1]), unordered(aabb[2]));
    const float3 hi = f3(unordered(aabb[3]), unordered(aabb[4]), unordered(aabb[5]));
    const float3 cen = (a + b + c) * (1.0f / 3.0f);
    uint32_t code = 0;
    for (int k = 0; k < 3; ++k) {
        const float ext = comp(hi, k) - comp(lo, k);
        float u = ext > 0.0f ? (comp(cen, k) - comp(lo, k)) / ext : 0.5f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);
        const uint32_t q = min((uint32_t)(u * 1024.0f), 1023u);
        code |= spread10(q) << (2 - k);
    }
    if (it.B.keys) {                         // Morton keys only for the per-call LBVH rebuild
        it.B.keys[f] = code;
        it.B.vals[f] = f;
    }
}

// Vertex normal = normalised sum of its faces' un-normalised normals, gathered
// in face-index order through the vertex->face CSR (no atomics).  w = |sum|.
__global__ void __launch_bounds__(256) k_vertex_normals(const DevItem* items, const int* __restrict__ off,
                                                        const int* __restrict__ idx, int N) {
    const DevItem& it = items[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float3 m = f3(0.0f, 0.0f, 0.0f);
    for (int k = off[i]; k < off[i + 1]; ++k) m += xyz(it.n_face[idx[k]]);
    const float len = length(m);
    const float inv = len > 0.0f ? 1.0f / len : 0.0f;
    it.vn[i] = make_float4(m.x * inv, m.y * inv, m.z * inv, len);
}

// dE/dm_i = (I - n n^T) dE/dn_i / |m_i|
__global__ void k_normals_adj_a(const DevItem* items, int N) {
    const DevItem& it = items[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 n4 = it.vn[i];
    const float3 n = xyz(n4);
    const fix64* d_n = it.G.d_n;
    const float3 g = f3((float)from_fix(d_n[3 * i]), (float)from_fix(d_n[3 * i + 1]), (float)from_fix(d_n[3 * i + 2]));
    const float inv = n4.w > 0.0f ? 1.0f / n4.w : 0.0f;
    const float3 r = (g - n * dot(n, g)) * inv;
    it.dm[3 * i] = r.x; it.dm[3 * i + 1] = r.y; it.dm[3 * i + 2] = r.z;
}

// Face normal n_f = (b - a) x (c - a) feeds m of its three vertices; gather the
// cross-product adjoint back to each vertex over its faces.
__global__ void k_normals_adj_b(const DevItem* items, const int4* __restrict__ faces, const int* __restrict__ off,
                                const int* __restrict__ idx, int N) {
    const DevItem& it = items[blockIdx.y];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float* dm = it.dm;
    const float4* v = it.v_cam;
    float3 acc = f3(0.0f, 0.0f, 0.0f);
    for (int k = off[i]; k < off[i + 1]; ++k) {
        const int4 t = faces[idx[k]];
        const float3 G = f3(dm[3 * t.x] + dm[3 * t.y] + dm[3 * t.z], dm[3 * t.x + 1] + dm[3 * t.y + 1] + dm[3 * t.z + 1],
                            dm[3 * t.x + 2] + dm[3 * t.y + 2] + dm[3 * t.z + 2]);
        const float3 a = xyz(v[t.x]), b = xyz(v[t.y]), c = xyz(v[t.z]);
        const float3 gu = cross(c - a, G);     // d/d(b - a)
        const float3 gw = cross(G, b - a);     // d/d(c - a)
        if (i == t.x) acc -= gu + gw;
        else if (i == t.y) acc += gu;
        else acc += gw;
    }
    fix64* d_v = it.G.d_v;                       // one writer per vertex here
    d_v[3 * i] += (fix64)to_fix(acc.x);
    d_v[3 * i + 1] += (fix64)to_fix(acc.y);
    d_v[3 * i + 2] += (fix64)to_fix(acc.z);
}

// dE/dv = R dE/dv'; per-block partials of M'[r][c] = sum_i g_r w_c and
// sum_i g (FP64), summed in block order by k_pose_finish.
__global__ void __launch_bounds__(256) k_pose_adj(const DevItem* items, int N) {
    __shared__ float R[9], T[3];
    __shared__ double part[8][12];
    const DevItem& it = items[blockIdx.y];
    if (threadIdx.x == 0) {
        euler_R(it.P.rot, R);
        T[0] = it.P.trans[0]; T[1] = it.P.trans[1]; T[2] = it.P.trans[2];
    }
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double loc[12];
    for (int k = 0; k < 12; ++k) loc[k] = 0.0;
    if (i < N) {
        const fix64* d_v = it.G.d_v;
        const float* vm = it.v_model;
        const float g[3] = {(float)from_fix(d_v[3 * i]), (float)from_fix(d_v[3 * i + 1]), (float)from_fix(d_v[3 * i + 2])};
        const float w[3] = {vm[3 * i] - T[0], vm[3 * i + 1] - T[1], vm[3 * i + 2] - T[2]};
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) loc[3 * r + c] = (double)g[r] * (double)w[c];
        for (int r = 0; r < 3; ++r) loc[9 + r] = g[r];
        for (int c = 0; c < 3; ++c)
            it.d_vmodel[3 * i + c] = R[3 * c + 0] * g[0] + R[3 * c + 1] * g[1] + R[3 * c + 2] * g[2];
    }
    for (int k = 0; k < 12; ++k)
        for (int o = 16; o > 0; o >>= 1) loc[k] += __shfl_xor_sync(0xffffffffu, loc[k], o);
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 12; ++k) part[threadIdx.x >> 5][k] = loc[k];
    __syncthreads();
    if (threadIdx.x < 12) {
        double s = 0.0;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += part[wv][threadIdx.x];
        it.pose_part[blockIdx.x * 12 + threadIdx.x] = s;
    }
}

// dE/dtheta_a = sum_rc M'[r][c] dR[c][r]/dtheta_a ; dE/dT = -R sum g; plus the
// FP64 focal and light-intensity accumulators.  One block of 192 threads per item.
__global__ void k_pose_finish(const DevItem* items, int NL, int n_blocks) {
    __shared__ double acc12[12];
    const DevItem& it = items[blockIdx.x];
    const int t = threadIdx.x;
    // the 12 sums over the blocks' partials: 16 lanes per value (a half warp),
    // lane l summing blocks l, l + 16, ... in order, then a fixed butterfly
    if (t < 12 * 16) {
        const int k = t >> 4, l = t & 15;
        double s = 0.0;
        for (int b = l; b < n_blocks; b += 16) s += it.pose_part[b * 12 + k];
        for (int o = 8; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) acc12[k] = s;
    }
    __syncthreads();
    const fix64* small = it.G.small;
    if (t == 0) {
        // the angles' sines and cosines in FP32 (~1e-7 relative; FP64 transcendentals
        // run on the narrow FP64 pipe), the contractions in FP64
        float fsx, fcx, fsy, fcy, fsz, fcz;
        sincosf(it.P.rot[0], &fsx, &fcx);
        sincosf(it.P.rot[1], &fsy, &fcy);
        sincosf(it.P.rot[2], &fsz, &fcz);
        const double sx = fsx, cx = fcx, sy = fsy, cy = fcy, sz = fsz, cz = fcz;
        double Rx[9] = {1, 0, 0, 0, cx, -sx, 0, sx, cx}, dRx[9] = {0, 0, 0, 0, -sx, -cx, 0, cx, -sx};
        double Ry[9] = {cy, 0, sy, 0, 1, 0, -sy, 0, cy}, dRy[9] = {-sy, 0, cy, 0, 0, 0, -cy, 0, -sy};
        double Rz[9] = {cz, -sz, 0, sz, cz, 0, 0, 0, 1}, dRz[9] = {-sz, -cz, 0, cz, -sz, 0, 0, 0, 0};
        auto mul = [](const double* A, const double* B, double* C) {
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double s = 0.0;
                    for (int k = 0; k < 3; ++k) s += A[3 * i + k] * B[3 * k + j];
                    C[3 * i + j] = s;
                }
        };
        double tmp[9], D[3][9], R[9];
        mul(Ry, Rx, tmp); mul(Rz, tmp, R);
        mul(Ry, dRx, tmp); mul(Rz, tmp, D[0]);
        mul(dRy, Rx, tmp); mul(Rz, tmp, D[1]);
        mul(Ry, Rx, tmp); mul(dRz, tmp, D[2]);
        for (int q = 0; q < 3; ++q) {
            double s = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c2 = 0; c2 < 3; ++c2) s += acc12[3 * r + c2] * D[q][3 * c2 + r];
            if (it.g_rot) it.g_rot[q] += (float)s;
        }
        for (int c2 = 0; c2 < 3; ++c2) {
            double s = 0.0;
            for (int r = 0; r < 3; ++r) s += R[3 * c2 + r] * acc12[9 + r];
            if (it.g_trans) it.g_trans[c2] += (float)(-s);
        }
        if (it.g_focal) it.g_focal[0] += (float)from_fix(small[0]);
    }
    if (it.g_light)
        for (int k = t; k < 3 * NL; k += blockDim.x) it.g_light[k] += (float)from_fix(small[1 + k]);
    if (it.g_env)
        for (int k = t; k < 3 * it.S.env_size * it.S.env_size; k += blockDim.x)
            it.g_env[k] += (float)from_fix(small[FR_ENV_OFF + k]);
    if (it.S.stage)
        for (int k = t; k < 4 * NL; k += blockDim.x) {
            const int j = k >> 2, q = k & 3;
            const float g = (float)from_fix(small[FR_GEO_OFF + k]);
            if (q == 0) { if (it.g_light_d) it.g_light_d[j] += g; }
            else if (q == 1) { if (it.g_light_a) it.g_light_a[j] += g; }
            else if (it.g_light_p) it.g_light_p[2 * j + q - 2] += g;
        }
}

// Lights of the virtual light stage (Sec. 3.3) from each item's parameters:
// light j is face j of the unit polyhedron (V0, V1, V2 about the stage centre
// C) scaled by d_j, shrunk by sqrt(a_j) about P = C + d_j (p0 V0 + p1 V1 + p2
// V2), p2 = 1 - p0 - p1, parallel to the face and emitting towards C: a
// triangle with vertices P + s (V0 - G), P + s (V2 - G), P + s (V1 - G),
// s = sqrt(a_j) d_j, G the face centroid; radiance scale d_j^2 / a_j.
__global__ void k_stage_lights(const DevItem* items, int NL) {
    const DevItem& it = items[blockIdx.y];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (!it.S.stage || j >= NL) return;
    const float* g = it.S.stage + 12 * j;
    const float3 C = f3(g[0], g[1], g[2]), A = f3(g[3], g[4], g[5]), B = f3(g[6], g[7], g[8]);
    const float3 V = f3(g[9], g[10], g[11]);
    const float d = it.P.light_d[j], a = it.P.light_a[j];
    const float p0 = it.P.light_p[2 * j], p1 = it.P.light_p[2 * j + 1], p2 = 1.0f - p0 - p1;
    const float3 G = (A + B + V) * (1.0f / 3.0f);
    const float3 P = C + (A * p0 + B * p1 + V * p2) * d;
    const float s = sqrtf(a) * d;
    const float3 t0 = P + (A - G) * s, t1 = P + (V - G) * s, t2 = P + (B - G) * s;
    LightDev L;
    L.type = 1;
    L.env = 0;
    L.c = t0;
    L.e1 = t1 - t0;
    L.e2 = t2 - t0;
    const float3 cr = cross(L.e1, L.e2);
    const float cl = length(cr);
    L.n = cr * (1.0f / cl);
    L.area = 0.5f * cl;
    L.scale = d * d / a;
    it.lights_w[j] = L;
}

// dE/dcoef_k = sum_i basis[k][i] dE/dv_i, one block per (k, item), FP64 accumulation.
__global__ void k_philox(uint2 key, const uint4* counters, int n, uint4* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = philox4x32_10(key, counters[i]);
}

int nb(long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void launch_set_items(const DevItem* host_items, int n, DevItem* dev_items, cudaStream_t st) {
    // the table travels as kernel parameters, ITEMS_PER_LAUNCH items per launch
    for (int k0 = 0; k0 < n; k0 += ITEMS_PER_LAUNCH) {
        ItemsParam p;
        p.n = std::min(ITEMS_PER_LAUNCH, n - k0);
        for (int k = 0; k < p.n; ++k) p.it[k] = host_items[k0 + k];
        k_set_items<<<1, 256, 0, st>>>(p, dev_items + k0);
        fr_count_launches(1);
    }
}

void launch_zero_accumulators(const DevItem* items, int n, int N, int M, cudaStream_t st) {
    k_zero_acc<<<dim3(nb(std::max(3L * N, 7L * M * M), 256), n), 256, 0, st>>>(items, N, M);
    fr_count_launches(1);
}

void launch_tex_flush(const DevItem* items, int n, int M, cudaStream_t st) {
    k_tex_flush<<<dim3(nb(7L * M * M, 256), n), 256, 0, st>>>(items, M);
    fr_count_launches(1);
}

void launch_stage_lights(const DevItem* items, int n, int NL, cudaStream_t st) {
    k_stage_lights<<<dim3(nb(NL, 128), n), 128, 0, st>>>(items, NL);
    fr_count_launches(1);
}

void launch_pose(const DevItem* items, int n, int N, cudaStream_t st) {
    k_aabb_reset<<<n, 32, 0, st>>>(items);
    k_pose<<<dim3(nb(N, 256), n), 256, 0, st>>>(items, N);
    fr_count_launches(2);
}

void launch_faces(const DevItem* items, int n, const int4* faces, int T, cudaStream_t st) {
    k_faces<<<dim3(nb(T, 256), n), 256, 0, st>>>(items, faces, T);
    fr_count_launches(1);
}

void launch_vertex_normals(const DevItem* items, int n, const int* vf_off, const int* vf_idx, int N,
                           cudaStream_t st) {
    k_vertex_normals<<<dim3(nb(N, 256), n), 256, 0, st>>>(items, vf_off, vf_idx, N);
    fr_count_launches(1);
}

void launch_normals_adjoint(const DevItem* items, int n, const int4* faces, const int* vf_off,
                            const int* vf_idx, int N, cudaStream_t st) {
    k_normals_adj_a<<<dim3(nb(N, 256), n), 256, 0, st>>>(items, N);
    k_normals_adj_b<<<dim3(nb(N, 256), n), 256, 0, st>>>(items, faces, vf_off, vf_idx, N);
    fr_count_launches(2);
}

void launch_pose_adjoint(const DevItem* items, int n, int N, cudaStream_t st) {
    k_pose_adj<<<dim3(nb(N, 256), n), 256, 0, st>>>(items, N);
    fr_count_launches(1);
}

void launch_pose_finish(const DevItem* items, int n, int NL, int N, cudaStream_t st) {
    k_pose_finish<<<n, 12 * 16, 0, st>>>(items, NL, nb(N, 256));
    fr_count_launches(1);
}

void launch_philox(uint32_t k0, uint32_t k1, const uint32_t* counters, int n, uint32_t* out, cudaStream_t st) {
    if (n <= 0) return;
    k_philox<<<nb(n, 256), 256, 0, st>>>(make_uint2(k0, k1), reinterpret_cast<const uint4*>(counters), n,
                                         reinterpret_cast<uint4*>(out));
    fr_count_launches(1);
}
