// Ray traversal of the LBVH with a per-thread stack in shared memory, and the
// watertight ray/triangle test of Woop, Benthin and Wald (JCGT 2013): FP32 edge
// functions, re-evaluated in FP64 when one of them is exactly zero.
#pragma once
#include "common.cuh"

struct RayPre {
    float3 o, d, inv, ood;     // ood = -o * inv, so a slab distance is one FMA
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

FR_D RayPre ray_setup(float3 o, float3 d) {
    RayPre r;
    r.o = o;
    r.d = d;
    const float ex = fabsf(d.x) > 1e-30f ? d.x : copysignf(1e-30f, d.x);
    const float ey = fabsf(d.y) > 1e-30f ? d.y : copysignf(1e-30f, d.y);
    const float ez = fabsf(d.z) > 1e-30f ? d.z : copysignf(1e-30f, d.z);
    r.inv = f3(1.0f / ex, 1.0f / ey, 1.0f / ez);
    r.ood = f3(-o.x * r.inv.x, -o.y * r.inv.y, -o.z * r.inv.z);
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    r.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    r.kx = r.kz == 2 ? 0 : r.kz + 1;
    r.ky = r.kx == 2 ? 0 : r.kx + 1;
    if (comp(d, r.kz) < 0.0f) { int t = r.kx; r.kx = r.ky; r.ky = t; }
    r.Sz = 1.0f / comp(d, r.kz);
    r.Sx = comp(d, r.kx) * r.Sz;
    r.Sy = comp(d, r.ky) * r.Sz;
    return r;
}

// Watertight test.  On a hit with tmin < t <= tmax returns true with t and the
// barycentrics (b1, b2) of v1, v2 (hit = b0 v0 + b1 v1 + b2 v2); both facings
// are accepted.
FR_D bool hit_triangle(const RayPre& r, float3 v0, float3 v1, float3 v2, float tmin, float tmax,
                       float& t, float& b1, float& b2) {
    const float3 A = v0 - r.o, B = v1 - r.o, C = v2 - r.o;
    const float Akz = comp(A, r.kz), Bkz = comp(B, r.kz), Ckz = comp(C, r.kz);
    const float Ax = comp(A, r.kx) - r.Sx * Akz, Ay = comp(A, r.ky) - r.Sy * Akz;
    const float Bx = comp(B, r.kx) - r.Sx * Bkz, By = comp(B, r.ky) - r.Sy * Bkz;
    const float Cx = comp(C, r.kx) - r.Sx * Ckz, Cy = comp(C, r.ky) - r.Sy * Ckz;
    float U = Cx * By - Cy * Bx;
    float V = Ax * Cy - Ay * Cx;
    float W = Bx * Ay - By * Ax;
    if (U == 0.0f || V == 0.0f || W == 0.0f) {
        U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
        V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
        W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
    }
    if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return false;
    const float det = U + V + W;
    if (det == 0.0f) return false;
    const float T = U * (r.Sz * Akz) + V * (r.Sz * Bkz) + W * (r.Sz * Ckz);
    const float inv = 1.0f / det;
    t = T * inv;
    if (!(t > tmin && t <= tmax)) return false;
    b1 = V * inv;
    b2 = W * inv;
    return true;
}

struct Hit {
    float t, b1, b2;
    int tri;   // original triangle index, -1 on a miss
};

// stack: this thread's column of a [FR_STACK][blockDim] shared array.
struct Stack {
    int* base;
    int stride;
    FR_D void put(int i, int v) { base[i * stride] = v; }
    FR_D int get(int i) const { return base[i * stride]; }
};

// Slab tests of a wide node's four child boxes against (tmin, tmax]:
// tn[k] = entry distance, or +inf when child k is missed or absent.
FR_D void wide_boxes(const BvhNode* node, const RayPre& r, float tmin, float tmax, float tn[4], int code[4]) {
    const float4 lx = __ldg(&node->lox), ly = __ldg(&node->loy), lz = __ldg(&node->loz);
    const float4 hx = __ldg(&node->hix), hy = __ldg(&node->hiy), hz = __ldg(&node->hiz);
    const int4 ch = __ldg(&node->child);
    const float lxa[4] = {lx.x, lx.y, lx.z, lx.w}, lya[4] = {ly.x, ly.y, ly.z, ly.w}, lza[4] = {lz.x, lz.y, lz.z, lz.w};
    const float hxa[4] = {hx.x, hx.y, hx.z, hx.w}, hya[4] = {hy.x, hy.y, hy.z, hy.w}, hza[4] = {hz.x, hz.y, hz.z, hz.w};
    code[0] = ch.x; code[1] = ch.y; code[2] = ch.z; code[3] = ch.w;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float tx0 = fmaf(lxa[k], r.inv.x, r.ood.x), tx1 = fmaf(hxa[k], r.inv.x, r.ood.x);
        const float ty0 = fmaf(lya[k], r.inv.y, r.ood.y), ty1 = fmaf(hya[k], r.inv.y, r.ood.y);
        const float tz0 = fmaf(lza[k], r.inv.z, r.ood.z), tz1 = fmaf(hza[k], r.inv.z, r.ood.z);
        const float tn_ = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
        const float tf_ = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
        tn[k] = (tn_ <= tf_ && code[k] != FR_EMPTY_CHILD) ? tn_ : INFINITY;
    }
}

FR_D void cswap(float& ta, int& ca, float& tb, int& cb) {
    if (tb < ta) {
        const float t = ta; ta = tb; tb = t;
        const int c = ca; ca = cb; cb = c;
    }
}

// Closest hit in (tmin, tmax]; ties on t go to the lower triangle index.
FR_D Hit trace_closest(const DevScene& s, const RayPre& r, float tmin, float tmax, Stack st, RayStats& rs) {
    rs.rays++;
    Hit h;
    h.t = tmax;
    h.tri = -1;
    h.b1 = h.b2 = 0.0f;
    int sp = 0;
    int node = 0;
    // a valid tree visits each of its T - 1 wide nodes at most once per ray
    for (int guard = s.T + 8; guard > 0; --guard) {
        rs.nodes++;
        float tn[4];
        int code[4];
        wide_boxes(&s.nodes[node], r, tmin, h.t, tn, code);
        // leaves are single triangles: test them right away
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (tn[k] < INFINITY && code[k] < 0) {
                const int slot = ~code[k];
                const float4 a = __ldg(&s.tris[3 * slot]), b = __ldg(&s.tris[3 * slot + 1]), c = __ldg(&s.tris[3 * slot + 2]);
                float t, b1, b2;
                const int id = __float_as_int(a.w);
                rs.tris++;
                if (hit_triangle(r, xyz(a), xyz(b), xyz(c), tmin, h.t, t, b1, b2) &&
                    (t < h.t || id < h.tri || h.tri < 0)) {
                    h.t = t; h.b1 = b1; h.b2 = b2; h.tri = id;
                }
                tn[k] = INFINITY;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (tn[k] > h.t) tn[k] = INFINITY;
        // order the internal children near to far
        cswap(tn[0], code[0], tn[1], code[1]);
        cswap(tn[2], code[2], tn[3], code[3]);
        cswap(tn[0], code[0], tn[2], code[2]);
        cswap(tn[1], code[1], tn[3], code[3]);
        cswap(tn[1], code[1], tn[2], code[2]);
        const int cnt = (tn[0] < INFINITY) + (tn[1] < INFINITY) + (tn[2] < INFINITY) + (tn[3] < INFINITY);
        if (cnt == 0) {
            if (sp == 0) return h;
            node = st.get(--sp);
            continue;
        }
        if (sp + cnt - 1 > FR_STACK) { set_status(s.status, FR_STATUS_STACK_OVERFLOW); return h; }
        for (int k = cnt - 1; k >= 1; --k) st.put(sp++, code[k]);
        node = code[0];
    }
    set_status(s.status, FR_STATUS_BAD_BVH);
    return h;
}

// Any hit in (tmin, tmax), skipping triangle `skip` (shadow rays).
FR_D bool trace_any(const DevScene& s, const RayPre& r, float tmin, float tmax, int skip, Stack st,
                    RayStats& rs) {
    rs.rays++;
    int sp = 0;
    int node = 0;
    for (int guard = s.T + 8; guard > 0; --guard) {
        rs.nodes++;
        float tn[4];
        int code[4];
        wide_boxes(&s.nodes[node], r, tmin, tmax, tn, code);
        int next = -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!(tn[k] < INFINITY)) continue;
            if (code[k] < 0) {
                const int slot = ~code[k];
                const float4 a = __ldg(&s.tris[3 * slot]);
                if (__float_as_int(a.w) != skip) {
                    const float4 b = __ldg(&s.tris[3 * slot + 1]), c = __ldg(&s.tris[3 * slot + 2]);
                    float t, b1, b2;
                    rs.tris++;
                    if (hit_triangle(r, xyz(a), xyz(b), xyz(c), tmin, tmax, t, b1, b2) && t < tmax) return true;
                }
            } else if (next < 0) {
                next = code[k];
            } else {
                if (sp >= FR_STACK) { set_status(s.status, FR_STATUS_STACK_OVERFLOW); return false; }
                st.put(sp++, code[k]);
            }
        }
        if (next < 0) {
            if (sp == 0) return false;
            next = st.get(--sp);
        }
        node = next;
    }
    set_status(s.status, FR_STATUS_BAD_BVH);
    return false;
}
