// Ray traversal of the binary BVH (the mesh's static SAH topology refitted per
// call, or an LBVH rebuilt per call) with a per-thread stack, and the
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

// The same watertight test for an any-hit query: true when the ray hits the
// triangle at some t in the open interval (tmin, tmax).  T and det share their
// sign at a hit, so the bounds are checked on T against tmin * det and
// tmax * det, without the division (the decision can differ from comparing
// T / det only within rounding of an end of the interval).
FR_D bool hit_triangle_any(const RayPre& r, float3 v0, float3 v1, float3 v2, float tmin, float tmax) {
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
    return det > 0.0f ? (T > tmin * det && T < tmax * det) : (T < tmin * det && T > tmax * det);
}

FR_D bool box_hit(const RayPre& r, float3 lo, float3 hi, float tmin, float tmax, float& tnear) {
    const float tx0 = fmaf(lo.x, r.inv.x, r.ood.x), tx1 = fmaf(hi.x, r.inv.x, r.ood.x);
    const float ty0 = fmaf(lo.y, r.inv.y, r.ood.y), ty1 = fmaf(hi.y, r.inv.y, r.ood.y);
    const float tz0 = fmaf(lo.z, r.inv.z, r.ood.z), tz1 = fmaf(hi.z, r.inv.z, r.ood.z);
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tmin));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    tnear = tn;
    return tn <= tf;
}

struct Hit {
    float t, b1, b2;
    int tri;   // original triangle index, -1 on a miss
    int slot;  // its leaf slot in the BVH (-1 on a miss)
};

FR_D void load_node(const BvhNode* nodes, int i, float3& lo0, float3& hi0, float3& lo1, float3& hi1,
                    int& c0, int& c1) {
    const float4 a = __ldg(&nodes[i].a), b = __ldg(&nodes[i].b), c = __ldg(&nodes[i].c);
    const int4 d = __ldg(&nodes[i].d);
    lo0 = f3(a.x, a.y, a.z);
    hi0 = f3(a.w, b.x, b.y);
    lo1 = f3(b.z, b.w, c.x);
    hi1 = f3(c.y, c.z, c.w);
    c0 = d.x;
    c1 = d.y;
}

// A thread's traversal stack: its own local array (stride 1, the default) or
// its column of a [FR_STACK][blockDim] shared array.
struct Stack {
    int* base;
    int stride;
    FR_D void put(int i, int v) { base[i * stride] = v; }
    FR_D int get(int i) const { return base[i * stride]; }
};

// A traversal stack: its entries live in the Stack's memory.  (Holding the top
// entry in a register, so that a pop's load overlaps the popped subtree, was
// measured 1.5% slower on the paper-scale face: more spills at the register cap.)
struct TravStack {
    Stack mem;
    int sp = 0;
    FR_D bool full() const { return sp >= FR_STACK; }
    FR_D bool empty() const { return sp == 0; }
    FR_D void push(int v) { mem.put(sp++, v); }
    FR_D int pop() { return mem.get(--sp); }
};

// Closest hit in (tmin, tmax); ties on t go to the lower triangle index.
FR_D Hit trace_closest(const DevScene& s, const RayPre& r, float tmin, float tmax, Stack st, RayStats& rs) {
    rs.rays++;
    Hit h;
    h.t = tmax;
    h.tri = h.slot = -1;
    h.b1 = h.b2 = 0.0f;
    TravStack ts{st};
    int node = 0;
    // a valid tree visits each of its 2T - 1 nodes at most once per ray
    for (int guard = 2 * s.T + 8; guard > 0; --guard) {
        float3 lo0, hi0, lo1, hi1;
        int c0, c1;
        load_node(s.nodes, node, lo0, hi0, lo1, hi1, c0, c1);
        rs.nodes++;
        float tn0, tn1;
        bool h0 = box_hit(r, lo0, hi0, tmin, h.t, tn0);
        bool h1 = box_hit(r, lo1, hi1, tmin, h.t, tn1);
        // leaves are single triangles: test the ones this ray enters right away,
        // in child order, by one loop (lanes entering different leaves test
        // them together)
        int leaf = -1, leaf2 = -1;
        if (h0 && c0 < 0) {
            leaf = ~c0;
            h0 = false;
        }
        if (h1 && c1 < 0) {
            if (leaf < 0) leaf = ~c1;
            else leaf2 = ~c1;
            h1 = false;
        }
        while (leaf >= 0) {
            const float4 a = __ldg(&s.tris[3 * leaf]), b = __ldg(&s.tris[3 * leaf + 1]), c = __ldg(&s.tris[3 * leaf + 2]);
            float t, b1, b2;
            const int id = __float_as_int(a.w);
            rs.tris++;
            if (hit_triangle(r, xyz(a), xyz(b), xyz(c), tmin, h.t, t, b1, b2) &&
                (t < h.t || id < h.tri || h.tri < 0)) {
                h.t = t; h.b1 = b1; h.b2 = b2; h.tri = id; h.slot = leaf;
            }
            leaf = leaf2;
            leaf2 = -1;
        }
        if (h0 && tn0 > h.t) h0 = false;
        if (h1 && tn1 > h.t) h1 = false;
        if (h0 && h1) {
            int near = c0, far = c1;
            if (tn1 < tn0) { near = c1; far = c0; }
            if (ts.full()) { set_status(s.status, FR_STATUS_STACK_OVERFLOW); return h; }
            ts.push(far);
            node = near;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (ts.empty()) return h;
            node = ts.pop();
        }
    }
    set_status(s.status, FR_STATUS_BAD_BVH);
    return h;
}

// Closest-hit result of a camera ray whose hit triangle is known from a record
// of the same ray: the same watertight test on the same triangle reproduces
// the traversal's t and barycentrics.  tri < 0 is a miss.
FR_D Hit hit_record(const DevScene& s, const RayPre& r, int tri) {
    Hit h;
    h.t = INFINITY;
    h.tri = h.slot = -1;
    h.b1 = h.b2 = 0.0f;
    if (tri < 0) return h;
    const int4 fc = __ldg(&s.faces[tri]);
    float t, b1, b2;
    if (hit_triangle(r, xyz(__ldg(&s.v[fc.x])), xyz(__ldg(&s.v[fc.y])), xyz(__ldg(&s.v[fc.z])), 0.0f, INFINITY, t, b1,
                     b2)) {
        h.t = t; h.b1 = b1; h.b2 = b2; h.tri = tri; h.slot = __ldg(&s.slot_of[tri]);
    }
    return h;
}

// Any hit in (tmin, tmax), skipping the triangle in leaf slot `skip_slot`
// (the shading triangle of a shadow ray): comparing slots needs no load, so a
// leaf's three vertex rows are fetched together.
FR_D bool trace_any(const DevScene& s, const RayPre& r, float tmin, float tmax, int skip_slot, Stack st,
                    RayStats& rs) {
    rs.rays++;
    TravStack ts{st};
    int node = 0;
    for (int guard = 2 * s.T + 8; guard > 0; --guard) {
        float3 lo0, hi0, lo1, hi1;
        int c0, c1;
        load_node(s.nodes, node, lo0, hi0, lo1, hi1, c0, c1);
        rs.nodes++;
        float tn0, tn1;
        bool h0 = box_hit(r, lo0, hi0, tmin, tmax, tn0);
        bool h1 = box_hit(r, lo1, hi1, tmin, tmax, tn1);
        // the leaf children this ray enters, tested in child order by one loop,
        // so that lanes entering different leaves test them together
        int leaf = -1, leaf2 = -1;
        if (h0 && c0 < 0) {
            leaf = ~c0;
            h0 = false;
        }
        if (h1 && c1 < 0) {
            if (leaf < 0) leaf = ~c1;
            else leaf2 = ~c1;
            h1 = false;
        }
        while (leaf >= 0) {
            if (leaf != skip_slot) {
                const float4 a = __ldg(&s.tris[3 * leaf]), b = __ldg(&s.tris[3 * leaf + 1]),
                             c = __ldg(&s.tris[3 * leaf + 2]);
                rs.tris++;
                if (hit_triangle_any(r, xyz(a), xyz(b), xyz(c), tmin, tmax)) return true;
            }
            leaf = leaf2;
            leaf2 = -1;
        }
        if (h0 && h1) {
            if (ts.full()) { set_status(s.status, FR_STATUS_STACK_OVERFLOW); return false; }
            // the nearer child first.  Measured on the paper-scale face: 2% faster
            // than a fixed child order although it visits 2% more nodes (the
            // farther child first: 2% fewer visits, 5% slower), as the lanes of
            // a warp, whose shadow rays start close together, keep taking the
            // same child
            int near = c0, far = c1;
            if (tn1 < tn0) { near = c1; far = c0; }
            ts.push(far);
            node = near;
        } else if (h0) {
            node = c0;
        } else if (h1) {
            node = c1;
        } else {
            if (ts.empty()) return false;
            node = ts.pop();
        }
    }
    set_status(s.status, FR_STATUS_BAD_BVH);
    return false;
}
