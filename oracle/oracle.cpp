// FP64 CPU oracle for the differentiable Monte Carlo ray-traced face render of
// Dib et al., "Practical Face Reconstruction via Differentiable Ray Tracing"
// (Eurographics 2021).
//
// TEST INFRASTRUCTURE ONLY.  Tests, the smoke check and the benchmark's CPU
// baseline load this library; the product path never does.  It shares no code,
// header, table or helper with the CUDA library: both sides implement the same
// published definitions (Philox4x32-10, the paper's equations) independently.
//
// Plain and slow on purpose: brute-force ray/triangle tests over every triangle,
// forward-mode dual numbers for every geometric derivative, straightforward
// loops.  Each function cites the part of the paper it follows.
//
// Readings of places where the paper is silent or garbled (all in one place):
//  * D (App. A, Eq. brdf_d): exponent 2/r - 2 with the normalising constant of
//    that exponent, (2/r)/(2 pi) = 1/(pi r).
//  * h (Eq. halfVector): (l + o)/|l + o|.
//  * F (Eq. brdf_f): Schlick's approximation with the fifth power (flag
//    ORA_SCHLICK_LINEAR gives the printed linear form).
//  * Contributions vanish unless n_s.l > 0; the specular lobe also needs
//    n_s.o > 0 (the denominator of Eq. brdf_spec); the Lambert term does not
//    depend on the view.  Surfaces are one-sided: a hit on a triangle whose
//    geometric normal faces away from the camera reflects nothing.  (Flag
//    ORA_VIEW_CUTOFF zeroes every contribution where n_s.o <= 0.)
//  * The lobe does not vanish as n_s.o -> 0+ (G1(o) / (n_s.o) has a finite
//    limit), so the image jumps on the curve n_s.o = 0 inside front-facing
//    triangles whose interpolated normals turn away from the camera.  Edge
//    sampling (Sec. 4) is applied to that curve too (ORA_TERM_SPECULAR): it is
//    found along image scanlines (one horizontal line per pixel row and one
//    vertical line per pixel column, edge_spp of each, at uniform offsets), and
//    each crossing is weighted by the share (n_x^2 on rows, n_y^2 on columns)
//    of the curve's unit normal n, so that the two families sum to the line
//    integral with a bounded weight everywhere on the curve.
//  * Eq. lightIntensity: emitted radiance L_j = (d_j^2 / a_j) i_j; emitter
//    geometry is given explicitly in camera space and does not depend on pose.
//  * One area sample per light per pixel sample (light-area importance
//    sampling); miss = black background; pixel = box filter over the pixel.
//  * Blur (Sec. 4 "Variance Reduction"): normalised 3x3 Gaussian, sigma 1,
//    replicate border; loss = L1 over pixels and channels (Eq. energy).
//  * Pose (Sec. 3.1): R = Rz Ry Rx from Euler angles, v' = R^T (v - T);
//    camera at the origin looking down -z, focal length f in pixels, principal
//    point at the image centre, image y down.
//  * Vertex normals: normalised sum of the un-normalised face normals.
//  * Textures: bilinear, texel centres at u*M - 1/2, clamp-to-edge.
//  * Shadow rays skip the shading triangle and count occluders with
//    1e-4 < t < 1 - 1e-4 along the segment y -> z.
//  * Closest-hit ties go to the lower triangle index.
//  * Environment map (Sec. 7, environment map vs light stage): each texel of
//    an M_e x M_e latitude-longitude map is a light at infinity whose
//    radiance is the texel's RGB value.  The map is split into blocks of
//    texels, one emitter record each; every camera sample draws one direction
//    per block: a texel uniformly among the block's, then a direction uniform
//    in solid angle inside it (estimator weight = texels x texel solid angle).
//    Shadow rays follow the direction with t > 1e-4.  The visibility boundary
//    lies on the sphere of directions: the projection from y of the occluder's
//    silhouette edges, with the same edge-sampling estimator as the area
//    lights (arc length and normal velocity measured on the unit sphere).
#include "oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// definition: ten rounds of two 32x32->64 multiplies with a Weyl key schedule.
// ---------------------------------------------------------------------------
void philox4x32_10(uint32_t k0, uint32_t k1, uint32_t c[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
}

// Sample stream: key = (seed, stream tag); counter = (index, (sample<<16)|block,
// iteration, face).  Dimension d comes from block d/4, word d%4, and becomes the
// uniform (x >> 8) * 2^-24.
struct Stream {
    uint32_t key0, key1, index, sample, iteration, face;
    int cached_block = -1;
    uint32_t words[4] = {0, 0, 0, 0};
    double u(int dim) {
        int block = dim >> 2;
        if (block != cached_block) {
            words[0] = index;
            words[1] = (sample << 16) | (uint32_t)block;
            words[2] = iteration;
            words[3] = face;
            philox4x32_10(key0, key1, words);
            cached_block = block;
        }
        return (double)(words[dim & 3] >> 8) * (1.0 / 16777216.0);
    }
};

enum { STREAM_PRIMARY = 0, STREAM_EDGE_PRIMARY = 1, STREAM_EDGE_SHADOW = 2, STREAM_EDGE_SPECULAR = 3 };

// ---------------------------------------------------------------------------
// Forward-mode dual numbers: value plus derivatives w.r.t. the active slots.
// ---------------------------------------------------------------------------
constexpr int DMAX = 256;
thread_local int g_nd = 0;  // active derivative slots on this thread (0: values only)

struct D {
    double v;
    double d[DMAX];
    D() : v(0.0) { for (int i = 0; i < g_nd; ++i) d[i] = 0.0; }
    D(double x) : v(x) { for (int i = 0; i < g_nd; ++i) d[i] = 0.0; }
    D(const D& o) : v(o.v) { for (int i = 0; i < g_nd; ++i) d[i] = o.d[i]; }
    D& operator=(const D& o) {
        v = o.v;
        for (int i = 0; i < g_nd; ++i) d[i] = o.d[i];
        return *this;
    }
};
D seed_slot(double x, int slot) { D r(x); if (slot >= 0 && slot < g_nd) r.d[slot] = 1.0; return r; }
D operator+(const D& a, const D& b) { D r; r.v = a.v + b.v; for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
D operator-(const D& a, const D& b) { D r; r.v = a.v - b.v; for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
D operator-(const D& a) { D r; r.v = -a.v; for (int i = 0; i < g_nd; ++i) r.d[i] = -a.d[i]; return r; }
D operator*(const D& a, const D& b) { D r; r.v = a.v * b.v; for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
D operator/(const D& a, const D& b) {
    D r; r.v = a.v / b.v;
    double ib = 1.0 / b.v;
    for (int i = 0; i < g_nd; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
    return r;
}
D operator+(const D& a, double b) { D r(a); r.v += b; return r; }
D operator+(double a, const D& b) { return b + a; }
D operator-(const D& a, double b) { D r(a); r.v -= b; return r; }
D operator-(double a, const D& b) { D r = -b; r.v += a; return r; }
D operator*(const D& a, double b) { D r; r.v = a.v * b; for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * b; return r; }
D operator*(double a, const D& b) { return b * a; }
D operator/(const D& a, double b) { return a * (1.0 / b); }
D operator/(double a, const D& b) { return D(a) / b; }
D dsqrt(const D& a) {
    D r; r.v = std::sqrt(a.v);
    double k = r.v > 0.0 ? 0.5 / r.v : 0.0;
    for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * k;
    return r;
}
D dexp(const D& a) { D r; r.v = std::exp(a.v); for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * r.v; return r; }
D dlog(const D& a) { D r; r.v = std::log(a.v); for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] / a.v; return r; }
D dpow(const D& x, const D& e) { return dexp(e * dlog(x)); }     // x > 0
D dpowi(const D& x, int k) { D r(1.0); for (int i = 0; i < k; ++i) r = r * x; return r; }

struct V3 { D x, y, z; };
V3 v3(const D& x, const D& y, const D& z) { return V3{x, y, z}; }
V3 v3c(double x, double y, double z) { return V3{D(x), D(y), D(z)}; }
V3 operator+(const V3& a, const V3& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(const V3& a, const V3& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(const V3& a, const D& s) { return {a.x * s, a.y * s, a.z * s}; }
V3 operator*(const V3& a, double s) { return {a.x * s, a.y * s, a.z * s}; }
D dot(const V3& a, const V3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(const V3& a, const V3& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
D norm(const V3& a) { return dsqrt(dot(a, a)); }
V3 normalize(const V3& a) { D n = norm(a); return {a.x / n, a.y / n, a.z / n}; }

// plain double vectors
struct P3 { double x, y, z; };
P3 p3(double x, double y, double z) { return {x, y, z}; }
P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
P3 operator*(P3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
double dotp(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
P3 crossp(P3 a, P3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double normp(P3 a) { return std::sqrt(dotp(a, a)); }
P3 val(const V3& a) { return {a.x.v, a.y.v, a.z.v}; }

// ---------------------------------------------------------------------------
// Scene preparation: morph (Sec. 3.1), pose (Sec. 3.1), normals, edges.
// ---------------------------------------------------------------------------
struct Light {
    int type;
    P3 c, e1, e2, n;   // n = unit normal of the emitting side
    double area;
    double scale;      // d^2 / a of Eq. (lightIntensity)
    // virtual light stage (Sec. 3.3): geometry built from (d, a, p) as duals
    bool geo = false;
    V3 cd, e1d, e2d;   // c, e1, e2 with derivatives on the light's slots
    D aread, scaled;   // area and d^2 / a likewise
    // environment block (type ORA_LIGHT_ENV): texel rows [i0, i1), columns [j0, j1)
    int i0 = 0, i1 = 0, j0 = 0, j1 = 0;
};

struct Edge { int a, b, f1, f2; };  // a < b; f2 = -1 on the boundary

struct Prep {
    const OraScene* s;
    const OraParams* p;
    int N, T, K, NL, W, H, M, spp;
    int nd;                    // active dual slots (0: values only)
    int slot_rot, slot_trans, slot_focal, slot_c, slot_s, slot_r, slot_t;
    int slot_sx, slot_sy;      // screen coordinates of a fixed image point (boundary of the lobe)
    int slot_light;            // light j's (d, a, p0, p1) at slot_light + 4 j (-1: fixed lights)
    std::vector<P3> v;         // camera-space vertices
    std::vector<P3> vn;        // unit vertex normals
    std::vector<double> dv;    // [N][3][nd] derivatives of v (when nd > 0)
    std::vector<double> dn;    // [N][3][nd] derivatives of vn
    std::vector<Light> lights;
    std::vector<Edge> edges;
    std::vector<int> prim_sil;                 // ordered primary silhouette edges
    std::vector<std::vector<int>> light_cand;  // ordered shadow candidates per light
    double focal;
};

D coef_dual(const Prep& P, int k) { return seed_slot(P.p->coef[k], k); }

// R = Rz(tz) Ry(ty) Rx(tx) as duals; returns the nine entries row-major.
void rotation(const Prep& P, D R[9]) {
    D tx = seed_slot(P.p->rot[0], P.slot_rot + 0);
    D ty = seed_slot(P.p->rot[1], P.slot_rot + 1);
    D tz = seed_slot(P.p->rot[2], P.slot_rot + 2);
    // cos/sin of a dual
    auto dcos = [](const D& a) { D r; r.v = std::cos(a.v); double k = -std::sin(a.v); for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * k; return r; };
    auto dsin = [](const D& a) { D r; r.v = std::sin(a.v); double k = std::cos(a.v); for (int i = 0; i < g_nd; ++i) r.d[i] = a.d[i] * k; return r; };
    D cx = dcos(tx), sx = dsin(tx), cy = dcos(ty), sy = dsin(ty), cz = dcos(tz), sz = dsin(tz);
    D Rx[9] = {D(1.0), D(0.0), D(0.0), D(0.0), cx, -sx, D(0.0), sx, cx};
    D Ry[9] = {cy, D(0.0), sy, D(0.0), D(1.0), D(0.0), -sy, D(0.0), cy};
    D Rz[9] = {cz, -sz, D(0.0), sz, cz, D(0.0), D(0.0), D(0.0), D(1.0)};
    D Ryx[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            D acc(0.0);
            for (int k = 0; k < 3; ++k) acc = acc + Ry[3 * i + k] * Rx[3 * k + j];
            Ryx[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            D acc(0.0);
            for (int k = 0; k < 3; ++k) acc = acc + Rz[3 * i + k] * Ryx[3 * k + j];
            R[3 * i + j] = acc;
        }
}

// Camera-space vertex i as duals: v' = R^T (a_s + Sigma coef - T)  (Sec. 3.1).
V3 vertex_dual(const Prep& P, int i, const D R[9], const V3& T) {
    const OraScene* s = P.s;
    D w[3];
    for (int c = 0; c < 3; ++c) {
        D acc(s->mean[3 * i + c]);
        for (int k = 0; k < P.K; ++k) {
            double b = s->basis[(size_t)k * 3 * P.N + 3 * i + c];
            acc = acc + coef_dual(P, k) * b;
        }
        w[c] = acc;
    }
    V3 m = v3(w[0], w[1], w[2]) - T;
    // R^T m
    return v3(R[0] * m.x + R[3] * m.y + R[6] * m.z,
              R[1] * m.x + R[4] * m.y + R[7] * m.z,
              R[2] * m.x + R[5] * m.y + R[8] * m.z);
}

// Values and derivative rows ([i][3][stride]) of per-vertex dual vectors.
void store(std::vector<P3>& vals, std::vector<double>& ders, int stride, int i, const V3& a) {
    vals[i] = val(a);
    int nd = std::min(stride, g_nd);
    if (nd) {
        const D* comp[3] = {&a.x, &a.y, &a.z};
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < nd; ++q) ders[((size_t)i * 3 + c) * stride + q] = comp[c]->d[q];
    }
}

V3 load(const std::vector<P3>& vals, const std::vector<double>& ders, int stride, int i) {
    V3 r = v3c(vals[i].x, vals[i].y, vals[i].z);
    int nd = std::min(stride, g_nd);
    if (nd) {
        D* comp[3] = {&r.x, &r.y, &r.z};
        for (int c = 0; c < 3; ++c)
            for (int q = 0; q < nd; ++q) comp[c]->d[q] = ders[((size_t)i * 3 + c) * stride + q];
    }
    return r;
}

// Interleaved loop over [0, n) on n_threads threads; workers inherit the
// caller's active dual slot count.
template <class F>
void parallel_for(int n_threads, int n, F fn) {
    if (n_threads <= 1 || n < 2) { for (int i = 0; i < n; ++i) fn(i, 0); return; }
    std::vector<std::thread> th;
    const int nd = g_nd;
    for (int t = 0; t < n_threads; ++t)
        th.emplace_back([&, t, nd]() { g_nd = nd; for (int i = t; i < n; i += n_threads) fn(i, t); });
    for (auto& x : th) x.join();
}

int threads_of(const OraScene* s) {
    int n = s->n_threads;
    if (n <= 0) n = (int)std::thread::hardware_concurrency();
    return std::max(1, n);
}

bool stage_lights(const OraScene* s, const OraParams* p) {
    return s->stage && p && p->light_d && p->light_a && p->light_p;
}

// Light j of the virtual light stage (Sec. 3.3) from its parameters: the face
// (V0, V1, V2) of the unit polyhedron scaled by d_j about the stage centre C,
// shrunk by sqrt(a_j) about the point with barycentric coordinates
// (p0, p1, 1 - p0 - p1), parallel to the face, emitting towards C: vertices
// P + s (V0 - G), P + s (V2 - G), P + s (V1 - G) with G the face centroid,
// P = C + d (p0 V0 + p1 V1 + p2 V2), s = sqrt(a) d; area a d^2 F (F the unit
// face area) and L_j = (d^2 / a) i_j.  Derivatives ride on the light's slots.
void build_stage_light(Prep& P, int j) {
    const float* g = P.s->stage + 12 * j;
    const int b = P.slot_light + 4 * j;
    D d = seed_slot(P.p->light_d[j], b), a = seed_slot(P.p->light_a[j], b + 1);
    D p0 = seed_slot(P.p->light_p[2 * j], b + 2), p1 = seed_slot(P.p->light_p[2 * j + 1], b + 3);
    D p2 = 1.0 - p0 - p1;
    V3 C = v3c(g[0], g[1], g[2]);
    V3 A = v3c(g[3], g[4], g[5]), B = v3c(g[6], g[7], g[8]), Cv = v3c(g[9], g[10], g[11]);
    V3 G = (A + B + Cv) * (1.0 / 3.0);
    V3 Pc = C + (A * p0 + B * p1 + Cv * p2) * d;
    D sz = dsqrt(a) * d;
    V3 t0 = Pc + (A - G) * sz, t1 = Pc + (Cv - G) * sz, t2 = Pc + (B - G) * sz;
    Light L;
    L.type = 1;
    L.geo = true;
    L.cd = t0;
    L.e1d = t1 - t0;
    L.e2d = t2 - t0;
    L.c = val(L.cd);
    L.e1 = val(L.e1d);
    L.e2 = val(L.e2d);
    P3 cr = crossp(L.e1, L.e2);
    double cl = normp(cr);
    L.n = cr * (1.0 / cl);                       // independent of (d, a, p)
    V3 crd = cross(L.e1d, L.e2d);
    L.aread = norm(crd) * 0.5;
    L.area = L.aread.v;
    L.scaled = d * d / a;
    L.scale = L.scaled.v;
    P.lights[j] = L;
}

// Emitter sample of a stage light with its derivatives (triangle mapping of
// light_point).
V3 light_point_d(const Light& L, double u, double v) {
    double su = std::sqrt(u);
    return L.cd + L.e1d * (su * (1.0 - v)) + L.e2d * (su * v);
}

// ---------------------------------------------------------------------------
// Environment-map emitters (Sec. 7): row i of the M_e x M_e map covers polar
// angles [i, i + 1] pi / M_e from +y, column j azimuths [j, j + 1] 2 pi / M_e
// from +z towards +x; w(theta, phi) = (sin theta sin phi, cos theta,
// sin theta cos phi).
// ---------------------------------------------------------------------------
double band_cos(int i, int Me) { return std::cos(M_PI * i / Me); }

// Exact range [lo, hi] of n . w over the directions of an environment block
// (rows [i0, i1), columns [j0, j1)).  With w = (sin t sin p, cos t, sin t cos p),
// n . w = n_y cos t + sin t A(p), A(p) = n_x sin p + n_z cos p.  A ranges over
// its values at the azimuth ends and at its extremes p = atan2(n_x, n_z) + k pi
// inside; sin t >= 0, so the minimum over the block takes A's minimum and the
// maximum A's maximum, and each is then a sinusoid in t whose extremes over
// [t0, t1] are at the ends or at its stationary points atan2(A, n_y) + k pi.
void env_range(const Light& L, int Me, P3 n, double& lo, double& hi) {
    const double t0 = M_PI * L.i0 / Me, t1 = M_PI * L.i1 / Me;
    const double f0 = 2.0 * M_PI * L.j0 / Me, f1 = 2.0 * M_PI * L.j1 / Me;
    auto A = [&](double p) { return n.x * std::sin(p) + n.z * std::cos(p); };
    double a_lo = std::min(A(f0), A(f1)), a_hi = std::max(A(f0), A(f1));
    const double pa = std::atan2(n.x, n.z);
    for (int k = -2; k <= 3; ++k) {
        const double p = pa + k * M_PI;
        if (p > f0 && p < f1) { a_lo = std::min(a_lo, A(p)); a_hi = std::max(a_hi, A(p)); }
    }
    auto g_ext = [&](double a, bool want_min) {
        auto g = [&](double t) { return n.y * std::cos(t) + a * std::sin(t); };
        double r = want_min ? std::min(g(t0), g(t1)) : std::max(g(t0), g(t1));
        const double tc = std::atan2(a, n.y);
        for (int k = -1; k <= 2; ++k) {
            const double t = tc + k * M_PI;
            if (t > t0 && t < t1) r = want_min ? std::min(r, g(t)) : std::max(r, g(t));
        }
        return r;
    };
    lo = g_ext(a_lo, true);
    hi = g_ext(a_hi, false);
}

// One direction of an environment block: a texel uniformly among the block's
// R x C (row = floor(k_u R / 2^24) from the 24-bit integer k_u behind u, the
// remainder placing the sample inside the row; columns likewise from v), then
// uniform in solid angle inside the texel (cos theta and phi uniform).
// weight = 1 / pdf = R C Omega_texel, Omega_texel = (cos top - cos bottom) 2 pi / M_e.
struct EnvSample { int row, col; P3 w; double weight; };
EnvSample env_sample(const Light& L, int Me, double u, double v) {
    const uint64_t ku = (uint64_t)(u * 16777216.0), kv = (uint64_t)(v * 16777216.0);
    const int R = L.i1 - L.i0, C = L.j1 - L.j0;
    const uint64_t pu = ku * (uint64_t)R, pv = kv * (uint64_t)C;
    EnvSample e;
    e.row = L.i0 + (int)(pu >> 24);
    e.col = L.j0 + (int)(pv >> 24);
    const double fu = (double)(pu & 0xFFFFFFu) / 16777216.0, fv = (double)(pv & 0xFFFFFFu) / 16777216.0;
    const double zt = band_cos(e.row, Me), zb = band_cos(e.row + 1, Me);
    const double y = zt + fu * (zb - zt);
    const double sn = std::sqrt(std::max(0.0, 1.0 - y * y));
    const double phi = 2.0 * M_PI * (e.col + fv) / Me;
    e.w = p3(sn * std::sin(phi), y, sn * std::cos(phi));
    e.weight = (double)R * C * (zt - zb) * (2.0 * M_PI / Me);
    return e;
}

// Texel of the map that contains unit direction w.
void env_texel_of(P3 w, int Me, int& row, int& col) {
    const double th = std::acos(std::min(1.0, std::max(-1.0, w.y)));
    double ph = std::atan2(w.x, w.z);
    if (ph < 0.0) ph += 2.0 * M_PI;
    row = std::min(Me - 1, std::max(0, (int)std::floor(th * Me / M_PI)));
    col = std::min(Me - 1, std::max(0, (int)std::floor(ph * Me / (2.0 * M_PI))));
}

bool inside_env_block(const Light& L, int Me, P3 w) {
    int r, c;
    env_texel_of(w, Me, r, c);
    return r >= L.i0 && r < L.i1 && c >= L.j0 && c < L.j1;
}

// radiance of texel (row, col), channel k
double env_value(const Prep& P, int row, int col, int k) {
    return (double)P.p->env[3 * ((size_t)row * P.s->env_size + col) + k];
}

void prepare(Prep& P, const OraScene* s, const OraParams* p, int nd) {
    P.s = s; P.p = p;
    P.N = s->n_vertices; P.T = s->n_triangles; P.K = s->n_basis; P.NL = s->n_lights;
    P.W = s->width; P.H = s->height; P.M = s->tex_size; P.spp = s->spp;
    P.nd = nd;
    P.slot_rot = P.K; P.slot_trans = P.K + 3; P.slot_focal = P.K + 6;
    P.slot_c = P.K + 7; P.slot_s = P.K + 10; P.slot_r = P.K + 13; P.slot_t = P.K + 14;
    P.slot_sx = P.K + 15; P.slot_sy = P.K + 16;
    P.slot_light = stage_lights(s, p) ? P.K + 17 : -1;
    g_nd = nd;
    P.focal = p->focal[0];
    P.v.assign(P.N, P3{0, 0, 0});
    P.vn.assign(P.N, P3{0, 0, 0});
    if (nd) { P.dv.assign((size_t)P.N * 3 * nd, 0.0); P.dn.assign((size_t)P.N * 3 * nd, 0.0); }
    D R[9];
    rotation(P, R);
    V3 T = v3(seed_slot(p->trans[0], P.slot_trans + 0),
              seed_slot(p->trans[1], P.slot_trans + 1),
              seed_slot(p->trans[2], P.slot_trans + 2));
    int nt = threads_of(s);
    parallel_for(nt, P.N, [&](int i, int) { store(P.v, P.dv, nd, i, vertex_dual(P, i, R, T)); });
    // vertex normals: normalised sum of un-normalised face normals, faces in index order
    std::vector<P3> acc(P.N, P3{0, 0, 0});
    std::vector<double> dacc(nd ? (size_t)P.N * 3 * nd : 0, 0.0);
    for (int f = 0; f < P.T; ++f) {
        const int* t = s->faces + 3 * f;
        V3 a = load(P.v, P.dv, nd, t[0]), b = load(P.v, P.dv, nd, t[1]), c = load(P.v, P.dv, nd, t[2]);
        V3 nf = cross(b - a, c - a);
        for (int k = 0; k < 3; ++k) {
            V3 cur = load(acc, dacc, nd, t[k]);
            store(acc, dacc, nd, t[k], cur + nf);
        }
    }
    parallel_for(nt, P.N, [&](int i, int) { store(P.vn, P.dn, nd, i, normalize(load(acc, dacc, nd, i))); });
    // lights
    P.lights.resize(P.NL);
    if (stage_lights(s, p)) {
        for (int j = 0; j < P.NL; ++j) build_stage_light(P, j);
        return;
    }
    for (int j = 0; j < P.NL; ++j) {
        const float* r = s->lights + 11 * j;
        Light L;
        L.type = (int)r[0];
        if (L.type == ORA_LIGHT_ENV) {
            L.i0 = (int)r[1]; L.i1 = (int)r[2]; L.j0 = (int)r[3]; L.j1 = (int)r[4];
            L.area = 0.0;
            L.scale = 1.0;
            P.lights[j] = L;
            continue;
        }
        L.c = p3(r[1], r[2], r[3]);
        L.e1 = p3(r[4], r[5], r[6]);
        L.e2 = p3(r[7], r[8], r[9]);
        P3 cr = crossp(L.e1, L.e2);
        double cl = normp(cr);
        L.n = cr * (1.0 / cl);
        if (L.type == 0) L.area = cl;
        else if (L.type == 1) L.area = 0.5 * cl;
        else L.area = M_PI * dotp(L.e1, L.e1);
        L.scale = (double)s->light_d[j] * (double)s->light_d[j] / (double)s->light_a[j];
        P.lights[j] = L;
    }
}

// Undirected edges sorted by (min vertex, max vertex) with their faces.
std::vector<Edge> build_edges(const OraScene* s) {
    struct HalfEdge { int a, b, f; };
    std::vector<HalfEdge> h;
    h.reserve((size_t)s->n_triangles * 3);
    for (int f = 0; f < s->n_triangles; ++f)
        for (int k = 0; k < 3; ++k) {
            int u = s->faces[3 * f + k], w = s->faces[3 * f + (k + 1) % 3];
            h.push_back({std::min(u, w), std::max(u, w), f});
        }
    std::sort(h.begin(), h.end(), [](const HalfEdge& x, const HalfEdge& y) {
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        return x.f < y.f;
    });
    std::vector<Edge> e;
    for (size_t i = 0; i < h.size();) {
        size_t j = i;
        while (j < h.size() && h[j].a == h[i].a && h[j].b == h[i].b) ++j;
        Edge E{h[i].a, h[i].b, h[i].f, (j - i >= 2) ? h[i + 1].f : -1};
        e.push_back(E);
        i = j;
    }
    return e;
}

int sgn(double x) { return (x > 0.0) - (x < 0.0); }

P3 face_normal(const Prep& P, int f) {
    const int* t = P.s->faces + 3 * f;
    return crossp(P.v[t[1]] - P.v[t[0]], P.v[t[2]] - P.v[t[0]]);
}

// Silhouette classification (edge sampling, Sec. 4): primary silhouettes w.r.t.
// the camera centre, and per light the conservative candidate set of edges that
// are silhouettes w.r.t. some point of the emitter.
void classify(Prep& P) {
    P.edges = build_edges(P.s);
    P.prim_sil.clear();
    P.light_cand.assign(P.NL, {});
    for (int e = 0; e < (int)P.edges.size(); ++e) {
        const Edge& E = P.edges[e];
        P3 a = P.v[E.a];
        if (E.f2 < 0) {
            P.prim_sil.push_back(e);
            for (int j = 0; j < P.NL; ++j) P.light_cand[j].push_back(e);
            continue;
        }
        P3 n1 = face_normal(P, E.f1), n2 = face_normal(P, E.f2);
        if (sgn(-dotp(n1, a)) != sgn(-dotp(n2, a))) P.prim_sil.push_back(e);
        for (int j = 0; j < P.NL; ++j) {
            const Light& L = P.lights[j];
            double lo[2], hi[2];
            P3 nn[2] = {n1, n2};
            for (int q = 0; q < 2; ++q) {
                if (L.type == ORA_LIGHT_ENV) {
                    // a point at infinity in direction w is in front of the face iff n . w > 0
                    env_range(L, P.s->env_size, nn[q], lo[q], hi[q]);
                    continue;
                }
                double base = dotp(nn[q], L.c - a);
                if (L.type == 0) {
                    double h1 = 0.5 * std::fabs(dotp(nn[q], L.e1)), h2 = 0.5 * std::fabs(dotp(nn[q], L.e2));
                    lo[q] = base - h1 - h2; hi[q] = base + h1 + h2;
                } else if (L.type == 1) {
                    double g1 = dotp(nn[q], L.e1), g2 = dotp(nn[q], L.e2);
                    lo[q] = base + std::min({0.0, g1, g2}); hi[q] = base + std::max({0.0, g1, g2});
                } else {
                    double g1 = dotp(nn[q], L.e1), g2 = dotp(nn[q], L.e2);
                    double r = std::sqrt(g1 * g1 + g2 * g2);
                    lo[q] = base - r; hi[q] = base + r;
                }
            }
            bool pos = lo[0] > 0.0 && lo[1] > 0.0;
            bool neg = hi[0] < 0.0 && hi[1] < 0.0;
            if (!(pos || neg)) P.light_cand[j].push_back(e);
        }
    }
}

std::atomic<unsigned long long> g_rays{0};   // rays traced (for throughput reports)

// ---------------------------------------------------------------------------
// Ray/triangle intersection (Moller-Trumbore), FP64, two-sided.
// ---------------------------------------------------------------------------
bool intersect(P3 o, P3 d, P3 v0, P3 v1, P3 v2, double& t, double& b1, double& b2) {
    P3 e1 = v1 - v0, e2 = v2 - v0;
    P3 pv = crossp(d, e2);
    double det = dotp(e1, pv);
    if (det == 0.0) return false;
    double inv = 1.0 / det;
    P3 sv = o - v0;
    b1 = dotp(sv, pv) * inv;
    if (b1 < 0.0 || b1 > 1.0) return false;
    P3 qv = crossp(sv, e1);
    b2 = dotp(d, qv) * inv;
    if (b2 < 0.0 || b1 + b2 > 1.0) return false;
    t = dotp(e2, qv) * inv;
    return true;
}

// Closest hit over every triangle (brute force); ties -> lower triangle index.
int closest_hit(const Prep& P, P3 o, P3 d, double& t_hit) {
    g_rays.fetch_add(1, std::memory_order_relaxed);
    int best = -1;
    double bt = INFINITY;
    for (int f = 0; f < P.T; ++f) {
        const int* tr = P.s->faces + 3 * f;
        double t, b1, b2;
        if (intersect(o, d, P.v[tr[0]], P.v[tr[1]], P.v[tr[2]], t, b1, b2) && t > 0.0 && t < bt) {
            bt = t;
            best = f;
        }
    }
    t_hit = bt;
    return best;
}

// Shadow ray y -> z: occluded if any triangle other than `skip` crosses the
// segment at 1e-4 < t < 1 - 1e-4 (direction z - y, not normalised).
bool occluded(const Prep& P, P3 y, P3 z, int skip) {
    g_rays.fetch_add(1, std::memory_order_relaxed);
    P3 d = z - y;
    for (int f = 0; f < P.T; ++f) {
        if (f == skip) continue;
        const int* tr = P.s->faces + 3 * f;
        double t, b1, b2;
        if (intersect(y, d, P.v[tr[0]], P.v[tr[1]], P.v[tr[2]], t, b1, b2) && t > 1e-4 && t < 1.0 - 1e-4)
            return true;
    }
    return false;
}

// Shadow ray from y towards a light at infinity in unit direction w: occluded
// if any triangle other than `skip` crosses it at t > 1e-4.
bool occluded_dir(const Prep& P, P3 y, P3 w, int skip) {
    g_rays.fetch_add(1, std::memory_order_relaxed);
    for (int f = 0; f < P.T; ++f) {
        if (f == skip) continue;
        const int* tr = P.s->faces + 3 * f;
        double t, b1, b2;
        if (intersect(y, w, P.v[tr[0]], P.v[tr[1]], P.v[tr[2]], t, b1, b2) && t > 1e-4) return true;
    }
    return false;
}

// Emitter sample (Sec. 3.3): uniform over the emitter's area.
P3 light_point(const Light& L, double u, double v) {
    if (L.type == 0) return L.c + L.e1 * (u - 0.5) + L.e2 * (v - 0.5);
    if (L.type == 1) {
        double su = std::sqrt(u);
        return L.c + L.e1 * (su * (1.0 - v)) + L.e2 * (su * v);
    }
    double r = std::sqrt(u), phi = 2.0 * M_PI * v;
    return L.c + L.e1 * (r * std::cos(phi)) + L.e2 * (r * std::sin(phi));
}

// ---------------------------------------------------------------------------
// Reflectance (Sec. 3.2, App. A): f_r = f_d + f_s.
// ---------------------------------------------------------------------------
// Walter et al. rational approximation of the Smith masking term (Eq. brdf_g1).
D smith_g1_walter(const D& nv, const D& hv, const D& r) {
    if (!(hv.v / nv.v > 0.0)) return D(0.0);          // Delta(h.v / n.v), Eq. brdf_g1_chi
    double s2 = 1.0 - nv.v * nv.v;
    if (s2 <= 0.0) return D(1.0);                      // tan(acos(1)) = 0 -> a = infinity
    D a = nv / (r * dsqrt(1.0 - nv * nv));             // Eq. brdf_g1_a: 1/(r tan(acos(n.v)))
    if (a.v >= 1.6) return D(1.0);
    return (3.535 * a + 2.181 * a * a) / (1.0 + 2.276 * a + 2.577 * a * a);
}

D smith_g1_ggx(const D& nv, const D& hv, const D& r) {
    if (!(hv.v / nv.v > 0.0)) return D(0.0);
    D a2 = r * r;
    return 2.0 * nv / (nv + dsqrt(a2 + (1.0 - a2) * nv * nv));
}

// f_r for unit n, l, o; returns the RGB BRDF value.  Zero unless n.l > 0; the
// specular part only where n.o > 0.
void brdf(uint32_t flags, const V3& n, const V3& l, const V3& o, const D c[3], const D s[3],
          const D& r, D out[3]) {
    D nl = dot(n, l), no = dot(n, o);
    if (!(nl.v > 0.0)) { for (int k = 0; k < 3; ++k) out[k] = D(0.0); return; }
    // the specular lobe needs n.o > 0 (its denominator and the Delta of Eq. brdf_g1);
    // the Lambert term does not depend on the view
    if ((flags & ORA_DIFFUSE_ONLY) || !(no.v > 0.0)) { for (int k = 0; k < 3; ++k) out[k] = c[k] / M_PI; return; }
    V3 h = normalize(l + o);                           // Eq. halfVector (reading)
    D nh = dot(n, h), oh = dot(o, h), lh = dot(l, h);
    D Dterm, G;
    if (flags & ORA_GGX) {
        D a2 = r * r;
        D den = nh * nh * (a2 - 1.0) + 1.0;
        Dterm = a2 / (M_PI * den * den);
        G = smith_g1_ggx(no, oh, r) * smith_g1_ggx(nl, lh, r);
    } else {
        // Eq. brdf_d (reading): (alpha + 2)/(2 pi) (n.h)^alpha with alpha = 2/r - 2
        D alpha = 2.0 / r - 2.0;
        Dterm = (alpha + 2.0) / (2.0 * M_PI) * dpow(nh, alpha);
        G = smith_g1_walter(no, oh, r) * smith_g1_walter(nl, lh, r);   // Eq. brdf_g
    }
    D base = 1.0 - oh;                                 // Eq. brdf_f (Schlick)
    D fres_w = (flags & ORA_SCHLICK_LINEAR) ? base : dpowi(base, 5);
    D denom = 4.0 * no * nl;                           // Eq. brdf_spec
    for (int k = 0; k < 3; ++k) {
        D F = s[k] + (1.0 - s[k]) * fres_w;
        out[k] = c[k] / M_PI + Dterm * G * F / denom;  // Eq. brdf, brdf_diffuse
    }
}

// ---------------------------------------------------------------------------
// Texture lookup: bilinear, texel centres at u*M - 1/2, clamp-to-edge.
// ---------------------------------------------------------------------------
struct Tap { int idx[4]; double w[4]; };

D bilinear(const float* tex, int M, int channels, int ch, const D& u, const D& v, Tap* tap) {
    D x = u * (double)M - 0.5, y = v * (double)M - 0.5;
    double x0 = std::floor(x.v), y0 = std::floor(y.v);
    D fx = x - x0, fy = y - y0;
    int ix[2] = {std::min(std::max((int)x0, 0), M - 1), std::min(std::max((int)x0 + 1, 0), M - 1)};
    int iy[2] = {std::min(std::max((int)y0, 0), M - 1), std::min(std::max((int)y0 + 1, 0), M - 1)};
    D w00 = (1.0 - fx) * (1.0 - fy), w10 = fx * (1.0 - fy), w01 = (1.0 - fx) * fy, w11 = fx * fy;
    auto T = [&](int yy, int xx) { return (double)tex[((size_t)yy * M + xx) * channels + ch]; };
    if (tap) {
        tap->idx[0] = iy[0] * M + ix[0]; tap->w[0] = w00.v;
        tap->idx[1] = iy[0] * M + ix[1]; tap->w[1] = w10.v;
        tap->idx[2] = iy[1] * M + ix[0]; tap->w[2] = w01.v;
        tap->idx[3] = iy[1] * M + ix[1]; tap->w[3] = w11.v;
    }
    return w00 * T(iy[0], ix[0]) + w10 * T(iy[0], ix[1]) + w01 * T(iy[1], ix[0]) + w11 * T(iy[1], ix[1]);
}

// ---------------------------------------------------------------------------
// One camera sample: the Monte Carlo estimator F of Sec. 4 (Eq. energy) for
// direct lighting from every light-stage emitter with shadow rays (Sec. 3.3).
// ---------------------------------------------------------------------------
constexpr int ORA_MAX_LIGHTS = 128;  // lights with an intensity gradient

struct SampleOut {
    int tri = -1;
    uint64_t mask[2] = {0, 0};  // bit j of word j / 64: shadow ray to light j traced and unoccluded
    D L[3];                     // radiance (duals when gradients are requested)
    double dLdi[ORA_MAX_LIGHTS][3];  // d L / d i_j per channel (visible lights only); for an
                                     // environment block d L / d (radiance of its sampled texel)
    int env_tex[ORA_MAX_LIGHTS];     // environment block j: index row * M_e + col of its texel
    Tap tap;                    // bilinear taps at the hit (texture gradients)
    P3 y;                       // hit point
    V3 yd;                      // hit point as duals
    V3 ns;                      // shading normal
    V3 o;                       // view direction
    bool lit = false;           // the hit is shaded: its triangle faces the camera (and, with
                                // ORA_VIEW_CUTOFF, n_s . o > 0)
    D cc[3], ss[3], rr;         // albedos at the hit
};

// Screen position (sx, sy) in pixels -> camera ray direction (not normalised).
V3 camera_dir(const Prep& P, double sx, double sy) {
    D f = seed_slot(P.focal, P.slot_focal);
    return v3((sx - 0.5 * P.W) / f, -(sy - 0.5 * P.H) / f, D(-1.0));
}

// Hit point of ray o + t d with triangle `tri` as duals (Moller-Trumbore solved
// symbolically; the hit triangle is fixed).
void hit_duals(const Prep& P, int tri, const V3& d, D& b1, D& b2, V3& y) {
    const int* t = P.s->faces + 3 * tri;
    V3 v0 = load(P.v, P.dv, P.nd, t[0]), v1 = load(P.v, P.dv, P.nd, t[1]), v2 = load(P.v, P.dv, P.nd, t[2]);
    V3 e1 = v1 - v0, e2 = v2 - v0;
    V3 pv = cross(d, e2);
    D det = dot(e1, pv);
    V3 sv = v3c(0, 0, 0) - v0;    // ray origin is the camera centre
    b1 = dot(sv, pv) / det;
    V3 qv = cross(sv, e1);
    b2 = dot(d, qv) / det;
    D b0 = 1.0 - b1 - b2;
    y = v0 * b0 + v1 * b1 + v2 * b2;
}

// Radiance of the camera ray through screen point (sx, sy).  `st` supplies the
// light dimensions starting at `light_dim0`.  If `fixed_tri` >= 0 the hit
// triangle is imposed (the ray meets its plane), and the visibility mask
// `fixed_mask` too when given (gradient pass); without it the shadow rays are
// traced.  view_side = +-1 shades with the view direction tilted just to that
// side of the curve n_s . o = 0 (the two one-sided limits there).
void shade_sample(const Prep& P, double sx, double sy, Stream& st, int light_dim0, SampleOut& out,
                  int fixed_tri = -2, const uint64_t* fixed_mask = nullptr, int view_side = 0) {
    const OraScene* s = P.s;
    V3 dd = camera_dir(P, sx, sy);
    int tri;
    if (fixed_tri == -2) {
        double th;
        tri = closest_hit(P, p3(0, 0, 0), val(dd), th);
    } else {
        tri = fixed_tri;
    }
    out.tri = tri;
    out.mask[0] = out.mask[1] = 0;
    for (int k = 0; k < 3; ++k) out.L[k] = D(0.0);
    for (int j = 0; j < P.NL && j < ORA_MAX_LIGHTS; ++j) {
        out.dLdi[j][0] = out.dLdi[j][1] = out.dLdi[j][2] = 0.0;
        out.env_tex[j] = 0;
    }
    if (tri < 0) return;
    D b1, b2;
    V3 y;
    hit_duals(P, tri, dd, b1, b2, y);
    D b0 = 1.0 - b1 - b2;
    const int* t = s->faces + 3 * tri;
    V3 n0 = load(P.vn, P.dn, P.nd, t[0]), n1 = load(P.vn, P.dn, P.nd, t[1]), n2 = load(P.vn, P.dn, P.nd, t[2]);
    V3 ns = normalize(n0 * b0 + n1 * b1 + n2 * b2);
    V3 o = normalize(v3c(0, 0, 0) - dd);
    if (view_side) {        // one side of the curve n_s . o = 0: o tilted to n_s . o = +-1e-5
        const V3 om = o - ns * dot(ns, o);
        o = normalize(om + ns * (view_side > 0 ? 1e-5 : -1e-5));
    }
    D u = b0 * (double)s->uv[2 * t[0]] + b1 * (double)s->uv[2 * t[1]] + b2 * (double)s->uv[2 * t[2]];
    D v = b0 * (double)s->uv[2 * t[0] + 1] + b1 * (double)s->uv[2 * t[1] + 1] + b2 * (double)s->uv[2 * t[2] + 1];
    D c[3], sp[3], r;
    for (int k = 0; k < 3; ++k) {
        c[k] = bilinear(P.p->diffuse, P.M, 3, k, u, v, &out.tap);
        sp[k] = bilinear(P.p->specular, P.M, 3, k, u, v, nullptr);
        if (g_nd) { c[k].d[P.slot_c + k] += 1.0; sp[k].d[P.slot_s + k] += 1.0; }
    }
    r = bilinear(P.p->roughness, P.M, 1, 0, u, v, nullptr);
    if (g_nd) r.d[P.slot_r] += 1.0;
    out.y = val(y); out.yd = y; out.ns = ns; out.o = o;
    for (int k = 0; k < 3; ++k) { out.cc[k] = c[k]; out.ss[k] = sp[k]; }
    out.rr = r;
    if (s->flags & ORA_FLAT) {
        for (int k = 0; k < 3; ++k) out.L[k] = c[k];
        return;
    }
    {
        // one-sided surfaces: a triangle seen from behind reflects nothing (the change
        // happens at geometric silhouettes, which the primary-edge term samples)
        V3 v0 = load(P.v, P.dv, P.nd, t[0]), v1 = load(P.v, P.dv, P.nd, t[1]), v2 = load(P.v, P.dv, P.nd, t[2]);
        if (!(dot(cross(v1 - v0, v2 - v0), o).v > 0.0)) return;
    }
    if ((s->flags & ORA_VIEW_CUTOFF) && !(dot(ns, o).v > 0.0)) return;
    out.lit = true;
    for (int j = 0; j < P.NL; ++j) {
        const Light& Lj = P.lights[j];
        const double uu = st.u(light_dim0 + 2 * j), vv = st.u(light_dim0 + 2 * j + 1);
        if (Lj.type == ORA_LIGHT_ENV) {       // a light at infinity: l fixed, no distance term
            const EnvSample es = env_sample(Lj, s->env_size, uu, vv);
            const V3 l = v3c(es.w.x, es.w.y, es.w.z);
            const D cos_s = dot(ns, l);
            if (!(cos_s.v > 0.0)) continue;
            bool vis;
            if (fixed_tri == -2 || !fixed_mask) vis = !occluded_dir(P, val(y), es.w, tri);
            else vis = (fixed_mask[j >> 6] >> (j & 63)) & 1ull;
            if (!vis) continue;
            out.mask[j >> 6] |= (1ull << (j & 63));
            D f[3];
            brdf(s->flags, ns, l, o, c, sp, r, f);
            const D geo = cos_s * es.weight;
            if (j < ORA_MAX_LIGHTS) out.env_tex[j] = es.row * s->env_size + es.col;
            for (int k = 0; k < 3; ++k) {
                const D term = f[k] * geo;
                out.L[k] = out.L[k] + term * env_value(P, es.row, es.col, k);
                if (j < ORA_MAX_LIGHTS) out.dLdi[j][k] = term.v;
            }
            continue;
        }
        V3 zd;
        if (Lj.geo) {
            zd = light_point_d(Lj, uu, vv);
        } else {
            P3 zp = light_point(Lj, uu, vv);
            zd = v3c(zp.x, zp.y, zp.z);
        }
        P3 z = val(zd);
        V3 lv = zd - y;
        D dist2 = dot(lv, lv);
        V3 l = lv * (1.0 / dsqrt(dist2));
        D cos_s = dot(ns, l);
        D cos_l = -dot(v3c(Lj.n.x, Lj.n.y, Lj.n.z), l);
        if (!(cos_s.v > 0.0) || !(cos_l.v > 0.0)) continue;
        bool vis;
        if (fixed_tri == -2 || !fixed_mask) vis = !occluded(P, val(y), z, tri);
        else vis = (fixed_mask[j >> 6] >> (j & 63)) & 1ull;
        if (!vis) continue;
        out.mask[j >> 6] |= (1ull << (j & 63));
        D f[3];
        brdf(s->flags, ns, l, o, c, sp, r, f);
        D geo = Lj.geo ? cos_s * cos_l / dist2 * Lj.aread : cos_s * cos_l / dist2 * Lj.area;
        for (int k = 0; k < 3; ++k) {
            D term = f[k] * geo;
            if (Lj.geo) {
                out.L[k] = out.L[k] + term * Lj.scaled * (double)P.p->light_i[3 * j + k];   // Eq. lightIntensity
            } else {
                double I = Lj.scale * (double)P.p->light_i[3 * j + k];
                out.L[k] = out.L[k] + term * I;
            }
            if (j < ORA_MAX_LIGHTS) out.dLdi[j][k] = term.v * Lj.scale;
        }
    }
}

// Unoccluded-light integrand h = f_r * cos_s * cos_l / dist^2 (RGB) at point z of
// light j, from shading state already computed in `so`.
void light_integrand(const Prep& P, const SampleOut& so, int j, const V3& z, D h[3]) {
    const Light& Lj = P.lights[j];
    if (Lj.type == ORA_LIGHT_ENV) {           // z is the unit direction w: h = f_r cos_s
        const D cos_s = dot(so.ns, z);
        if (!(cos_s.v > 0.0) || !so.lit) {
            for (int k = 0; k < 3; ++k) h[k] = D(0.0);
            return;
        }
        D f[3];
        brdf(P.s->flags, so.ns, z, so.o, so.cc, so.ss, so.rr, f);
        for (int k = 0; k < 3; ++k) h[k] = f[k] * cos_s;
        return;
    }
    V3 lv = z - so.yd;
    D dist2 = dot(lv, lv);
    V3 l = lv * (1.0 / dsqrt(dist2));
    D cos_s = dot(so.ns, l);
    D cos_l = -dot(v3c(Lj.n.x, Lj.n.y, Lj.n.z), l);
    if (!(cos_s.v > 0.0) || !(cos_l.v > 0.0) || !so.lit) {
        for (int k = 0; k < 3; ++k) h[k] = D(0.0);
        return;
    }
    D f[3];
    brdf(P.s->flags, so.ns, l, so.o, so.cc, so.ss, so.rr, f);
    D geo = cos_s * cos_l / dist2;
    for (int k = 0; k < 3; ++k) h[k] = f[k] * geo;
}

// Is point z (on light j's plane) inside the emitter?
bool inside_emitter(const Light& L, P3 z) {
    P3 w = z - L.c;
    if (L.type == 2) return dotp(w, w) <= dotp(L.e1, L.e1);
    double g11 = dotp(L.e1, L.e1), g12 = dotp(L.e1, L.e2), g22 = dotp(L.e2, L.e2);
    double r1 = dotp(w, L.e1), r2 = dotp(w, L.e2);
    double det = g11 * g22 - g12 * g12;
    double a = (r1 * g22 - r2 * g12) / det, b = (r2 * g11 - r1 * g12) / det;
    if (L.type == 0) return std::fabs(a) <= 0.5 && std::fabs(b) <= 0.5;
    return a >= 0.0 && b >= 0.0 && a + b <= 1.0;
}

// Geometric slots of a dual folded with an adjoint weight into a gradient array.
void accumulate_geo(const Prep& P, const D& x, double w, double* g) {
    for (int q = 0; q < P.slot_c; ++q) g[q] += w * x.d[q];
}

// Shadow-boundary term of the light integral at shading state `so` (edge
// sampling, Sec. 4), one sample: returns sum over channels of adj_k * d/dtheta
// of sum_j int h_k V dA via geometric slots in g.  Boundary curve = projection
// from y of an occluder edge onto the emitter plane.
void shadow_edge_sample(const Prep& P, const SampleOut& so, int tri_self, double u_light,
                        double u_edge, double u_t, const double adj[3], double* g, bool* hit_out = nullptr,
                        double* g_light = nullptr) {
    if (hit_out) *hit_out = false;
    int j = std::min((int)(u_light * P.NL), P.NL - 1);
    const std::vector<int>& cand = P.light_cand[j];
    int S = (int)cand.size();
    if (S == 0) return;
    const Edge& E = P.edges[cand[std::min((int)(u_edge * S), S - 1)]];
    if (tri_self >= 0) {
        const int* t = P.s->faces + 3 * tri_self;
        bool ha = (E.a == t[0] || E.a == t[1] || E.a == t[2]);
        bool hb = (E.b == t[0] || E.b == t[1] || E.b == t[2]);
        if (ha && hb) return;           // an edge of the shading triangle itself
    }
    P3 y = so.y;
    if (E.f2 >= 0) {                    // silhouette w.r.t. y (FP64)
        P3 a = P.v[E.a];
        int s1 = sgn(dotp(face_normal(P, E.f1), y - a));
        int s2 = sgn(dotp(face_normal(P, E.f2), y - a));
        if (s1 == s2) return;
    }
    const Light& L = P.lights[j];
    // point on the edge as duals, with slot_t carrying d/dt
    V3 A = load(P.v, P.dv, P.nd, E.a), B = load(P.v, P.dv, P.nd, E.b);
    D tt = seed_slot(u_t, P.slot_t);
    V3 pe = A + (B - A) * tt;
    if (L.type == ORA_LIGHT_ENV) {
        // boundary on the sphere of directions: w(t) = (p(t) - y) / |p(t) - y|
        const int Me = P.s->env_size;
        const V3 wd = normalize(pe - so.yd);
        const P3 wv = val(wd);
        if (!inside_env_block(L, Me, wv)) return;
        D h[3];
        light_integrand(P, so, j, wd, h);
        if (h[0].v == 0.0 && h[1].v == 0.0 && h[2].v == 0.0) return;
        const P3 tan = p3(wd.x.d[P.slot_t], wd.y.d[P.slot_t], wd.z.d[P.slot_t]);
        const double tl = normp(tan);
        if (!(tl > 0.0)) return;
        const P3 m = crossp(wv, tan) * (1.0 / tl);   // unit normal of the curve, tangent to the sphere
        const double eps = 1e-4;
        const P3 wp = wv + m * eps, wm = wv - m * eps;
        const bool vp = !occluded_dir(P, y, wp * (1.0 / normp(wp)), tri_self);
        const bool vm = !occluded_dir(P, y, wm * (1.0 / normp(wm)), tri_self);
        const double dV = (double)vp - (double)vm;
        if (dV == 0.0) return;
        if (hit_out) *hit_out = true;
        const double scale = -dV * (double)P.NL * (double)S * tl;
        const D vn = wd.x * m.x + wd.y * m.y + wd.z * m.z;   // normal velocity of the boundary direction
        int row, col;
        env_texel_of(wv, Me, row, col);
        for (int k = 0; k < 3; ++k) {
            const double w = adj[k] * scale * h[k].v * env_value(P, row, col, k);
            if (w != 0.0) accumulate_geo(P, vn, w, g);
        }
        return;
    }
    V3 nL = v3c(L.n.x, L.n.y, L.n.z);
    V3 cL = L.geo ? L.cd : v3c(L.c.x, L.c.y, L.c.z);   // a moving plane moves the boundary point
    D den = dot(pe - so.yd, nL);
    D num = dot(cL - so.yd, nL);
    if (den.v == 0.0) return;
    D sc = num / den;
    if (!(sc.v > 1.0)) return;          // edge point must lie between y and the emitter plane
    V3 z = so.yd + (pe - so.yd) * sc;
    P3 zv = val(z);
    if (!inside_emitter(L, zv)) return;
    D h[3];
    light_integrand(P, so, j, z, h);
    if (h[0].v == 0.0 && h[1].v == 0.0 && h[2].v == 0.0) return;
    P3 tan = p3(z.x.d[P.slot_t], z.y.d[P.slot_t], z.z.d[P.slot_t]);
    double tl = normp(tan);
    if (!(tl > 0.0)) return;
    P3 m = crossp(L.n, tan) * (1.0 / tl);   // in-plane unit normal of the boundary curve
    double eps = 1e-4;
    bool vp = !occluded(P, y, zv + m * eps, tri_self);
    bool vm = !occluded(P, y, zv - m * eps, tri_self);
    double dV = (double)vp - (double)vm;
    if (dV == 0.0) return;
    if (hit_out) *hit_out = true;
    double scale = -dV * (double)P.NL * (double)S * tl;
    D vn = z.x * m.x + z.y * m.y + z.z * m.z;    // normal velocity of the boundary point
    if (L.geo && g_light) {
        // the emitter moves under the boundary: what counts is the boundary's
        // velocity relative to the emitter's own points, so subtract the
        // velocity of the emitter point at the boundary's emitter
        // coordinates (z - c = al e1 + be e2), held fixed
        P3 wv = zv - L.c;
        double g11 = dotp(L.e1, L.e1), g12 = dotp(L.e1, L.e2), g22 = dotp(L.e2, L.e2);
        double r1 = dotp(wv, L.e1), r2 = dotp(wv, L.e2), det = g11 * g22 - g12 * g12;
        double al = (r1 * g22 - r2 * g12) / det, be = (r2 * g11 - r1 * g12) / det;
        V3 zm = L.cd + L.e1d * al + L.e2d * be;
        D vm = zm.x * m.x + zm.y * m.y + zm.z * m.z;
        D rel = vn - vm;
        for (int k = 0; k < 3; ++k) {
            double I = L.scale * (double)P.p->light_i[3 * j + k];
            double w = adj[k] * scale * h[k].v * I;
            if (w == 0.0) continue;
            accumulate_geo(P, vn, w, g);
            for (int q = 0; q < 4 * P.NL; ++q) g_light[q] += w * rel.d[P.slot_light + q];
        }
        return;
    }
    for (int k = 0; k < 3; ++k) {
        double I = L.scale * (double)P.p->light_i[3 * j + k];
        double w = adj[k] * scale * h[k].v * I;
        if (w != 0.0) accumulate_geo(P, vn, w, g);
    }
}

// ---------------------------------------------------------------------------
// The curve n_s . o = 0 inside front-facing triangles, where the specular lobe
// (App. A, Eq. brdf_spec) switches on and off, met along image scanlines.
// ---------------------------------------------------------------------------
struct Crossing {
    int tri, root;      // triangle; 0 / 1 in order along the scanline
    double x, y;        // screen point (the scanline's own coordinate exact)
};

// Scanline `scan`: rows first (y = (i + u) / k for row line i), then columns
// (x = (i + u) / k), k = max(edge_spp, 1), u the line's uniform offset.
bool scanline(const Prep& P, int scan, uint32_t iteration, uint32_t face_id, double& c) {
    const int k = std::max(P.s->edge_spp, 1);
    const bool row = scan < P.H * k;
    const int idx = row ? scan : scan - P.H * k;
    Stream so{P.s->seed, STREAM_EDGE_SPECULAR, 0xFFFFFFFFu, (uint32_t)scan, iteration, face_id};
    c = (idx + so.u(0)) / k;
    return row;
}

// Every crossing of scanline `scan` with the curve q(b) = m(b) . (-p(b)) = 0
// (m = sum b_i n_i the unnormalised shading normal, p = sum b_i v_i the
// surface point: q has the sign of n_s . o) inside the front-facing triangles,
// in triangle order.  The rays of the scanline fill a plane through the camera
// centre; it cuts a triangle along a chord whose barycentrics are linear in the
// chord parameter s, so q is an exact quadratic in s.
void spec_crossings(const Prep& P, int scan, uint32_t iteration, uint32_t face_id, std::vector<Crossing>& out) {
    double c;
    const bool row = scanline(P, scan, iteration, face_id, c);
    const double f = P.focal;
    // plane normal: rows hold the directions (x, -(c - H/2)/f, -1), columns ((c - W/2)/f, y, -1)
    const P3 nrm = row ? p3(0.0, 1.0, -(c - 0.5 * P.H) / f) : p3(1.0, 0.0, (c - 0.5 * P.W) / f);
    for (int t = 0; t < P.T; ++t) {
        const int* fv = P.s->faces + 3 * t;
        const P3 v[3] = {P.v[fv[0]], P.v[fv[1]], P.v[fv[2]]};
        const P3 n[3] = {P.vn[fv[0]], P.vn[fv[1]], P.vn[fv[2]]};
        if (!(v[0].z < 0.0 && v[1].z < 0.0 && v[2].z < 0.0)) continue;        // in front of the camera
        if (!(dotp(crossp(v[1] - v[0], v[2] - v[0]), v[0]) < 0.0)) continue;  // faces the camera
        double ph[3];
        for (int i = 0; i < 3; ++i) ph[i] = dotp(nrm, v[i]);
        double bc[2][3];
        int ne = 0;
        for (int e = 0; e < 3 && ne < 2; ++e) {        // chord ends: edges whose ends straddle the plane
            const int i = e, j = (e + 1) % 3;
            if ((ph[i] > 0.0) == (ph[j] > 0.0)) continue;
            const double tt = ph[i] / (ph[i] - ph[j]);
            bc[ne][0] = bc[ne][1] = bc[ne][2] = 0.0;
            bc[ne][i] = 1.0 - tt;
            bc[ne][j] = tt;
            ++ne;
        }
        if (ne != 2) continue;
        double Q[3][3];                                // q(b) = sum_ij b_i b_j Q_ij
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Q[i][j] = -dotp(n[i], v[j]);
        auto form = [&](const double* a, const double* b) {
            double r = 0.0;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) r += a[i] * b[j] * Q[i][j];
            return r;
        };
        const double dl[3] = {bc[1][0] - bc[0][0], bc[1][1] - bc[0][1], bc[1][2] - bc[0][2]};
        const double a2 = form(dl, dl), a1 = form(bc[0], dl) + form(dl, bc[0]), a0 = form(bc[0], bc[0]);
        double sr[2];
        int nr = 0;
        if (a2 == 0.0) {
            if (a1 != 0.0) sr[nr++] = -a0 / a1;
        } else {
            const double disc = a1 * a1 - 4.0 * a2 * a0;
            if (disc > 0.0) {                          // a double root touches the curve without crossing it
                const double sq = std::sqrt(disc);
                const double qq = -0.5 * (a1 + (a1 >= 0.0 ? sq : -sq));
                sr[nr++] = qq / a2;
                sr[nr++] = a0 / qq;
            }
        }
        Crossing cr[2];
        int m = 0;
        for (int r = 0; r < nr; ++r) {
            if (!(sr[r] >= 0.0 && sr[r] <= 1.0)) continue;
            double b[3];
            for (int i = 0; i < 3; ++i) b[i] = bc[0][i] + sr[r] * dl[i];
            const P3 pt = v[0] * b[0] + v[1] * b[1] + v[2] * b[2];
            Crossing x;
            x.tri = t;
            x.x = row ? 0.5 * P.W + f * pt.x / -pt.z : c;
            x.y = row ? c : 0.5 * P.H - f * pt.y / -pt.z;
            cr[m++] = x;
        }
        if (m == 2 && (row ? cr[1].x < cr[0].x : cr[1].y < cr[0].y)) std::swap(cr[0], cr[1]);
        for (int r = 0; r < m; ++r) {
            cr[r].root = r;
            out.push_back(cr[r]);
        }
    }
}

// Camera ray direction through a screen point given as duals.
V3 camera_dir_d(const Prep& P, const D& sx, const D& sy) {
    D f = seed_slot(P.focal, P.slot_focal);
    return v3((sx - 0.5 * P.W) / f, -(sy - 0.5 * P.H) / f, D(-1.0));
}

// Boundary term of the curve n_s . o = 0 at one crossing (edge sampling,
// Sec. 4): with G = n_s . o at the fixed screen point x (duals on the
// parameters and on x), the curve moves along its unit normal n = grad G /
// |grad G| (towards G > 0, where the lobe is on) at speed -G_theta / |grad G|,
// and the image changes by -(L+ - L-) per unit of that motion, L+- the two
// one-sided limits of the radiance of the crossing's own triangle at x (the
// same hit, shadow rays and light samples; the view direction tilted to
// n_s . o = +-1e-5): the jump of the cutoff alone, with no part of the
// continuous change across the curve and nothing of a silhouette that the
// curve may run next to.  The curve is seen only where that triangle is the
// visible surface: nothing along the camera ray is nearer.  The scanline
// family's share n_x^2 (rows) or n_y^2 (columns) and its line density k turn
// the line integral into a sum over crossings:
// d/dtheta += sum_k adj_k (L+ - L-)_k G_theta |n_x| / (|grad G|^2 k) on rows.
void spec_boundary_sample(const Prep& P, const Crossing& c, int scan, bool row, uint32_t iteration,
                          uint32_t face_id, const double adj[3], double* g) {
    const int* t = P.s->faces + 3 * c.tri;
    D sx = seed_slot(c.x, P.slot_sx), sy = seed_slot(c.y, P.slot_sy);
    V3 d = camera_dir_d(P, sx, sy);
    D b1, b2;
    V3 y;
    hit_duals(P, c.tri, d, b1, b2, y);
    D b0 = 1.0 - b1 - b2;
    V3 n0 = load(P.vn, P.dn, P.nd, t[0]), n1 = load(P.vn, P.dn, P.nd, t[1]), n2 = load(P.vn, P.dn, P.nd, t[2]);
    V3 ns = normalize(n0 * b0 + n1 * b1 + n2 * b2);
    V3 o = normalize(v3c(0, 0, 0) - d);
    D G = dot(ns, o);
    const double gx = G.d[P.slot_sx], gy = G.d[P.slot_sy], g2 = gx * gx + gy * gy;
    if (!(g2 > 0.0)) return;
    double t_near;
    if (closest_hit(P, p3(0, 0, 0), val(d), t_near) >= 0 && t_near < -y.z.v * (1.0 - 1e-9)) return;
    Stream st{P.s->seed, STREAM_EDGE_SPECULAR, (uint32_t)(2 * c.tri + c.root), (uint32_t)scan, iteration, face_id};
    SampleOut sp, sm;
    {
        int keep = g_nd;
        g_nd = 0;
        shade_sample(P, c.x, c.y, st, 4, sp, c.tri, nullptr, +1);
        shade_sample(P, c.x, c.y, st, 4, sm, c.tri, nullptr, -1);
        g_nd = keep;
    }
    double jump = 0.0;
    for (int k = 0; k < 3; ++k) jump += adj[k] * (sp.L[k].v - sm.L[k].v);
    const int k = std::max(P.s->edge_spp, 1);
    const double w = jump * (row ? std::fabs(gx) : std::fabs(gy)) / (g2 * k);
    if (w != 0.0) accumulate_geo(P, G, w, g);
}

// ---------------------------------------------------------------------------
// Blur + L1 loss (Sec. 4 Eq. energy and "Variance Reduction").
// ---------------------------------------------------------------------------
void gauss3(double w[3][3]) {
    double s = 0.0;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            w[dy + 1][dx + 1] = std::exp(-0.5 * (dx * dx + dy * dy));
            s += w[dy + 1][dx + 1];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) w[i][j] /= s;
}

}  // namespace

// ===========================================================================
// C API
// ===========================================================================
extern "C" {

unsigned long long ora_ray_count(int reset) {
    unsigned long long v = g_rays.load();
    if (reset) g_rays.store(0);
    return v;
}

void ora_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                uint32_t out[4]) {
    uint32_t c[4] = {c0, c1, c2, c3};
    philox4x32_10(k0, k1, c);
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

int ora_geometry(const OraScene* s, const OraParams* p, double* v_cam, double* n_vert) {
    Prep P;
    prepare(P, s, p, 0);
    for (int i = 0; i < P.N; ++i) {
        if (v_cam) { v_cam[3 * i] = P.v[i].x; v_cam[3 * i + 1] = P.v[i].y; v_cam[3 * i + 2] = P.v[i].z; }
        if (n_vert) { n_vert[3 * i] = P.vn[i].x; n_vert[3 * i + 1] = P.vn[i].y; n_vert[3 * i + 2] = P.vn[i].z; }
    }
    return 0;
}

int ora_edges(const OraScene* s, int32_t* edge_v, int32_t* edge_f) {
    std::vector<Edge> e = build_edges(s);
    for (size_t i = 0; i < e.size(); ++i) {
        if (edge_v) { edge_v[2 * i] = e[i].a; edge_v[2 * i + 1] = e[i].b; }
        if (edge_f) { edge_f[2 * i] = e[i].f1; edge_f[2 * i + 1] = e[i].f2; }
    }
    return (int)e.size();
}

int ora_silhouettes(const OraScene* s, const OraParams* p, int32_t* prim, int32_t* n_prim,
                    int32_t* per_light, int32_t* light_counts) {
    Prep P;
    prepare(P, s, p, 0);
    classify(P);
    *n_prim = (int)P.prim_sil.size();
    if (prim) for (size_t i = 0; i < P.prim_sil.size(); ++i) prim[i] = P.prim_sil[i];
    size_t E = P.edges.size();
    for (int j = 0; j < P.NL; ++j) {
        light_counts[j] = (int)P.light_cand[j].size();
        if (per_light)
            for (size_t i = 0; i < P.light_cand[j].size(); ++i) per_light[j * E + i] = P.light_cand[j][i];
    }
    return (int)E;
}

int ora_closest_hit(const OraScene* s, const OraParams* p, const double* org, const double* dir,
                    int32_t n, int32_t* tri, double* t) {
    Prep P;
    prepare(P, s, p, 0);
    parallel_for(threads_of(s), n, [&](int i, int) {
        double th;
        P3 o = p3(org[3 * i], org[3 * i + 1], org[3 * i + 2]);
        P3 d = p3(dir[3 * i], dir[3 * i + 1], dir[3 * i + 2]);
        int best = -1;
        double bt = INFINITY;
        for (int f = 0; f < P.T; ++f) {
            const int* tr = s->faces + 3 * f;
            double tt, b1, b2;
            if (intersect(o, d, P.v[tr[0]], P.v[tr[1]], P.v[tr[2]], tt, b1, b2) && tt > 0.0 && tt < bt) {
                bt = tt;
                best = f;
            }
        }
        (void)th;
        tri[i] = best;
        t[i] = best >= 0 ? bt : -1.0;
    });
    return 0;
}

// Forward render: image[H][W][3] = mean over spp of the per-sample estimator.
int ora_render(const OraScene* s, const OraParams* p, uint32_t iteration, uint32_t face_id,
               const int32_t* pixels, int32_t n_pixels, double* image, int32_t* tri_rec,
               uint64_t* mask_rec) {
    Prep P;
    prepare(P, s, p, 0);
    int npx = (pixels && n_pixels > 0) ? n_pixels : P.W * P.H;
    parallel_for(threads_of(s), npx, [&](int i, int) {
        int pix = (pixels && n_pixels > 0) ? pixels[i] : i;
        int px = pix % P.W, py = pix / P.W;
        double acc[3] = {0, 0, 0};
        for (int smp = 0; smp < P.spp; ++smp) {
            Stream st{s->seed, STREAM_PRIMARY, (uint32_t)pix, (uint32_t)smp, iteration, face_id};
            SampleOut so;
            shade_sample(P, px + st.u(0), py + st.u(1), st, 2, so);
            for (int k = 0; k < 3; ++k) acc[k] += so.L[k].v;
            size_t rec = (size_t)pix * P.spp + smp;
            if (tri_rec) tri_rec[rec] = so.tri;
            if (mask_rec) {                             // lights 0..63, 64..127
                mask_rec[2 * (size_t)rec] = so.mask[0];
                mask_rec[2 * (size_t)rec + 1] = so.mask[1];
            }
        }
        for (int k = 0; k < 3; ++k) image[(size_t)pix * 3 + k] = acc[k] / P.spp;
    });
    return 0;
}

double ora_loss(int32_t H, int32_t W, const double* image, const float* target, double* blurred,
                double* adjoint) {
    double w[3][3];
    gauss3(w);
    std::vector<double> bl((size_t)H * W * 3, 0.0), sg((size_t)H * W * 3, 0.0);
    double loss = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int k = 0; k < 3; ++k) {
                double acc = 0.0;
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        int yy = std::min(std::max(y + dy, 0), H - 1), xx = std::min(std::max(x + dx, 0), W - 1);
                        acc += w[dy + 1][dx + 1] * image[((size_t)yy * W + xx) * 3 + k];
                    }
                size_t i = ((size_t)y * W + x) * 3 + k;
                bl[i] = acc;
                double r = acc - (double)target[i];
                loss += std::fabs(r);
                sg[i] = (r > 0.0) - (r < 0.0);
            }
    if (blurred) std::copy(bl.begin(), bl.end(), blurred);
    if (adjoint) {
        std::fill(adjoint, adjoint + (size_t)H * W * 3, 0.0);
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x)
                for (int k = 0; k < 3; ++k)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dx = -1; dx <= 1; ++dx) {
                            int yy = std::min(std::max(y + dy, 0), H - 1), xx = std::min(std::max(x + dx, 0), W - 1);
                            adjoint[((size_t)yy * W + xx) * 3 + k] += w[dy + 1][dx + 1] * sg[((size_t)y * W + x) * 3 + k];
                        }
    }
    return loss;
}

// Gradient of sum_p adjoint_p . image_p w.r.t. every parameter group.
int ora_grad(const OraScene* s, const OraParams* p, uint32_t iteration, uint32_t face_id,
             const double* adjoint, uint32_t terms, double* g_coef, double* g_rot, double* g_trans,
             double* g_focal, double* g_light, double* g_diffuse, double* g_specular,
             double* g_roughness, double* g_light_geom, double* g_env) {
    const int n_lg = stage_lights(s, p) ? 4 * s->n_lights : 0;
    if (s->n_basis + 17 + n_lg > DMAX || s->n_lights > ORA_MAX_LIGHTS) return -1;
    Prep P;
    prepare(P, s, p, s->n_basis + 17 + n_lg);
    classify(P);
    int nt = threads_of(s);
    int ngeo = P.slot_c;
    size_t MM = (size_t)P.M * P.M;
    const size_t n_env = (size_t)s->env_size * s->env_size * 3;
    struct Acc {
        std::vector<double> geo, light, dif, spec, rough, lg, env;
    };
    std::vector<Acc> acc(nt);
    for (auto& a : acc) {
        a.env.assign(std::max<size_t>(n_env, 1), 0.0);
        a.geo.assign(ngeo, 0.0);
        a.lg.assign((size_t)std::max(n_lg, 1), 0.0);
        a.light.assign((size_t)P.NL * 3, 0.0);
        a.dif.assign(MM * 3, 0.0);
        a.spec.assign(MM * 3, 0.0);
        a.rough.assign(MM, 0.0);
    }
    const int npx = P.W * P.H;
    auto adj_of = [&](int pix, double out[3]) {
        for (int k = 0; k < 3; ++k) out[k] = adjoint[(size_t)pix * 3 + k];
        return out[0] != 0.0 || out[1] != 0.0 || out[2] != 0.0;
    };
    // interior term and shadow-boundary term, per camera sample
    if (terms & (ORA_TERM_INTERIOR | ORA_TERM_SHADOW)) {
        parallel_for(nt, npx, [&](int pix, int th) {
            double adj[3];
            if (!adj_of(pix, adj)) return;
            Acc& A = acc[th];
            int px = pix % P.W, py = pix / P.W;
            for (int smp = 0; smp < P.spp; ++smp) {
                Stream st{s->seed, STREAM_PRIMARY, (uint32_t)pix, (uint32_t)smp, iteration, face_id};
                double sx = px + st.u(0), sy = py + st.u(1);
                SampleOut fw;
                {   // values-only pass for the hit and visibility
                    int keep = g_nd;
                    g_nd = 0;
                    shade_sample(P, sx, sy, st, 2, fw);
                    g_nd = keep;
                }
                SampleOut so;
                shade_sample(P, sx, sy, st, 2, so, fw.tri, fw.mask);
                if (so.tri < 0) continue;
                double w[3] = {adj[0] / P.spp, adj[1] / P.spp, adj[2] / P.spp};
                if (terms & ORA_TERM_INTERIOR) {
                    for (int k = 0; k < 3; ++k) accumulate_geo(P, so.L[k], w[k], A.geo.data());
                    for (int q = 0; q < n_lg; ++q)
                        for (int k = 0; k < 3; ++k) A.lg[q] += w[k] * so.L[k].d[P.slot_light + q];
                    double dr = 0.0;
                    for (int k = 0; k < 3; ++k) dr += w[k] * so.L[k].d[P.slot_r];
                    for (int q = 0; q < 4; ++q) {
                        int ti = so.tap.idx[q];
                        double tw = so.tap.w[q];
                        for (int k = 0; k < 3; ++k) {
                            A.dif[(size_t)ti * 3 + k] += tw * w[k] * so.L[k].d[P.slot_c + k];
                            A.spec[(size_t)ti * 3 + k] += tw * w[k] * so.L[k].d[P.slot_s + k];
                        }
                        A.rough[ti] += tw * dr;
                    }
                    for (int j = 0; j < P.NL; ++j) {
                        if (P.lights[j].type == ORA_LIGHT_ENV) {     // the sampled texel's radiance
                            for (int k = 0; k < 3; ++k) A.env[3 * (size_t)so.env_tex[j] + k] += w[k] * so.dLdi[j][k];
                            continue;
                        }
                        for (int k = 0; k < 3; ++k) A.light[3 * j + k] += w[k] * so.dLdi[j][k];
                    }
                }
                if ((terms & ORA_TERM_SHADOW) && !(s->flags & ORA_FLAT) && so.lit) {
                    Stream se{s->seed, STREAM_EDGE_SHADOW, (uint32_t)pix, (uint32_t)smp, iteration, face_id};
                    shadow_edge_sample(P, so, so.tri, se.u(0), se.u(1), se.u(2), w, A.geo.data(), nullptr,
                                       n_lg ? A.lg.data() : nullptr);
                }
            }
        });
    }
    // primary boundary term: edge samples in screen space
    if ((terms & ORA_TERM_PRIMARY) && !P.prim_sil.empty()) {
        const int S = (int)P.prim_sil.size();
        const long n_edge = (long)npx * s->edge_spp;
        const int chunks = 4096;
        parallel_for(nt, chunks, [&](int ch, int th) {
            Acc& A = acc[th];
            long lo = n_edge * ch / chunks, hi = n_edge * (ch + 1) / chunks;
            for (long e = lo; e < hi; ++e) {
                Stream st{s->seed, STREAM_EDGE_PRIMARY, (uint32_t)e, 0u, iteration, face_id};
                const Edge& E = P.edges[P.prim_sil[std::min((int)(st.u(0) * S), S - 1)]];
                V3 a = load(P.v, P.dv, P.nd, E.a), b = load(P.v, P.dv, P.nd, E.b);
                D tt = seed_slot(st.u(1), P.slot_t);
                V3 pe = a + (b - a) * tt;
                if (!(pe.z.v < 0.0)) continue;
                D f = seed_slot(P.focal, P.slot_focal);
                D X = 0.5 * P.W + f * pe.x / (-pe.z);
                D Y = 0.5 * P.H - f * pe.y / (-pe.z);
                if (!(X.v >= 0.0 && X.v < P.W && Y.v >= 0.0 && Y.v < P.H)) continue;
                int pix = (int)std::floor(Y.v) * P.W + (int)std::floor(X.v);
                double adj[3];
                if (!adj_of(pix, adj)) continue;
                double tx = X.d[P.slot_t], ty = Y.d[P.slot_t];
                double tl = std::sqrt(tx * tx + ty * ty);
                if (!(tl > 0.0)) continue;
                double mx = -ty / tl, my = tx / tl;
                const double eps = 1e-3;
                SampleOut sp, sm;
                {
                    int keep = g_nd;
                    g_nd = 0;
                    shade_sample(P, X.v + eps * mx, Y.v + eps * my, st, 4, sp);
                    shade_sample(P, X.v - eps * mx, Y.v - eps * my, st, 4, sm);
                    g_nd = keep;
                }
                double scale = (double)S * tl / (double)n_edge;
                D vn = X * mx + Y * my;
                for (int k = 0; k < 3; ++k) {
                    double dL = sp.L[k].v - sm.L[k].v;
                    double w = -adj[k] * dL * scale;
                    if (w != 0.0) accumulate_geo(P, vn, w, A.geo.data());
                }
            }
        });
    }
    // boundary term of the specular lobe: crossings of image scanlines with the
    // curve n_s . o = 0
    if ((terms & ORA_TERM_SPECULAR) && !(s->flags & ORA_FLAT)) {
        const int n_scan = (P.H + P.W) * std::max(s->edge_spp, 1);
        parallel_for(nt, n_scan, [&](int scan, int th) {
            std::vector<Crossing> cr;
            spec_crossings(P, scan, iteration, face_id, cr);
            double c;
            const bool row = scanline(P, scan, iteration, face_id, c);
            for (const Crossing& x : cr) {
                if (!(x.x >= 0.0 && x.x < P.W && x.y >= 0.0 && x.y < P.H)) continue;
                double adj[3];
                if (!adj_of((int)std::floor(x.y) * P.W + (int)std::floor(x.x), adj)) continue;
                spec_boundary_sample(P, x, scan, row, iteration, face_id, adj, acc[th].geo.data());
            }
        });
    }
    // reduce
    std::vector<double> geo(ngeo, 0.0), light((size_t)P.NL * 3, 0.0);
    for (auto& a : acc) {
        for (int q = 0; q < ngeo; ++q) geo[q] += a.geo[q];
        for (size_t q = 0; q < light.size(); ++q) light[q] += a.light[q];
    }
    for (int k = 0; k < P.K; ++k) if (g_coef) g_coef[k] = geo[k];
    for (int k = 0; k < 3; ++k) {
        if (g_rot) g_rot[k] = geo[P.slot_rot + k];
        if (g_trans) g_trans[k] = geo[P.slot_trans + k];
    }
    if (g_focal) g_focal[0] = geo[P.slot_focal];
    if (g_light) std::copy(light.begin(), light.end(), g_light);
    if (g_light_geom && n_lg) {
        std::fill(g_light_geom, g_light_geom + n_lg, 0.0);
        for (auto& a : acc)
            for (int q = 0; q < n_lg; ++q) g_light_geom[q] += a.lg[q];
    }
    if (g_diffuse) { std::fill(g_diffuse, g_diffuse + MM * 3, 0.0); for (auto& a : acc) for (size_t q = 0; q < MM * 3; ++q) g_diffuse[q] += a.dif[q]; }
    if (g_specular) { std::fill(g_specular, g_specular + MM * 3, 0.0); for (auto& a : acc) for (size_t q = 0; q < MM * 3; ++q) g_specular[q] += a.spec[q]; }
    if (g_roughness) { std::fill(g_roughness, g_roughness + MM, 0.0); for (auto& a : acc) for (size_t q = 0; q < MM; ++q) g_roughness[q] += a.rough[q]; }
    if (g_env && n_env) { std::fill(g_env, g_env + n_env, 0.0); for (auto& a : acc) for (size_t q = 0; q < n_env; ++q) g_env[q] += a.env[q]; }
    g_nd = 0;
    return 0;
}

// Crossings of scanline `scan` with the curve n_s . o = 0 (values only): up to
// `max` of them as (triangle, root) and screen (x, y); returns their count.
int ora_spec_crossings(const OraScene* s, const OraParams* p, uint32_t iteration, uint32_t face_id, int32_t scan,
                       int32_t max, int32_t* tri_root, double* xy) {
    Prep P;
    prepare(P, s, p, 0);
    const int n_scan = (P.H + P.W) * std::max(s->edge_spp, 1);
    if (scan < 0 || scan >= n_scan) return -1;
    std::vector<Crossing> cr;
    spec_crossings(P, scan, iteration, face_id, cr);
    for (int i = 0; i < (int)cr.size() && i < max; ++i) {
        tri_root[2 * i] = cr[i].tri;
        tri_root[2 * i + 1] = cr[i].root;
        xy[2 * i] = cr[i].x;
        xy[2 * i + 1] = cr[i].y;
    }
    return (int)cr.size();
}

double ora_brdf(uint32_t flags, const double* n, const double* l, const double* o, const double* c,
                const double* s, double r, double* out_rgb) {
    g_nd = 0;
    V3 N = v3c(n[0], n[1], n[2]), Lv = v3c(l[0], l[1], l[2]), O = v3c(o[0], o[1], o[2]);
    D cc[3] = {D(c[0]), D(c[1]), D(c[2])}, ss[3] = {D(s[0]), D(s[1]), D(s[2])};
    D out[3];
    brdf(flags, N, Lv, O, cc, ss, D(r), out);
    for (int k = 0; k < 3; ++k) out_rgb[k] = out[k].v;
    return out[0].v;
}

// Factors of the specular lobe for unit n, l, o (App. A): D, G1(o), G1(l), and
// the Schlick weight w so that F = s + (1 - s) w.
void ora_brdf_terms(uint32_t flags, const double* n, const double* l, const double* o, double r,
                    double* out) {
    g_nd = 0;
    V3 N = v3c(n[0], n[1], n[2]), Lv = v3c(l[0], l[1], l[2]), O = v3c(o[0], o[1], o[2]);
    V3 h = normalize(Lv + O);
    D nh = dot(N, h), no = dot(N, O), nl = dot(N, Lv), oh = dot(O, h), lh = dot(Lv, h);
    D rr(r);
    if (flags & ORA_GGX) {
        D a2 = rr * rr;
        D den = nh * nh * (a2 - 1.0) + 1.0;
        out[0] = (a2 / (M_PI * den * den)).v;
        out[1] = smith_g1_ggx(no, oh, rr).v;
        out[2] = smith_g1_ggx(nl, lh, rr).v;
    } else {
        D alpha = 2.0 / rr - 2.0;
        out[0] = nh.v > 0.0 ? ((alpha + 2.0) / (2.0 * M_PI) * dpow(nh, alpha)).v : 0.0;
        out[1] = smith_g1_walter(no, oh, rr).v;
        out[2] = smith_g1_walter(nl, lh, rr).v;
    }
    D base = 1.0 - oh;
    out[3] = ((flags & ORA_SCHLICK_LINEAR) ? base : dpowi(base, 5)).v;
}

// Light integral at a fixed point y with normal n for a white Lambertian
// surface (f_r = 1/pi): value = sum_j L_j int V cos cos / d^2 dA / pi estimated
// with n_samples area samples per light, and the shadow-boundary derivative of
// that value w.r.t. the shape coefficients (occluder motion), n_samples edge
// samples.  Used to pin the shadow-edge estimator against closed forms.
int ora_point_light_grad(const OraScene* s, const OraParams* p, const double* y, const double* n,
                         int32_t tri_self, int32_t n_samples, uint32_t seed_stream, double* value_rgb,
                         double* g_coef, double* g_light_geom) {
    OraScene sc = *s;
    sc.flags = ORA_DIFFUSE_ONLY;
    const int n_lg = stage_lights(s, p) ? 4 * s->n_lights : 0;
    if (s->n_basis + 17 + n_lg > DMAX) return -1;
    Prep P;
    prepare(P, &sc, p, s->n_basis + 17 + n_lg);
    classify(P);
    int nt = threads_of(s);
    std::vector<std::vector<double>> gs(nt, std::vector<double>(P.slot_c, 0.0));
    std::vector<std::vector<double>> vs(nt, std::vector<double>(3, 0.0));
    std::vector<std::vector<double>> gl(nt, std::vector<double>((size_t)std::max(n_lg, 1), 0.0));
    const D zero3[3] = {D(0.0), D(0.0), D(0.0)};
    parallel_for(nt, n_samples, [&](int i, int th) {
        SampleOut so;
        so.tri = tri_self;
        so.y = p3(y[0], y[1], y[2]);
        so.yd = v3c(y[0], y[1], y[2]);
        so.ns = v3c(n[0], n[1], n[2]);
        so.o = v3c(n[0], n[1], n[2]);
        so.lit = true;
        for (int k = 0; k < 3; ++k) { so.cc[k] = D(1.0); so.ss[k] = zero3[k]; }
        so.rr = D(0.5);
        Stream st{s->seed, seed_stream, (uint32_t)i, 0u, 0u, 0u};
        // interior estimate: one area sample per light
        for (int j = 0; j < P.NL; ++j) {
            const Light& L = P.lights[j];
            if (L.geo) {            // with derivatives on the light's (d, a, p), channel 0
                V3 zd = light_point_d(L, st.u(4 + 2 * j), st.u(5 + 2 * j));
                V3 lvd = zd - so.yd;
                D d2 = dot(lvd, lvd);
                V3 l = lvd * (1.0 / dsqrt(d2));
                D cs = dot(so.ns, l), cl = -dot(v3c(L.n.x, L.n.y, L.n.z), l);
                if (cs.v <= 0.0 || cl.v <= 0.0) continue;
                if (occluded(P, so.y, val(zd), tri_self)) continue;
                D g = L.scaled * cs * cl / d2 * L.aread * (1.0 / M_PI);
                for (int k = 0; k < 3; ++k) vs[th][k] += g.v * p->light_i[3 * j + k];
                for (int q = 0; q < n_lg; ++q) gl[th][q] += g.d[P.slot_light + q] * p->light_i[3 * j];
                continue;
            }
            if (L.type == ORA_LIGHT_ENV) {
                const EnvSample es = env_sample(L, s->env_size, st.u(4 + 2 * j), st.u(5 + 2 * j));
                const double cs = dotp(p3(n[0], n[1], n[2]), es.w);
                if (cs <= 0.0) continue;
                if (occluded_dir(P, so.y, es.w, tri_self)) continue;
                for (int k = 0; k < 3; ++k) vs[th][k] += env_value(P, es.row, es.col, k) * cs * es.weight / M_PI;
                continue;
            }
            P3 z = light_point(L, st.u(4 + 2 * j), st.u(5 + 2 * j));
            P3 lv = z - so.y;
            double d2 = dotp(lv, lv);
            P3 l = lv * (1.0 / std::sqrt(d2));
            double cs = dotp(p3(n[0], n[1], n[2]), l), cl = -dotp(L.n, l);
            if (cs <= 0.0 || cl <= 0.0) continue;
            if (occluded(P, so.y, z, tri_self)) continue;
            for (int k = 0; k < 3; ++k)
                vs[th][k] += L.scale * p->light_i[3 * j + k] * cs * cl / d2 * L.area / M_PI;
        }
        double w[3] = {1.0, 0.0, 0.0};
        // light_integrand uses brdf() in diffuse-only mode: white Lambertian
        shadow_edge_sample(P, so, tri_self, st.u(0), st.u(1), st.u(2), w, gs[th].data(), nullptr,
                           n_lg ? gl[th].data() : nullptr);
    });
    for (int k = 0; k < 3; ++k) {
        double a = 0.0;
        for (int t = 0; t < nt; ++t) a += vs[t][k];
        value_rgb[k] = a / n_samples;
    }
    for (int k = 0; k < P.K; ++k) {
        double a = 0.0;
        for (int t = 0; t < nt; ++t) a += gs[t][k];
        g_coef[k] = a / n_samples;
    }
    if (g_light_geom)
        for (int q = 0; q < n_lg; ++q) {
            double a = 0.0;
            for (int t = 0; t < nt; ++t) a += gl[t][q];
            g_light_geom[q] = a / n_samples;
        }
    g_nd = 0;
    return 0;
}

}  // extern "C"
