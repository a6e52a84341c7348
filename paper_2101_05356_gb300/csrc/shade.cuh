// Emitters (Sec. 3.3), texture lookup (Sec. 3.2) and the Cook-Torrance BRDF of
// App. A with its hand-written reverse mode.
#pragma once
#include "common.cuh"

#define FR_FLAG_GGX_D 1u
#define FR_FLAG_SCHLICK_LINEAR_D 2u
#define FR_FLAG_FLAT_D 4u
#define FR_FLAG_NO_INTERIOR_D 16u
#define FR_FLAG_NO_PRIMARY_EDGE_D 32u
#define FR_FLAG_NO_SHADOW_EDGE_D 64u
#define FR_FLAG_NO_SPECULAR_EDGE_D 2048u
#define FR_FLAG_VIEW_CUTOFF_D 1024u
#define FR_LIGHT_ENV_D 3

// Uniform area sample of an emitter.
FR_D float3 light_point(const LightDev& L, float u, float v) {
    if (L.type == 0) return L.c + L.e1 * (u - 0.5f) + L.e2 * (v - 0.5f);
    if (L.type == 1) {
        const float su = sqrtf(u);
        return L.c + L.e1 * (su * (1.0f - v)) + L.e2 * (su * v);
    }
    float sn, cs;
    sincospif(2.0f * v, &sn, &cs);
    const float r = sqrtf(u);
    return L.c + L.e1 * (r * cs) + L.e2 * (r * sn);
}

// Point z of the emitter plane inside the emitter?
FR_D bool inside_emitter(const LightDev& L, float3 z) {
    const float3 w = z - L.c;
    if (L.type == 2) return dot(w, w) <= dot(L.e1, L.e1);
    const float g11 = dot(L.e1, L.e1), g12 = dot(L.e1, L.e2), g22 = dot(L.e2, L.e2);
    const float r1 = dot(w, L.e1), r2 = dot(w, L.e2);
    const float det = g11 * g22 - g12 * g12;
    const float a = (r1 * g22 - r2 * g12) / det, b = (r2 * g11 - r1 * g12) / det;
    if (L.type == 0) return fabsf(a) <= 0.5f && fabsf(b) <= 0.5f;
    return a >= 0.0f && b >= 0.0f && a + b <= 1.0f;
}

// ---------------------------------------------------------------------------
// Environment blocks: lights at infinity (Sec. 7).  Row i of the M_e x M_e map
// spans polar angles [i, i + 1] pi / M_e from +y, column j azimuths
// [j, j + 1] 2 pi / M_e from +z towards +x, w = (sin t sin p, cos t, sin t cos p).
// ---------------------------------------------------------------------------
struct EnvDir {
    float3 w;       // unit direction towards the light
    float weight;   // 1 / pdf: texels in the block x the texel's solid angle
    int texel;      // row * M_e + column
};

// A texel uniformly among the block's R x C, from the 24-bit integers k behind
// the uniforms (row = i0 + floor(k_u R / 2^24); the remainder places the sample
// inside the row, columns likewise), then a direction uniform in solid angle
// inside the texel (cos t and p uniform).
FR_D EnvDir env_sample(const LightDev& L, float u, float v) {
    const int Me = L.env;
    const uint32_t i0 = (uint32_t)L.c.x, R = (uint32_t)L.c.y - i0;
    const uint32_t j0 = (uint32_t)L.c.z, C = (uint32_t)L.e1.x - j0;
    const uint64_t pu = (uint64_t)__float2uint_rz(u * 16777216.0f) * R;   // u = k_u 2^-24 exactly
    const uint64_t pv = (uint64_t)__float2uint_rz(v * 16777216.0f) * C;
    const int row = (int)i0 + (int)(pu >> 24), col = (int)j0 + (int)(pv >> 24);
    const float fu = (float)(uint32_t)(pu & 0xFFFFFFu) * (1.0f / 16777216.0f);
    const float fv = (float)(uint32_t)(pv & 0xFFFFFFu) * (1.0f / 16777216.0f);
    const float zt = cospif((float)row / (float)Me), zb = cospif((float)(row + 1) / (float)Me);
    const float y = zt + fu * (zb - zt);
    const float sn = sqrtf(fmaxf(0.0f, (1.0f - y) * (1.0f + y)));
    float sp, cp;
    sincospif(2.0f * ((float)col + fv) / (float)Me, &sp, &cp);
    EnvDir e;
    e.w = f3(sn * sp, y, sn * cp);
    e.weight = L.area * (zt - zb) * (2.0f * FR_PI / (float)Me);
    e.texel = row * Me + col;
    return e;
}

// Texel (row, col) containing unit direction w.
FR_D void env_texel_of(float3 w, int Me, int& row, int& col) {
    const float th = acosf(fminf(1.0f, fmaxf(-1.0f, w.y)));
    float ph = atan2f(w.x, w.z);
    if (ph < 0.0f) ph += 2.0f * FR_PI;
    row = min(Me - 1, max(0, (int)floorf(th * (float)Me / FR_PI)));
    col = min(Me - 1, max(0, (int)floorf(ph * (float)Me / (2.0f * FR_PI))));
}

FR_D bool env_block_has(const LightDev& L, int row, int col) {
    return row >= (int)L.c.x && row < (int)L.c.y && col >= (int)L.c.z && col < (int)L.e1.x;
}

// Bilinear footprint: texel centres at u*M - 1/2, clamp-to-edge.
struct Tap {
    int i00, i10, i01, i11;
    float fx, fy;
};

FR_D Tap make_tap(int M, float u, float v) {
    const float x = u * (float)M - 0.5f, y = v * (float)M - 0.5f;
    const float x0 = floorf(x), y0 = floorf(y);
    Tap t;
    t.fx = x - x0;
    t.fy = y - y0;
    const int ix0 = min(max((int)x0, 0), M - 1), ix1 = min(max((int)x0 + 1, 0), M - 1);
    const int iy0 = min(max((int)y0, 0), M - 1), iy1 = min(max((int)y0 + 1, 0), M - 1);
    t.i00 = iy0 * M + ix0;
    t.i10 = iy0 * M + ix1;
    t.i01 = iy1 * M + ix0;
    t.i11 = iy1 * M + ix1;
    return t;
}

FR_D float bil(const Tap& t, float a00, float a10, float a01, float a11) {
    return (1.0f - t.fx) * (1.0f - t.fy) * a00 + t.fx * (1.0f - t.fy) * a10 +
           (1.0f - t.fx) * t.fy * a01 + t.fx * t.fy * a11;
}

// value, d/du and d/dv (u, v in texture-coordinate units) of channel ch of a
// C-channel texture
FR_D float tap_fetch(const float* tex, int C, int ch, const Tap& t, int M, float* du, float* dv) {
    const float a00 = __ldg(&tex[t.i00 * C + ch]), a10 = __ldg(&tex[t.i10 * C + ch]);
    const float a01 = __ldg(&tex[t.i01 * C + ch]), a11 = __ldg(&tex[t.i11 * C + ch]);
    if (du) *du = (float)M * ((1.0f - t.fy) * (a10 - a00) + t.fy * (a11 - a01));
    if (dv) *dv = (float)M * ((1.0f - t.fx) * (a01 - a00) + t.fx * (a11 - a10));
    return bil(t, a00, a10, a01, a11);
}

struct Material {
    float3 c, s;
    float r;
};

// ---------------------------------------------------------------------------
// Smith masking G1 with its partials w.r.t. n.v and r (App. A, Eq. brdf_g1).
// Shading arithmetic uses the hardware's approximate divide, reciprocal
// square root, power and logarithm (a few ulp: far inside the 1e-4 radiance
// and 1e-3 gradient tolerances); the ray-triangle and traversal arithmetic
// stays IEEE.
// ---------------------------------------------------------------------------
// callers pass n.v > 0, so Delta(h.v / n.v) (Eq. brdf_g1_chi) is h.v > 0
FR_D float g1_walter(float nv, float hv, float r, float& d_nv, float& d_r) {
    d_nv = d_r = 0.0f;
    if (!(hv > 0.0f)) return 0.0f;
    const float s2 = 1.0f - nv * nv;
    if (s2 <= 0.0f) return 1.0f;
    const float rs = rsqrtf(s2);                   // 1 / sin
    const float a = __fdividef(nv * rs, r);        // Eq. brdf_g1_a: cot / r
    if (a >= 1.6f) return 1.0f;
    const float num = 3.535f * a + 2.181f * a * a;
    const float den = 1.0f + 2.276f * a + 2.577f * a * a;
    const float inv_den = __fdividef(1.0f, den);
    const float dG_da = ((3.535f + 4.362f * a) * den - num * (2.276f + 5.154f * a)) * inv_den * inv_den;
    d_nv = __fdividef(dG_da * rs * rs * rs, r);    // da/d(n.v) = 1 / (r sin^3)
    d_r = -__fdividef(dG_da * a, r);
    return num * inv_den;
}

FR_D float g1_ggx(float nv, float hv, float r, float& d_nv, float& d_r) {
    d_nv = d_r = 0.0f;
    if (!(hv > 0.0f)) return 0.0f;
    const float a2 = r * r;
    const float S2 = a2 + (1.0f - a2) * nv * nv;
    const float iS = rsqrtf(S2), S = S2 * iS;
    const float den = nv + S;
    const float inv_den2 = __fdividef(1.0f, den * den);
    const float dS_dnv = (1.0f - a2) * nv * iS;
    const float dS_dr = r * (1.0f - nv * nv) * iS;
    d_nv = 2.0f * (S - nv * dS_dnv) * inv_den2;
    d_r = -2.0f * nv * dS_dr * inv_den2;
    return __fdividef(2.0f * nv, den);
}

// Reverse-mode accumulators of one shading point.
struct ShadeAdj {
    float3 n, l, o, c, s;
    float r;
};

// f_r = f_d + f_s (Eq. brdf).  Zero unless n.l > 0; the specular lobe only
// where n.o > 0 (its denominator, Eq. brdf_spec), the Lambert term whatever
// the view.  With ADJ, propagates the upstream gradient gf (d/d f_r per
// channel) into g.
template <bool ADJ>
FR_D float3 brdf(uint32_t flags, float3 n, float3 l, float3 o, const Material& m, float3 gf,
                 ShadeAdj* g) {
    const float nl = dot(n, l), no = dot(n, o);
    if (!(nl > 0.0f)) return f3(0.0f, 0.0f, 0.0f);
    if (!(no > 0.0f)) {                                      // Lambert term alone
        if (ADJ) g->c += gf * (1.0f / FR_PI);
        return m.c * (1.0f / FR_PI);
    }
    const float3 hv = l + o;
    const float inv_hlen = rsqrtf(dot(hv, hv));
    const float3 h = hv * inv_hlen;                          // Eq. halfVector (reading)
    const float nh = dot(n, h), oh = dot(o, h), lh = dot(l, h);
    float Dt, dD_dnh, dD_dr;
    const float r = m.r;
    float dG1o_dno, dG1o_dr, dG1l_dnl, dG1l_dr, G1o, G1l;
    if (flags & FR_FLAG_GGX_D) {
        const float a2 = r * r;
        const float den = nh * nh * (a2 - 1.0f) + 1.0f;
        const float i2 = __fdividef(1.0f, FR_PI * den * den), i3 = __fdividef(i2, den);
        Dt = a2 * i2;
        dD_dnh = -4.0f * a2 * nh * (a2 - 1.0f) * i3;
        dD_dr = 2.0f * r * i2 - 4.0f * a2 * r * nh * nh * i3;
        G1o = g1_ggx(no, oh, r, dG1o_dno, dG1o_dr);
        G1l = g1_ggx(nl, lh, r, dG1l_dnl, dG1l_dr);
    } else {
        // Eq. brdf_d (reading): (alpha + 2)/(2 pi) (n.h)^alpha, alpha = 2/r - 2
        const float ir = __fdividef(1.0f, r);
        const float alpha = 2.0f * ir - 2.0f;
        const float p = __powf(nh, alpha);                   // n.h > 0 here (n.l, n.o > 0)
        Dt = p * ir * (1.0f / FR_PI);
        if (ADJ) {
            dD_dnh = __fdividef(Dt * alpha, nh);
            dD_dr = Dt * (-ir - 2.0f * __logf(nh) * ir * ir);
        } else {
            dD_dnh = dD_dr = 0.0f;
        }
        G1o = g1_walter(no, oh, r, dG1o_dno, dG1o_dr);     // Eq. brdf_g
        G1l = g1_walter(nl, lh, r, dG1l_dnl, dG1l_dr);
    }
    const float G = G1o * G1l;
    const float base = 1.0f - oh;
    const bool lin = (flags & FR_FLAG_SCHLICK_LINEAR_D) != 0;
    const float b2 = base * base;
    const float w5 = lin ? base : b2 * b2 * base;            // Eq. brdf_f (Schlick)
    const float inv_denom = __fdividef(1.0f, 4.0f * no * nl);   // Eq. brdf_spec
    const float Q = Dt * G * inv_denom;
    const float3 F = f3(m.s.x + (1.0f - m.s.x) * w5, m.s.y + (1.0f - m.s.y) * w5,
                        m.s.z + (1.0f - m.s.z) * w5);
    const float inv_pi = 1.0f / FR_PI;
    const float3 f = f3(m.c.x * inv_pi + Q * F.x, m.c.y * inv_pi + Q * F.y, m.c.z * inv_pi + Q * F.z);
    if (ADJ) {
        g->c += gf * inv_pi;
        const float gQ = gf.x * F.x + gf.y * F.y + gf.z * F.z;
        g->s += f3(gf.x * Q * (1.0f - w5), gf.y * Q * (1.0f - w5), gf.z * Q * (1.0f - w5));
        const float gw5 = Q * (gf.x * (1.0f - m.s.x) + gf.y * (1.0f - m.s.y) + gf.z * (1.0f - m.s.z));
        const float goh_f = gw5 * (lin ? -1.0f : -5.0f * b2 * b2);
        const float gDt = gQ * G * inv_denom, gG = gQ * Dt * inv_denom;
        float gno = -__fdividef(gQ * Q, no), gnl = -__fdividef(gQ * Q, nl);
        const float gG1o = gG * G1l, gG1l = gG * G1o;
        gno += gG1o * dG1o_dno;
        gnl += gG1l * dG1l_dnl;
        g->r += gG1o * dG1o_dr + gG1l * dG1l_dr + gDt * dD_dr;
        const float gnh = gDt * dD_dnh;
        const float3 gh = n * gnh + o * goh_f;
        g->n += h * gnh;
        g->o += h * goh_f;
        const float3 ghv = (gh - h * dot(h, gh)) * inv_hlen;
        g->l += ghv;
        g->o += ghv;
        g->n += o * gno + l * gnl;
        g->o += n * gno;
        g->l += n * gnl;
    }
    return f;
}
