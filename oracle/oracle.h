/*
 * FP64 CPU oracle for the differentiable ray-traced face render (Dib et al.,
 * Eurographics 2021).  TEST INFRASTRUCTURE ONLY: it is loaded by the tests, by
 * the smoke check and by the benchmark's CPU-baseline leg, never by the product
 * path.  It shares no code with the CUDA library.
 *
 * All inputs are the float32 arrays drawn by the synthetic generators; they are
 * widened exactly to double and every step runs in double precision.
 */
#ifndef FACE_ORACLE_H
#define FACE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* flags */
#define ORA_GGX            1u   /* GGX D and exact GGX Smith G1 instead of the paper's Blinn-Phong/Walter */
#define ORA_SCHLICK_LINEAR 2u   /* Fresnel exactly as printed in App. A, without the 5th power */
#define ORA_FLAT           4u   /* debug: radiance = diffuse albedo at the hit, no lights */
#define ORA_DIFFUSE_ONLY   8u   /* debug: f_r = c / pi (no specular lobe) */
#define ORA_VIEW_CUTOFF 1024u   /* every contribution zero where n_s . o <= 0 (the grazing cutoff applied to
                                   the diffuse term too); the boundary term of the curve n_s . o = 0
                                   (ORA_TERM_SPECULAR) then carries the whole jump there */

/* emitter type of a light record (the other types are 0 quad, 1 triangle, 2 disk):
 * a block of texels of an environment map of lights at infinity (Sec. 7,
 * environment map vs light stage).  Record {3, i0, i1, j0, j1, unused...}: rows
 * [i0, i1) x columns [j0, j1) of the env_size x env_size map; row i holds the
 * polar angles [i, i + 1] pi / env_size from camera-space +y, column j the
 * azimuths [j, j + 1] 2 pi / env_size from +z towards +x.  The radiance from
 * direction w is the map's texel containing w (OraParams.env, RGB). */
#define ORA_LIGHT_ENV 3

/* gradient terms */
#define ORA_TERM_INTERIOR  1u
#define ORA_TERM_PRIMARY   2u
#define ORA_TERM_SHADOW    4u
#define ORA_TERM_SPECULAR  8u   /* boundary of the specular lobe inside triangles: the curve n_s . o = 0 */

typedef struct OraScene {
    int32_t n_vertices, n_triangles, n_basis;
    const float* mean;      /* [N*3] */
    const float* basis;     /* [K][N*3] */
    const int32_t* faces;   /* [T*3] */
    const float* uv;        /* [N*2] */
    int32_t n_lights;
    const float* lights;    /* [N_L*11] emitter records */
    const float* light_d;   /* [N_L] */
    const float* light_a;   /* [N_L] */
    int32_t width, height, spp, tex_size, edge_spp;
    uint32_t seed, flags;
    int32_t n_threads;
    /* optional virtual light stage (Sec. 3.3), [N_L][12]: stage centre, then the
     * unit-scale face vertices V0, V1, V2 of light j's polyhedron face; with
     * OraParams light_d/a/p the emitters are built from them (triangles) */
    const float* stage;
    int32_t env_size;       /* texels per side of the environment map (0: no ORA_LIGHT_ENV records) */
} OraScene;

typedef struct OraParams {
    const float *coef, *rot, *trans, *focal, *light_i, *diffuse, *specular, *roughness;
    /* optional light geometry of a stage scene: distance d_j [N_L], relative
     * area a_j [N_L], barycentric centre (p_j0, p_j1) [N_L][2] (p_j2 = 1 - both) */
    const float *light_d, *light_a, *light_p;
    /* environment-map radiance [env_size][env_size][3] (scenes with ORA_LIGHT_ENV records) */
    const float* env;
} OraParams;

/* rays traced by this library since the last reset (closest-hit + shadow) */
unsigned long long ora_ray_count(int reset);

void ora_philox(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1, uint32_t c2,
                uint32_t c3, uint32_t out[4]);

int ora_geometry(const OraScene* s, const OraParams* p, double* v_cam, double* n_vert);

int ora_edges(const OraScene* s, int32_t* edge_v, int32_t* edge_f);

int ora_silhouettes(const OraScene* s, const OraParams* p, int32_t* prim, int32_t* n_prim,
                    int32_t* per_light, int32_t* light_counts);

int ora_closest_hit(const OraScene* s, const OraParams* p, const double* org,
                    const double* dir, int32_t n, int32_t* tri, double* t);

int ora_render(const OraScene* s, const OraParams* p, uint32_t iteration, uint32_t face_id,
               const int32_t* pixels, int32_t n_pixels, double* image,
               int32_t* tri_rec, uint64_t* mask_rec);

double ora_loss(int32_t height, int32_t width, const double* image, const float* target,
                double* blurred, double* adjoint);

int ora_grad(const OraScene* s, const OraParams* p, uint32_t iteration, uint32_t face_id,
             const double* adjoint, uint32_t terms, double* g_coef, double* g_rot,
             double* g_trans, double* g_focal, double* g_light, double* g_diffuse,
             double* g_specular, double* g_roughness, double* g_light_geom /* [N_L][4] or NULL */,
             double* g_env /* [env_size][env_size][3] or NULL */);

/* Crossings of image scanline `scan` with the curve n_s . o = 0 inside the
 * front-facing triangles (the boundary of the specular lobe): scanlines
 * 0 .. H*k-1 are rows y = (i + u)/k, then W*k columns, k = max(edge_spp, 1),
 * u a uniform offset per line from the specular-edge stream.  Writes up to
 * `max` crossings as (triangle, root index along the line) pairs and screen
 * points (x, y); returns their count (-1: scan out of range). */
int ora_spec_crossings(const OraScene* s, const OraParams* p, uint32_t iteration, uint32_t face_id, int32_t scan,
                       int32_t max, int32_t* tri_root, double* xy);

double ora_brdf(uint32_t flags, const double* n, const double* l, const double* o,
                const double* c, const double* s, double r, double* out_rgb);

void ora_brdf_terms(uint32_t flags, const double* n, const double* l, const double* o, double r,
                    double* out);

int ora_point_light_grad(const OraScene* s, const OraParams* p, const double* y,
                         const double* n, int32_t tri_self, int32_t n_samples,
                         uint32_t seed_stream, double* value_rgb, double* g_coef,
                         double* g_light_geom /* [N_L][4] channel 0, or NULL */);

#ifdef __cplusplus
}
#endif
#endif
