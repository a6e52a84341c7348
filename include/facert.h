/*
 * facert: differentiable Monte Carlo ray-traced rendering of a morphable face
 * lit by a virtual light stage (Dib et al., "Practical Face Reconstruction via
 * Differentiable Ray Tracing", Eurographics 2021), as a C-ABI library of
 * hand-written CUDA kernels for sm_103a.
 *
 * Problem statement (Sec. 4, Eq. energy): for parameters chi, render the image
 * p^S = F(chi) with the Monte Carlo estimator F of the rendering equation
 * (direct light from every light-stage emitter, shadow rays, Cook-Torrance
 * reflectance of App. A), compare it with a target through the L1 photometric
 * loss E_ph after the 3x3 Gaussian smoothing of Sec. 4 ("Variance Reduction"),
 * and return dE/dchi including the edge-sampling boundary terms (Sec. 4,
 * "Edge Sampling").
 *
 * Conventions shared by every call
 *  - Return value: FR_OK (0) or an error code; no exceptions cross the ABI.
 *    Argument checks happen synchronously before anything is enqueued.
 *    fr_last_error() describes the last failure of a context.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Compute calls only enqueue work and return; they never allocate.  The
 *    reverse pass also uses a stream the context owns (created at fr_create),
 *    forked from `stream` and joined back into it with events inside the call,
 *    so all of a call's work is ordered before later work on `stream`.
 *  - Device-side problems (traversal stack overflow, bounded waits that ran
 *    out) set a status word that fr_sync_status() reads; no kernel traps.
 *  - Ownership: the caller owns every buffer it passes (parameters, targets,
 *    images, gradients) and the stream; the context owns its own scratch (mesh
 *    copies, BVH, edge lists, adjoint accumulators), sized at fr_create /
 *    fr_set_mesh / fr_set_lights and freed by fr_destroy.
 *  - A context is not re-entrant: calls on one context must be serialised on
 *    one stream.  Separate contexts are independent.
 *  - Layouts are C-contiguous float32 unless stated: image/target [H][W][3];
 *    textures diffuse/specular [M][M][3], roughness [M][M] (row = v axis).
 */
#ifndef FACERT_H
#define FACERT_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t fr_status;
#define FR_OK        0
#define FR_EINVAL    1   /* bad argument (null pointer, size out of range, state) */
#define FR_ENOMEM    2   /* device allocation failed at create/set time */
#define FR_ECUDA     3   /* a CUDA runtime call failed */
#define FR_EOVERFLOW 4   /* device status: traversal stack overflowed (rays dropped) */
#define FR_ETIMEOUT  5   /* device status: a bounded wait gave up */

/* config flags */
#define FR_FLAG_GGX              1u   /* GGX D + exact GGX Smith G1 instead of App. A's Blinn-Phong/Walter */
#define FR_FLAG_SCHLICK_LINEAR   2u   /* Fresnel exactly as printed in App. A (no 5th power) */
#define FR_FLAG_FLAT             4u   /* debug: radiance = diffuse albedo at the hit, no lights */
#define FR_FLAG_NO_INTERIOR     16u   /* gradient: skip the interior (visibility-fixed) term */
#define FR_FLAG_NO_PRIMARY_EDGE 32u   /* gradient: skip the primary-visibility boundary term */
#define FR_FLAG_NO_SHADOW_EDGE  64u   /* gradient: skip the shadow boundary term */
#define FR_FLAG_NO_SPECULAR_EDGE 2048u /* gradient: skip the boundary term of the specular lobe's
                                         cutoff curve n_s . o = 0 inside triangles */
#define FR_FLAG_MORPH_BF16     128u   /* morph as one BF16 tensor-core GEMM over the batch (FP32
                                         accumulate, FP32 mean); context-wide, read by every call */
#define FR_FLAG_RECOMPUTE      256u   /* the adjoint re-traces its camera and shadow rays inside the
                                         adjoint kernel, neither reading the forward's hit records nor
                                         recomputing them in tiles (see fr_render) */
#define FR_FLAG_VIEW_CUTOFF   1024u   /* zero every contribution where the shading normal faces away from
                                         the camera (n_s . o <= 0), the diffuse term included; by default
                                         only the specular lobe needs n_s . o > 0.  Either way the image
                                         jumps on the curve n_s . o = 0 inside triangles, which the
                                         specular-boundary term samples */
#define FR_FLAG_LBVH           512u   /* rebuild an LBVH (Morton sort + Karras tree) every call instead
                                         of refitting the SAH topology built from the mean face at
                                         fr_set_mesh; for deformations far from the mean face.
                                         Context-wide, read from the context's flags */

/* Per-slot budget for hit records (bytes): the hit triangle and two 64-bit
 * light-visibility words per camera sample (20 bytes; with at most 64 lights
 * only the first word is written and read).  When the context's
 * width * height * spp records fit, a fused step's forward writes them and its
 * adjoint reads them instead of re-tracing.  Larger images are split into equal
 * tiles that fit (whole pixels, whole 128-sample blocks): the forward keeps the
 * records of the image's last tile, and the adjoint, from the last tile to the
 * first, reads those and recomputes every other tile's records with a
 * visibility-only forward pass (the same Philox counters, no shading) before
 * reading them.  The gradient is the same either way. */
#define FR_RECORDS_BUDGET (256u << 20)

/* emitter types in light records */
#define FR_LIGHT_QUAD 0
#define FR_LIGHT_TRI  1
#define FR_LIGHT_DISK 2
#define FR_LIGHT_ENV  3   /* block of an environment map of lights at infinity (Sec. 7) */
#define FR_MAX_ENV   64   /* largest environment map: FR_MAX_ENV x FR_MAX_ENV texels */

typedef struct fr_ctx fr_ctx;

typedef struct fr_config {
    int32_t width, height;   /* image size, 1..8192 each */
    int32_t spp;             /* camera samples per pixel: a power of two, 1..256 */
    int32_t tex_size;        /* M: textures are M x M, 1..8192 */
    int32_t edge_spp;        /* primary-edge samples per pixel (0..64) */
    uint32_t flags;          /* FR_FLAG_* */
    uint32_t seed;           /* Philox key word 0 */
    int32_t max_batch;       /* faces per fr_render_batch call, 0..64 (0 means 1); each gets a slot
                                of scratch sized for width x height pixels */
} fr_config;

/* Face model of Sec. 3.1 (host pointers, copied into the context):
 *   mean  [N][3]      mean shape a_s (model space)
 *   basis [K][N][3]   columns of [Sigma_s | Sigma_e]; v = mean + basis^T coef
 *   faces [T][3]      triangle vertex indices (manifold: each edge in <= 2 faces)
 *   uv    [N][2]      texture coordinates (u, v) in [0, 1]  (Sec. 3.2) */
typedef struct fr_mesh {
    int32_t n_vertices, n_triangles, n_basis;
    const float* mean;
    const float* basis;
    const int32_t* faces;
    const float* uv;
} fr_mesh;

/* Virtual light stage of Sec. 3.3 (host pointers, copied):
 *   records [N_L][11] = {type, c[3], e1[3], e2[3], unused}; quad: c + (u-1/2) e1 +
 *   (v-1/2) e2; triangle: c, c+e1, c+e2; disk: centre c, radius vectors e1, e2.
 *   The emitting side is the one e1 x e2 points to.  Geometry is in camera space.
 *   d [N_L], a [N_L]: distance and relative area of Eq. (lightIntensity); the
 *   emitted radiance is (d^2 / a) * i_j.  N_L <= 128.
 *   FR_LIGHT_ENV records {3, i0, i1, j0, j1, unused...} replace the light stage
 *   by an environment map of lights at infinity (the alternative the paper
 *   compares in Sec. 7): the record is the block of texel rows [i0, i1) and
 *   columns [j0, j1) of an env_size x env_size latitude-longitude map, row i
 *   spanning polar angles [i, i + 1] pi / env_size from camera-space +y and
 *   column j azimuths [j, j + 1] 2 pi / env_size from +z towards +x.  The
 *   radiance arriving from direction w is the texel of fr_params.env containing
 *   w (d, a and i_j are not used).  Each camera sample draws one direction per
 *   block: a texel uniformly among the block's (from the 24-bit integers behind
 *   the block's two uniforms: row = i0 + floor(k_u R / 2^24), the remainder
 *   placing the sample inside the row; columns likewise), then a direction
 *   uniform in solid angle inside the texel; its shadow ray runs from the hit
 *   point along w with t > 1e-4.  Blocks may be mixed with area emitters, not
 *   with a virtual light stage. */
typedef struct fr_light_stage {
    int32_t n_lights;
    const float* records;
    const float* d;
    const float* a;
    /* optional (NULL: the records are the lights): the virtual light stage of
     * Sec. 3.3, [N_L][12] per light: stage centre C, then the unit-scale face
     * V0, V1, V2 of its polyhedron face (counter-clockwise seen from outside).
     * A call whose fr_params carries light_d, light_a and light_p builds light
     * j from them instead of the record: the face scaled by d_j about C,
     * shrunk by sqrt(a_j) about the point p0 V0 + p1 V1 + (1 - p0 - p1) V2
     * (scaled), parallel to the face, emitting towards C, with emitted radiance
     * (d_j^2 / a_j) i_j; the gradients then include d/d(d_j, a_j, p_j)
     * (interior and moving-emitter shadow-boundary terms). */
    const float* stage;
    /* texels per side of the environment map of FR_LIGHT_ENV records,
     * 1..FR_MAX_ENV (0: no such records) */
    int32_t env_size;
} fr_light_stage;

/* Parameters chi-hat of Sec. 4 (device pointers, float32):
 *   coef [K] (alpha then delta), rot [3] Euler angles with R = Rz Ry Rx,
 *   trans [3] T (pose v' = R^T (v - T), Sec. 3.1), focal [1] in pixels,
 *   light_i [N_L][3] perceived intensities i_j, diffuse [M][M][3],
 *   specular [M][M][3], roughness [M][M]; optionally (all three or none, with
 *   a stage set by fr_set_lights) the light geometry light_d [N_L],
 *   light_a [N_L] in (0, 1], light_p [N_L][2] (barycentric p0, p1); env
 *   [env_size][env_size][3] the environment map's radiance (required when the
 *   lights include FR_LIGHT_ENV records, else ignored). */
typedef struct fr_params {
    const float *coef, *rot, *trans, *focal, *light_i, *diffuse, *specular, *roughness;
    const float *light_d, *light_a, *light_p;
    const float* env;
} fr_params;

/* Gradients, same shapes as fr_params (device pointers).  Every call ADDS
 * into them; the caller zeroes them.  A NULL member skips that group's
 * output (the work is still done). */
typedef struct fr_grads {
    float *coef, *rot, *trans, *focal, *light_i, *diffuse, *specular, *roughness;
    float *light_d, *light_a, *light_p;
    float* env;
} fr_grads;

/* Create a context for one image configuration.  Allocates the image-sized
 * loss scratch and the status/counter words.  Errors: FR_EINVAL (bad sizes),
 * FR_ENOMEM. */
fr_status fr_create(fr_ctx** out, const fr_config* cfg);

/* Copy a face model (Sec. 3.1) and build its static topology (vertex->face
 * lists, the undirected edge list sorted by (min vertex, max vertex)); sizes the
 * context's scratch.  Synchronous.  Errors: FR_EINVAL (indices out of range,
 * non-manifold edge, T < 1, K > 256), FR_ENOMEM, FR_ECUDA. */
fr_status fr_set_mesh(fr_ctx* ctx, const fr_mesh* mesh);

/* Copy the light-stage emitters (Sec. 3.3).  Synchronous.  Errors: FR_EINVAL
 * (unknown type, N_L out of range, an FR_LIGHT_ENV block outside the map or
 * env_size out of range, environment blocks together with a stage). */
fr_status fr_set_lights(fr_ctx* ctx, const fr_light_stage* stage);

/* Statistical albedo model of Sec. 3.2 in UV texture space (host pointers,
 * copied): diffuse C = a_r + Sigma_r beta and specular S = a_b + Sigma_b gamma,
 * each [M][M][3] with M = tex_size.  mean_* [M*M*3]; basis_* [K][M*M*3]
 * (column k contiguous); 0 <= K <= 256 per model (K = 0: the mean alone).
 * Stage I of Sec. 4 optimises beta and gamma through these; Stage II starts
 * the per-texel albedos from the result.  Synchronous.  Errors: FR_EINVAL,
 * FR_ENOMEM, FR_ECUDA. */
typedef struct fr_albedo_model {
    int32_t k_diffuse, k_specular;
    const float* mean_diffuse;
    const float* basis_diffuse;
    const float* mean_specular;
    const float* basis_specular;
} fr_albedo_model;
fr_status fr_set_albedo(fr_ctx* ctx, const fr_albedo_model* model);

/* Landmark vertices for the sparse landmark loss of Sec. 4, Eq. (landmark):
 * n (1..256) vertex indices of the mesh (host, copied).  Requires the mesh.
 * Errors: FR_EINVAL (index out of range), FR_ENOMEM. */
fr_status fr_set_landmarks(fr_ctx* ctx, int32_t n, const int32_t* vertex_index);

/* E_land = sum_l || Pi(Gamma(v_l)) - z_l ||^2 for the face p (coef, rot,
 * trans, focal are read; textures and lights are not), image width x height
 * (principal point at its centre, y down, pixel units as the camera rays use),
 * z [L][2] target positions (device).  *loss (device double) = weight * E_land;
 * if g != NULL, weight * dE_land/d(coef, rot, trans, focal) is ADDED into g
 * (null members skipped); if projected != NULL it receives Pi(Gamma(v_l))
 * [L][2] (device).  FP64 throughout, one small launch. */
fr_status fr_landmark_loss(fr_ctx* ctx, const fr_params* p, int32_t width, int32_t height, const float* z,
                           float weight, double* loss, fr_grads* g, float* projected, void* stream);

/* Statistical albedos of n faces (1 <= n <= max_batch; host arrays of n device
 * pointers): diffuse[b] = a_r + Sigma_r beta[b] and specular[b] = a_b +
 * Sigma_b gamma[b], textures [M][M][3] (16-byte aligned), beta[b] [K_r],
 * gamma[b] [K_b].  One launch per model for the whole batch: BF16 x BF16 ->
 * FP32 tensor-core GEMM when the context has FR_FLAG_MORPH_BF16, else FP32.
 * A NULL diffuse or specular array skips that model.  Errors: FR_EINVAL (no
 * model set, bad n, null or misaligned pointer). */
fr_status fr_albedo_morph(fr_ctx* ctx, int32_t n, const float* const* beta, const float* const* gamma,
                          float* const* diffuse, float* const* specular, void* stream);

/* Transpose of fr_albedo_morph for the adjoint: g_beta[b] += Sigma_r^T
 * g_diffuse[b] and g_gamma[b] += Sigma_b^T g_specular[b] (FP32 products, FP64
 * sums in a fixed order, so results are reproducible).  g_diffuse/g_specular
 * are texture gradients [M][M][3] as fr_render adds them (16-byte aligned).
 * A NULL g_beta or g_gamma array skips that model. */
fr_status fr_albedo_adjoint(fr_ctx* ctx, int32_t n, const float* const* g_diffuse, const float* const* g_specular,
                            float* const* g_beta, float* const* g_gamma, void* stream);

/* Forward render (Sec. 4, F): morph, pose, normals, LBVH build, primary rays,
 * Cook-Torrance shading (App. A) with one area sample and one shadow ray per
 * light per camera sample.  image [H][W][3] receives the per-pixel mean.
 * `iteration` and `face_id` enter the Philox counters, so a call is a pure
 * function of (params, iteration, face_id, seed). */
fr_status fr_forward(fr_ctx* ctx, const fr_params* p, float* image, uint32_t iteration,
                     uint32_t face_id, void* stream);

/* Adjoint of fr_forward: adds d(sum adj_image * image)/dchi into g.  Re-traces
 * with the same Philox counters instead of storing hit records, and includes
 * the primary-visibility and shadow boundary terms (edge sampling, Sec. 4)
 * and the boundary term of the specular lobe's cutoff inside triangles (the
 * curve n_s . o = 0 of App. A, Eq. brdf_spec, met along one row line per
 * pixel row and one column line per pixel column, edge_spp of each, rows
 * first; (W + H) * max(edge_spp, 1) <= 65535) unless disabled by flags.
 * adj_image [H][W][3] (device).  The boundary terms of the primary edges and
 * of the specular cutoff, and the texture-gradient flush, run on a stream of
 * the context, forked from `stream` and joined back into it with events. */
fr_status fr_backward(fr_ctx* ctx, const fr_params* p, const float* adj_image, fr_grads* g,
                      uint32_t iteration, uint32_t face_id, void* stream);

/* Photometric loss of Sec. 4: blurred = G3x3 * image (sigma 1, normalised,
 * replicate border); *loss = sum |blurred - target| (device double, stored, not
 * accumulated); adj_image = dloss/dimage.  blurred may be NULL.  The sum is an
 * FP64 reduction in a fixed order (per-block partials added in block order),
 * so repeated calls give bitwise the same loss. */
fr_status fr_loss(fr_ctx* ctx, const float* image, const float* target, double* loss,
                  float* adj_image, float* blurred, void* stream);

/* One full step of the hot path: fr_forward, fr_loss against `target`, and (if
 * g != NULL) fr_backward with the loss adjoint.  loss is a device double.
 * Within the step the adjoint reuses the forward's per-sample hit records
 * (hit triangle and shadow visibility) when they fit FR_RECORDS_BUDGET, else
 * those of the image's last tile and recomputes the others tile by tile; with
 * FR_FLAG_RECOMPUTE it re-traces every sample inside the adjoint kernel
 * instead.  The gradient is the same either
 * way.  With g, the part of the adjoint that needs only the posed geometry
 * runs on a stream of the context beside the forward, the boundary terms of
 * the primary edges and of the specular lobe's cutoff run there beside the
 * interior term, and the texture gradients are flushed there beside the chain
 * to the vertex parameters; each piece is forked from `stream` and joined back
 * into it with events before the call's last work on `stream` (the call still
 * returns without synchronising, and a stream capture of it records the forks
 * and joins). */
fr_status fr_render(fr_ctx* ctx, const fr_params* p, const float* target, float* image,
                    double* loss, fr_grads* g, uint32_t iteration, uint32_t face_id,
                    void* stream);

/* One face of a batched call: its image configuration (width * height at most
 * the context's width * height; spp a power of two <= 256; edge_spp <= 64),
 * flags, Philox iteration and face id, parameters (device), target image,
 * output image [height][width][3], loss (device double) and gradients (NULL:
 * forward + loss only; otherwise ADDED into, like fr_grads). */
typedef struct fr_item {
    int32_t width, height, spp, edge_spp;
    uint32_t flags, iteration, face_id;
    fr_params params;
    const float* target;
    float* image;
    double* loss;
    fr_grads* grads;
} fr_item;

/* fr_render for n faces at once (1 <= n <= max_batch), sharing the context's
 * face model and light stage: item k uses slot k.  Each stage of the hot path
 * (morph, pose and normals, LBVH build, forward, loss, adjoint, edge terms,
 * chain to parameters) is one launch over all items, so faces of different
 * sizes and sample counts share the GPU inside one launch.  Results equal n
 * separate fr_render calls with the same arguments; the reverse pass uses the
 * context's second stream as fr_render does. */
fr_status fr_render_batch(fr_ctx* ctx, const fr_item* items, int32_t n, void* stream);

/* Replace the FR_FLAG_* set of ctx for the following calls (e.g. drop the edge
 * terms when only textures are optimised).  Errors: FR_EINVAL. */
fr_status fr_set_flags(fr_ctx* ctx, uint32_t flags);

/* Test hook: recompute hit records in tiles of `samples` camera samples
 * (rounded down to a multiple of max(128, spp), at most the slots' record
 * buffer) instead of the buffer's full size, so that small images exercise
 * the tiled adjoint; 0 restores the default.  Images whose records no longer
 * fit one tile are then not recorded by the forward.  FR_EINVAL if samples < 0. */
fr_status fr_debug_record_tile(fr_ctx* ctx, int64_t samples);

/* Synchronise `stream`, read and clear the device status word.
 * Returns FR_OK, FR_EOVERFLOW or FR_ETIMEOUT (or FR_ECUDA).  FR_ETIMEOUT after a
 * wait whose CTA could not also drain its own copies or tensor-core MMAs in a
 * second bounded wait marks the context unusable: a late write could land in
 * memory that has since been reused, so every later compute call on it returns
 * FR_ECUDA; destroy it and create a new one. */
fr_status fr_sync_status(fr_ctx* ctx, void* stream);

/* Human-readable description of the last error on ctx (never NULL). */
const char* fr_last_error(const fr_ctx* ctx);

/* Free every device buffer of the context (synchronises the device first). */
void fr_destroy(fr_ctx* ctx);

/* ---- diagnostics (used by the parity tests; same rules as above) ---- */

/* Philox4x32-10 (Salmon et al., SC'11) on the device: out[i][0..3] =
 * philox(key=(k0,k1), counter=counters[i][0..3]) for i < n (device arrays). */
fr_status fr_philox(uint32_t k0, uint32_t k1, const uint32_t* counters, int32_t n,
                    uint32_t* out, void* stream);

/* Camera-space vertices v' [N][3] and unit vertex normals [N][3] (device) of
 * the morph + pose of Sec. 3.1 for parameters p. */
fr_status fr_debug_geometry(fr_ctx* ctx, const fr_params* p, float* v_cam, float* n_vert,
                            void* stream);

/* Closest hit of n rays (device org [n][3], dir [n][3]) through the LBVH built
 * for p: tri [n] (-1 = miss), t [n] (-1 on a miss). */
fr_status fr_debug_trace(fr_ctx* ctx, const fr_params* p, const float* org, const float* dir,
                         int32_t n, int32_t* tri, float* t, void* stream);

/* Forward render that also writes per-sample records: tri_rec [H*W*spp] hit
 * triangle (-1 miss) and mask_rec [H*W*spp][2] visibility words: bit j of word
 * w = the shadow ray to light 64 w + j was traced and is unoccluded; record
 * index = (y*W + x)*spp + sample. */
fr_status fr_debug_records(fr_ctx* ctx, const fr_params* p, float* image, int32_t* tri_rec,
                           uint64_t* mask_rec, uint32_t iteration, uint32_t face_id,
                           void* stream);

/* The bounded-wait error path without a fault: one CTA waits on an mbarrier
 * that nothing completes, with the poll loop of the tensor-core morph's
 * waits, gives up after `polls` polls (1..2^22) and sets the status word, so
 * the next fr_sync_status returns FR_ETIMEOUT and clears it; the context
 * stays usable. */
fr_status fr_debug_wait_timeout(fr_ctx* ctx, uint32_t polls, void* stream);

/* Ordered silhouette lists after a forward pass for p: prim [E] primary
 * silhouette edge ids, n_prim [1]; per_light [N_L][E] shadow candidates,
 * counts [N_L] (all device int32). */
fr_status fr_debug_silhouettes(fr_ctx* ctx, const fr_params* p, int32_t* prim, int32_t* n_prim,
                               int32_t* per_light, int32_t* counts, void* stream);

/* BVH validity check for p: writes out[0] = number of leaves reachable from the
 * root, out[1] = number of parent boxes that fail to contain a child box,
 * out[2] = maximum depth (device int32[3]). */
fr_status fr_debug_bvh(fr_ctx* ctx, const fr_params* p, int32_t* out, void* stream);

/* Morph only (Sec. 3.1), for n faces with parameters params[0..n) (host array
 * of device-pointer sets): out [n][N][3] (device) receives each face's
 * model-space vertices, through the BF16 tensor-core path when the context has
 * FR_FLAG_MORPH_BF16, else the FP32 path.  1 <= n <= max_batch. */
fr_status fr_debug_morph(fr_ctx* ctx, const fr_params* params, int32_t n, float* out, void* stream);

/* Edge count E of the mesh set on ctx (host int). */
int32_t fr_num_edges(const fr_ctx* ctx);

/* ---- measurement ---- */

/* Traversal work accumulated on ctx since the last reset, per kernel: out[3k+0]
 * rays traced, out[3k+1] BVH nodes visited, out[3k+2] ray/triangle tests, for
 * k = 0 forward, 1 adjoint (re-trace + shadow-boundary rays), 2 primary-edge
 * and specular-boundary rays (host uint64[9]).  Synchronises `stream`; reset != 0 zeroes them. */
fr_status fr_counters(fr_ctx* ctx, uint64_t* out, int32_t reset, void* stream);

/* Enable (on != 0) CUDA-event marks between the stages of fr_render. */
fr_status fr_set_timing(fr_ctx* ctx, int32_t on);

/* Milliseconds of the stages of the last timed fr_render (synchronises):
 * out[8] = {geometry+LBVH, forward, loss, classify, adjoint, screen-space
 * boundary terms (primary edges and the specular lobe's boundary), chain to
 * parameters, total}.  The marks are events on the caller's stream: work on
 * the context's side stream counts in the stage it overlaps (the
 * classification in the forward's, the boundary terms in the adjoint's), and
 * its own stage holds only what is left of it after that stage ends. */
fr_status fr_get_timing(fr_ctx* ctx, float* out);

/* Number of kernels this library has launched in this process. */
uint64_t fr_kernel_launches(void);

/* ---- optimiser: Adam with the regularisers of Sec. 4 (Eq. loss1, loss3) ---- */

#define FR_MAX_OPT_GROUPS 128
#define FR_GROUP_PLAIN    0   /* Adam only */
#define FR_GROUP_COEF     1   /* first n_prior elements: shape prior w_prior * x^2 (sigma_k = 1);
                                 the rest: soft box [0, 1] (expression), w_box * dist^2 */
#define FR_GROUP_LIGHT    2   /* intensities [N_L][3]: light prior w_prior * |I_j - m_j|^2 with
                                 I_j = aux[j] * i_j and m_j = mean(I_j) held fixed; soft box i >= 0 */
#define FR_GROUP_TEX_RGB  3   /* M x M x 3 texture: smoothness w_smooth * sum_i sum_{4-nbrs} |X_j - X_i|^2,
                                 symmetry w_sym * sum |X - flip(X)|_1 (flip: column c -> M-1-c),
                                 chromaticity w_chroma * sum |kappa(X) - kappa(aux)|_1 with
                                 kappa(c) = c / (c_r + c_g + c_b + 1e-6), soft box [0, 1] (w_box) */
#define FR_GROUP_TEX_MONO 4   /* M x M texture: smoothness, symmetry, soft box [0, 1] */
#define FR_GROUP_STAGE    5   /* virtual light stage geometry (Sec. 3.3) of N_L lights, x = [d (N_L) |
                                 a (N_L) | p (N_L x 2)], aux = the intensities i [N_L][3]: gradient of
                                 the light prior above through I_j = (d_j^2 / a_j) i_j (where a_j > 0;
                                 its energy is the LIGHT group's) and soft boxes (w_box) d_j >= 0,
                                 a_j in [0, 1] and light j inside its homothetic face: each corner's
                                 barycentric coordinate p_jm - sqrt(a_j) / 3 + sqrt(a_j) delta >= 0,
                                 i.e. p_jm >= sqrt(a_j) / 3 for m = 0, 1, 2, p_j2 = 1 - p_j0 - p_j1 */

/* One parameter group.  x, m, v (and g, aux when used) are device float32
 * arrays of n elements (aux: N_L scales for LIGHT, the M x M x 3 reference
 * albedo for TEX_RGB, the N_L x 3 intensities for STAGE).  aux2 is used by
 * LIGHT only: when aux is NULL the scales are d_j^2 / a_j computed from aux2
 * = [d (N_L) | a (N_L) | ...]: the x of the STAGE group ([d | a | p], 4 N_L
 * floats) at its pre-step values, or the lights' fixed d and a (2 N_L floats).
 * m and v must be zero before step 1.  After the update x
 * is clamped to [clamp_lo, clamp_hi] when clamp_lo < clamp_hi.  step > 0 gives
 * this group its own Adam step count (groups of different faces in one call);
 * step = 0 uses the call's step. */
typedef struct fr_opt_group {
    float* x;
    const float* g;
    float* m;
    float* v;
    const float* aux;
    const float* aux2;
    int32_t n, kind, width, n_prior;
    float lr, w_prior, w_box, w_sym, w_chroma, w_smooth, clamp_lo, clamp_hi;
    int32_t step;
} fr_opt_group;

/* One Adam step (Kingma & Ba; bias-corrected, step >= 1) over every group:
 * gradient = g + gradient of the group's regularisers at the current x, then
 * m = b1 m + (1 - b1) grad, v = b2 v + (1 - b2) grad^2,
 * x -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * Two launches on `stream` (moments, then update), so the stencils read the
 * pre-step values.  If reg_energy (device double) is given it receives the
 * regulariser energy at the pre-step values.  Errors: FR_EINVAL on bad groups. */
fr_status fr_adam(const fr_opt_group* groups, int32_t n_groups, int32_t step, float beta1, float beta2,
                  float eps, double* reg_energy, void* stream);

/* ---- native continuous-batching server ---- */

/* A reconstruction server owns one context (fully set up: mesh, lights and,
 * when used, albedo model and landmarks) and a worker thread with its own
 * stream.  Requests (a target image, a sample count, the two-stage schedule of
 * Sec. 4 with the optional landmark-only initialisation, initial parameters)
 * are queued by fr_submit from any host thread.  At every step boundary the
 * worker admits waiting requests in arrival order while a slot is free and
 * the device state of the admitted requests stays within the memory cap, then
 * advances every admitted request by one iteration: the Stage I statistical
 * albedos of all of them in one fr_albedo_morph call, one fr_render_batch
 * call, one fr_albedo_adjoint call, the landmark terms, and one fr_adam call
 * over every request's parameter groups (the same groups, learning rates and
 * weights as Sec. 5 gives).  A request's parameters, Adam moments and buffers
 * stay on the device, in one allocation made at admission, until it finishes;
 * its final photometric loss is then evaluated with a fixed Philox iteration
 * (a request whose loss or parameters are not finite, e.g. from NaN initial
 * parameters, ends FAILED), its parameters optionally kept on the host, and
 * its memory freed.  Philox
 * streams are keyed by the request id (the face id) and the request's own
 * iteration, so a request's result does not depend on what it was batched
 * with.  The paper serves nothing; this is the serving form of its method. */
typedef struct fr_server fr_server;

typedef struct fr_server_config {
    int32_t max_slots;        /* requests advanced together, 1..the context's max_batch */
    uint64_t mem_cap_bytes;   /* device bytes the admitted requests' state may hold (the first
                                 request is admitted whatever its size) */
    int32_t n_identity;       /* K_s: coef[0, K_s) are identity (prior), the rest expression
                                 (soft box [0, 1]) */
    int32_t edge_spp;         /* primary-edge samples per pixel of every step (0..64) */
    uint32_t item_flags;      /* FR_FLAG_* bits of every render item (Stage II adds
                                 FR_FLAG_NO_PRIMARY_EDGE | FR_FLAG_NO_SHADOW_EDGE |
                                 FR_FLAG_NO_SPECULAR_EDGE: the geometry is fixed there) */
    uint32_t eval_iteration;  /* Philox iteration of the final loss evaluation */
    int32_t eval_spp;         /* spp of the final loss evaluation (0: the request's own) */
    int32_t keep_params;      /* != 0: copy each finished request's parameters to the host */
} fr_server_config;

/* One request.  Host pointers, copied by fr_submit: target [height][width][3];
 * init holds HOST pointers to the initial parameters with the shapes of
 * fr_params (light_d/light_a/light_p all three or none; with them, and a
 * light stage on the context, Stage I also optimises the light geometry);
 * landmarks [n_landmarks][2] target pixels or NULL (then no E_land and no
 * initialisation stage; n_landmarks must equal the context's). */
typedef struct fr_request {
    int32_t width, height, spp;
    int32_t init_iters, stage1_iters, stage2_iters;
    const float* target;
    fr_params init;
    const float* landmarks;
    int32_t n_landmarks;
} fr_request;

#define FR_REQ_QUEUED  0
#define FR_REQ_RUNNING 1
#define FR_REQ_DONE    2
#define FR_REQ_FAILED  3
#define FR_EAGAIN      6   /* fr_poll: the request has not finished */

typedef struct fr_result {
    int32_t state;            /* FR_REQ_* */
    int32_t iterations;       /* iterations run so far */
    double final_loss;        /* E_ph at the final parameters (DONE) */
    double submit_s, admit_s, finish_s;   /* seconds since fr_server_create (-1: not yet) */
    char error[128];          /* why a request FAILED */
} fr_result;

typedef struct fr_server_stats {
    int64_t steps;            /* batched steps run */
    int64_t item_steps;       /* sum over steps of the admitted requests */
    int32_t max_active;       /* most requests admitted at once */
    int32_t active, queued;   /* now */
    uint64_t peak_bytes;      /* most device state held by admitted requests at once */
    uint64_t used_bytes;      /* device state held by admitted requests now */
    uint64_t finished;        /* requests that reached DONE or FAILED */
} fr_server_stats;

/* Start a server on ctx (which must not be used otherwise until
 * fr_server_destroy; the device current on the calling thread is the one the
 * worker uses).  Errors: FR_EINVAL (context not set up, bad config, a
 * context lit by FR_LIGHT_ENV blocks: requests carry no environment map),
 * FR_ECUDA. */
fr_status fr_server_create(fr_server** out, fr_ctx* ctx, const fr_server_config* cfg);

/* Queue a request; *id receives its id (0, 1, 2, ... in submission order),
 * which is also its Philox face id.  A request the server can never run
 * (image above the context's width * height, spp above the context's, no
 * landmarks set on the context, bad schedule) is queued as FAILED with a
 * reason.  Errors: FR_EINVAL (null pointers). */
fr_status fr_submit(fr_server* srv, const fr_request* req, uint64_t* id);

/* State of request id.  Returns FR_OK once it is DONE or FAILED (and, if
 * params_out is not NULL and the request is DONE with keep_params, copies its
 * final parameters into params_out's HOST buffers, which have the shapes of
 * fr_params; null members are skipped), FR_EAGAIN while it is queued or
 * running, FR_EINVAL for an unknown id. */
fr_status fr_poll(fr_server* srv, uint64_t id, fr_result* out, const fr_grads* params_out);

/* Block until every submitted request is DONE or FAILED, or timeout_s
 * seconds pass (FR_ETIMEOUT). */
fr_status fr_server_wait(fr_server* srv, double timeout_s);

fr_status fr_server_get_stats(fr_server* srv, fr_server_stats* out);

/* Cancel request id: a queued request becomes FAILED ("cancelled") at once; a
 * running one is retired at the next step boundary (its device state freed,
 * no final evaluation) as FAILED ("cancelled").  Other requests are not
 * affected.  Returns FR_OK, or FR_EINVAL for an unknown id or one already
 * DONE or FAILED. */
fr_status fr_cancel(fr_server* srv, uint64_t id);

/* Stop the worker (requests still queued or running are dropped), free every
 * request's device state and the stream.  The context stays the caller's. */
void fr_server_destroy(fr_server* srv);

/* Test hook for the server's error path, with no device fault: the n-th
 * device-to-host read of a result from now (n = 0: the next one; a final loss
 * or a request's final parameters) is treated as failed on the host.  The
 * requests of that step then fail with the read's message; those retired
 * before the failed read keep their results.  FR_EINVAL if n < 0. */
fr_status fr_server_inject_read_failure(fr_server* srv, int32_t n);

/* ---- allocation-free variant ---- */

/* The photometric loss of fr_loss for callers that cannot allocate device
 * memory: a host application that owns the device memory budget through its
 * own pool and forbids libraries to allocate behind it, or a latency-critical
 * loop that cannot absorb an allocation.  The paper has no counterpart; this is
 * an interface convenience.  No context is needed: the caller passes the image
 * size (height * width <= 512 * 512, else FR_EINVAL) and its own buffers, with
 * the same meaning and results as fr_loss.  The only scratch is two static
 * device arrays (3 MiB of residual signs and 8 KiB of partial sums, held by
 * every GPU that loads the library until exit) shared by all calls: calls whose
 * kernels overlap on the GPU race on them.  Every call looks up the arrays'
 * device addresses with the current device; the first call on a device may load
 * the library's module there, so make it before any stream capture.  If a CUDA
 * error from an earlier call is pending, returns FR_ECUDA without launching and
 * leaves that error in place.  Allocates nothing: no cudaMalloc, cudaFree or
 * allocating library routine. */
fr_status fr_loss_noalloc(int32_t height, int32_t width, const float* image, const float* target,
                          double* loss, float* adj_image, float* blurred, void* stream);

/* Message of the last failed fr_loss_noalloc call on this host thread. */
const char* fr_loss_noalloc_error(void);

#ifdef __cplusplus
}
#endif
#endif
