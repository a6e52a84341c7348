/* A plain C client of the C ABI: one fused render (forward + loss + adjoint)
 * of a scene read from raw little-endian files, with device buffers from the
 * CUDA runtime; prints the loss and the coefficient and rotation gradients.
 * Test infrastructure: the GPU tests compare its output with the Python
 * binding's for the same inputs. */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <cuda_runtime.h>
#include "facert.h"

static void* load(const char* dir, const char* name, size_t bytes) {
    char path[4096];
    snprintf(path, sizeof path, "%s/%s", dir, name);
    FILE* f = fopen(path, "rb");
    if (!f) { fprintf(stderr, "cannot open %s\n", path); exit(2); }
    void* p = malloc(bytes ? bytes : 1);
    if (bytes && fread(p, 1, bytes, f) != bytes) { fprintf(stderr, "short read %s\n", path); exit(2); }
    fclose(f);
    return p;
}

static void* dev_copy(const void* h, size_t bytes) {
    void* d = NULL;
    if (cudaMalloc(&d, bytes) != cudaSuccess) { fprintf(stderr, "cudaMalloc failed\n"); exit(3); }
    if (h) cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice);
    else cudaMemset(d, 0, bytes);
    return d;
}

#define CHECK(call)                                                              \
    do {                                                                         \
        fr_status s_ = (call);                                                   \
        if (s_ != FR_OK) {                                                       \
            fprintf(stderr, "%s -> %d: %s\n", #call, (int)s_, fr_last_error(ctx)); \
            return 1;                                                            \
        }                                                                        \
    } while (0)

int main(int argc, char** argv) {
    if (argc < 2) { fprintf(stderr, "usage: render_once DIR\n"); return 2; }
    const char* dir = argv[1];
    int W, H, spp, M, K, N, T, NL, it, face;
    {
        char path[4096];
        snprintf(path, sizeof path, "%s/sizes.txt", dir);
        FILE* f = fopen(path, "r");
        if (!f || fscanf(f, "%d %d %d %d %d %d %d %d %d %d", &W, &H, &spp, &M, &K, &N, &T, &NL, &it, &face) != 10) {
            fprintf(stderr, "bad sizes.txt\n");
            return 2;
        }
        fclose(f);
    }
    const size_t px = (size_t)W * H * 3, tex = (size_t)M * M;
    float* mean = (float*)load(dir, "mean.bin", sizeof(float) * 3 * N);
    float* basis = (float*)load(dir, "basis.bin", sizeof(float) * 3 * (size_t)N * K);
    int32_t* faces = (int32_t*)load(dir, "faces.bin", sizeof(int32_t) * 3 * T);
    float* uv = (float*)load(dir, "uv.bin", sizeof(float) * 2 * N);
    float* rec = (float*)load(dir, "lights.bin", sizeof(float) * 11 * NL);
    float* ld = (float*)load(dir, "light_d.bin", sizeof(float) * NL);
    float* la = (float*)load(dir, "light_a.bin", sizeof(float) * NL);

    fr_ctx* ctx = NULL;
    fr_config cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.width = W; cfg.height = H; cfg.spp = spp; cfg.tex_size = M; cfg.edge_spp = 1; cfg.max_batch = 1;
    CHECK(fr_create(&ctx, &cfg));
    fr_mesh mesh = {N, T, K, mean, basis, faces, uv};
    CHECK(fr_set_mesh(ctx, &mesh));
    fr_light_stage ls;
    memset(&ls, 0, sizeof ls);
    ls.n_lights = NL; ls.records = rec; ls.d = ld; ls.a = la;
    CHECK(fr_set_lights(ctx, &ls));

    const size_t sizes[8] = {(size_t)K, 3, 3, 1, 3 * (size_t)NL, 3 * tex, 3 * tex, tex};
    const char* names[8] = {"coef.bin", "rot.bin", "trans.bin", "focal.bin", "light_i.bin", "diffuse.bin",
                            "specular.bin", "roughness.bin"};
    float* pd[8];
    float* gd[8];
    for (int k = 0; k < 8; ++k) {
        float* h = (float*)load(dir, names[k], sizeof(float) * sizes[k]);
        pd[k] = (float*)dev_copy(h, sizeof(float) * sizes[k]);
        gd[k] = (float*)dev_copy(NULL, sizeof(float) * sizes[k]);
        free(h);
    }
    fr_params p;
    fr_grads g;
    memset(&p, 0, sizeof p);
    memset(&g, 0, sizeof g);
    p.coef = pd[0]; p.rot = pd[1]; p.trans = pd[2]; p.focal = pd[3];
    p.light_i = pd[4]; p.diffuse = pd[5]; p.specular = pd[6]; p.roughness = pd[7];
    g.coef = gd[0]; g.rot = gd[1]; g.trans = gd[2]; g.focal = gd[3];
    g.light_i = gd[4]; g.diffuse = gd[5]; g.specular = gd[6]; g.roughness = gd[7];
    float* target_h = (float*)load(dir, "target.bin", sizeof(float) * px);
    float* target = (float*)dev_copy(target_h, sizeof(float) * px);
    float* image = (float*)dev_copy(NULL, sizeof(float) * px);
    double* loss = (double*)dev_copy(NULL, sizeof(double));

    CHECK(fr_render(ctx, &p, target, image, loss, &g, (uint32_t)it, (uint32_t)face, NULL));
    CHECK(fr_sync_status(ctx, NULL));
    double loss_h = 0.0;
    cudaMemcpy(&loss_h, loss, sizeof(double), cudaMemcpyDeviceToHost);
    printf("loss %.17g\n", loss_h);
    float* gc = (float*)malloc(sizeof(float) * (K + 3));
    cudaMemcpy(gc, gd[0], sizeof(float) * K, cudaMemcpyDeviceToHost);
    cudaMemcpy(gc + K, gd[1], sizeof(float) * 3, cudaMemcpyDeviceToHost);
    for (int k = 0; k < K; ++k) printf("coef %d %.9g\n", k, gc[k]);
    for (int k = 0; k < 3; ++k) printf("rot %d %.9g\n", k, gc[K + k]);
    fr_destroy(ctx);
    return 0;
}
