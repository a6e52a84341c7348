// Native continuous-batching reconstruction server: the two-stage
// reconstruction of Sec. 4 (landmark-only initialisation, Stage I with
// E_ph + alpha_1 E_land + priors + soft boxes, Stage II with the texture
// regularisers of Eq. loss3) run for many requests at once on one context.
//
// A worker thread owns the context and a stream.  Each step it admits queued
// requests (FIFO) while a slot is free and the admitted requests' device state
// fits under the memory cap, advances every admitted request by one iteration
// with one call per stage of the path over all of them (statistical albedo
// morph, fr_render_batch, albedo transpose, landmark terms, one fr_adam over
// every request's groups), then evaluates and retires the requests that are
// done.  Every request's device state (parameters, gradients, Adam moments,
// target, image, Stage II references, landmarks) is one allocation made at
// admission and freed at retirement.
//
// The optimiser groups, learning rates and weights are those of Sec. 5 with
// the same readings as the Python reconstruction (shape prior squared,
// quadratic soft boxes, roughness kept in [0.02, 1.5], light geometry kept
// >= 1e-3); Philox streams are keyed by the request id and its own
// iteration, so a request's result does not depend on its batch.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/facert.h"
#include "kernels.h"

namespace {

// Sec. 5: learning rates per group and regulariser weights.
constexpr float LR_LIGHT = 1e-3f, LR_IDENTITY = 1e-2f, LR_EXPRESSION = 1e-3f, LR_ROT = 1e-3f, LR_TRANS = 1e-3f;
constexpr float LR_TEXTURE = 5e-3f, LR_ALBEDO = 2e-2f;
constexpr float W_I = 0.0025f, W_C = 0.0025f, W_S = 0.0025f, W1 = 0.01f, W2 = 0.3f, W3 = 0.3f, W4 = 0.0002f;
constexpr float W_BOX = 1.0f;
constexpr float ALPHA1 = 1.0f;                          // weight of E_land in E_d
constexpr float ROUGH_LO = 0.02f, ROUGH_HI = 1.5f;      // roughness range after each step (keeps D finite)
constexpr float STAGE_LO = 1e-3f, STAGE_HI = 1e3f;      // floor of d, a, p after each step (keeps d^2/a finite)
constexpr uint32_t STAGE2_FLAGS = FR_FLAG_NO_PRIMARY_EDGE | FR_FLAG_NO_SHADOW_EDGE | FR_FLAG_NO_SPECULAR_EDGE;
constexpr float ADAM_B1 = 0.9f, ADAM_B2 = 0.999f, ADAM_EPS = 1e-8f;

// Parameter segments of a request's parameter vector (and of its gradient and
// moments): the fr_params groups, the light geometry as one [d | a | p] block.
enum { P_COEF, P_ROT, P_TRANS, P_FOCAL, P_LIGHT, P_DIFFUSE, P_SPECULAR, P_ROUGH, P_STAGE, P_COUNT };
constexpr size_t ALIGN_FLOATS = 64;                     // 256-byte segment alignment

size_t up(size_t n) { return (n + ALIGN_FLOATS - 1) / ALIGN_FLOATS * ALIGN_FLOATS; }
bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

struct Request {
    uint64_t id = 0;
    int W = 0, H = 0, spp = 0, n_init = 0, s1 = 0, s2 = 0;
    bool stage_geo = false, landmarks = false;
    std::vector<float> target, lm, init[P_COUNT];
    // progress (read by fr_poll under the server mutex)
    int state = FR_REQ_QUEUED, it = 0;
    double t_submit = -1.0, t_admit = -1.0, t_finish = -1.0, final_loss = 0.0;
    std::string err;
    std::vector<float> out;                             // final parameter vector (keep_params)
    // device state
    char* block = nullptr;
    size_t bytes = 0;
    size_t off[P_COUNT] = {}, seg[P_COUNT] = {}, n_par = 0;
    float *x = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
    float* ab[2][4] = {};                               // beta, gamma: x, g, m, v
    float *d_target = nullptr, *image = nullptr, *ref_d = nullptr, *ref_s = nullptr, *d_lm = nullptr;
    double *loss = nullptr, *land_loss = nullptr;
    bool refs_taken = false;
    bool cancel = false;                                // set by fr_cancel while running

    int stage() const { return it < n_init ? 0 : (it < n_init + s1 ? 1 : 2); }
    bool done() const { return it >= n_init + s1 + s2; }
    float* X(int k) const { return x + off[k]; }
    float* G(int k) const { return g + off[k]; }
    float* M(int k) const { return m + off[k]; }
    float* V(int k) const { return v + off[k]; }
};

double now_s(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct fr_server {
    fr_ctx* ctx = nullptr;
    fr_server_config cfg{};
    CtxInfo info;
    int device = 0;
    cudaStream_t stream = nullptr;
    float* light_da = nullptr;                          // [d (N_L) | a (N_L)] of the lights (device, shared)
    std::chrono::steady_clock::time_point t0;

    std::mutex mu;
    std::condition_variable wake, idle;
    std::deque<Request*> queue;
    std::vector<std::unique_ptr<Request>> all;          // by id
    std::vector<Request*> active;                       // worker only
    size_t used = 0;
    uint64_t finished = 0;
    bool stop = false;
    std::atomic<int> inject_read_fail{-1};              // test hook: fail the n-th result read from now
    fr_server_stats stats{};
    std::thread worker;

    size_t seg_size(int k, bool stage_geo) const {
        const size_t M2 = (size_t)info.tex * info.tex;
        switch (k) {
        case P_COEF: return info.K;
        case P_ROT: case P_TRANS: return 3;
        case P_FOCAL: return 1;
        case P_LIGHT: return 3 * (size_t)info.NL;
        case P_DIFFUSE: case P_SPECULAR: return 3 * M2;
        case P_ROUGH: return M2;
        default: return stage_geo ? 4 * (size_t)info.NL : 0;
        }
    }

    // Lay out a request's device state and return its size in bytes.
    size_t layout(Request& r) const {
        size_t n = 0;
        for (int k = 0; k < P_COUNT; ++k) {
            r.seg[k] = seg_size(k, r.stage_geo);
            r.off[k] = n;
            n += up(r.seg[k]);
        }
        r.n_par = n;
        size_t floats = 4 * n;                                       // x, g, m, v
        const int kab[2] = {info.k_diffuse, info.k_specular};
        if (info.have_albedo)
            for (int q = 0; q < 2; ++q) floats += 4 * up(std::max(kab[q], 1));
        const size_t M2 = (size_t)info.tex * info.tex;
        floats += 2 * up(3 * (size_t)r.W * r.H) + 2 * up(3 * M2) + up(2 * (size_t)std::max(info.n_landmarks, 1));
        return floats * sizeof(float) + 2 * 256;                     // + the two loss doubles
    }

    fr_params params(const Request& r) const {
        fr_params p{};
        p.coef = r.X(P_COEF); p.rot = r.X(P_ROT); p.trans = r.X(P_TRANS); p.focal = r.X(P_FOCAL);
        p.light_i = r.X(P_LIGHT); p.diffuse = r.X(P_DIFFUSE); p.specular = r.X(P_SPECULAR); p.roughness = r.X(P_ROUGH);
        if (r.stage_geo) {
            p.light_d = r.X(P_STAGE);
            p.light_a = r.X(P_STAGE) + info.NL;
            p.light_p = r.X(P_STAGE) + 2 * info.NL;
        }
        return p;
    }

    fr_grads grads(const Request& r) const {
        fr_grads g{};
        g.coef = r.G(P_COEF); g.rot = r.G(P_ROT); g.trans = r.G(P_TRANS); g.focal = r.G(P_FOCAL);
        g.light_i = r.G(P_LIGHT); g.diffuse = r.G(P_DIFFUSE); g.specular = r.G(P_SPECULAR); g.roughness = r.G(P_ROUGH);
        if (r.stage_geo) {
            g.light_d = r.G(P_STAGE);
            g.light_a = r.G(P_STAGE) + info.NL;
            g.light_p = r.G(P_STAGE) + 2 * info.NL;
        }
        return g;
    }

    // Allocate and initialise a request's device state (worker thread).
    bool admit_one(Request& r) {
        r.bytes = layout(r);
        void* p = nullptr;
        if (cudaMalloc(&p, r.bytes) != cudaSuccess) {
            cudaGetLastError();
            r.err = "device allocation of the request's state failed";
            return false;
        }
        r.block = static_cast<char*>(p);
        float* f = reinterpret_cast<float*>(r.block + 2 * 256);
        r.loss = reinterpret_cast<double*>(r.block);
        r.land_loss = reinterpret_cast<double*>(r.block + 256);
        r.x = f; f += r.n_par;
        r.g = f; f += r.n_par;
        r.m = f; f += r.n_par;
        r.v = f; f += r.n_par;
        const int kab[2] = {info.k_diffuse, info.k_specular};
        if (info.have_albedo)
            for (int q = 0; q < 2; ++q)
                for (int t = 0; t < 4; ++t) { r.ab[q][t] = f; f += up(std::max(kab[q], 1)); }
        const size_t M2 = (size_t)info.tex * info.tex;
        r.d_target = f; f += up(3 * (size_t)r.W * r.H);
        r.image = f; f += up(3 * (size_t)r.W * r.H);
        r.ref_d = f; f += up(3 * M2);
        r.ref_s = f; f += up(3 * M2);
        r.d_lm = f;
        // zero everything (moments, gradients, albedo coefficients = the mean albedo), then the inputs
        bool ok = cudaMemsetAsync(r.block, 0, r.bytes, stream) == cudaSuccess;
        for (int k = 0; k < P_COUNT && ok; ++k)
            if (r.seg[k]) ok = cudaMemcpyAsync(r.X(k), r.init[k].data(), sizeof(float) * r.seg[k],
                                               cudaMemcpyHostToDevice, stream) == cudaSuccess;
        if (ok) ok = cudaMemcpyAsync(r.d_target, r.target.data(), sizeof(float) * r.target.size(),
                                     cudaMemcpyHostToDevice, stream) == cudaSuccess;
        if (ok && r.landmarks)
            ok = cudaMemcpyAsync(r.d_lm, r.lm.data(), sizeof(float) * r.lm.size(), cudaMemcpyHostToDevice,
                                 stream) == cudaSuccess;
        if (ok) ok = cudaStreamSynchronize(stream) == cudaSuccess;   // host staging buffers are released next
        if (!ok) {
            cudaGetLastError();
            r.err = "copying the request's inputs to the device failed";
            cudaFree(r.block);
            r.block = nullptr;
            return false;
        }
        r.target.clear(); r.target.shrink_to_fit();
        for (auto& a : r.init) { a.clear(); a.shrink_to_fit(); }
        return true;
    }

    void release(Request& r) {
        if (r.block) cudaFree(r.block);
        r.block = nullptr;
    }

    fr_opt_group group(float* x, float* g, float* m, float* v, int n, int kind, float lr, int step) const {
        fr_opt_group o{};
        o.x = x; o.g = g; o.m = m; o.v = v;
        o.n = n; o.kind = kind; o.lr = lr; o.step = step;
        return o;
    }

    // Adam + regulariser groups of the request's current stage (Sec. 4, 5).
    void groups(const Request& r, std::vector<fr_opt_group>& out) const {
        const int ks = cfg.n_identity, K = info.K, st = r.stage();
        auto expression = [&](int step) {
            if (K > ks) {
                fr_opt_group o = group(r.X(P_COEF) + ks, r.G(P_COEF) + ks, r.M(P_COEF) + ks, r.V(P_COEF) + ks, K - ks,
                                       FR_GROUP_COEF, LR_EXPRESSION, step);
                o.w_box = W_BOX;
                out.push_back(o);
            }
        };
        if (st == 0) {
            const int step = r.it + 1;
            out.push_back(group(r.X(P_ROT), r.G(P_ROT), r.M(P_ROT), r.V(P_ROT), 3, FR_GROUP_PLAIN, LR_ROT, step));
            out.push_back(group(r.X(P_TRANS), r.G(P_TRANS), r.M(P_TRANS), r.V(P_TRANS), 3, FR_GROUP_PLAIN, LR_TRANS, step));
            expression(step);
            return;
        }
        if (st == 1) {
            const int step = r.it - r.n_init + 1;
            if (ks > 0) {
                fr_opt_group o = group(r.X(P_COEF), r.G(P_COEF), r.M(P_COEF), r.V(P_COEF), ks, FR_GROUP_COEF,
                                       LR_IDENTITY, step);
                o.n_prior = ks;
                o.w_prior = W_I;
                out.push_back(o);
            }
            expression(step);
            out.push_back(group(r.X(P_ROT), r.G(P_ROT), r.M(P_ROT), r.V(P_ROT), 3, FR_GROUP_PLAIN, LR_ROT, step));
            out.push_back(group(r.X(P_TRANS), r.G(P_TRANS), r.M(P_TRANS), r.V(P_TRANS), 3, FR_GROUP_PLAIN, LR_TRANS, step));
            fr_opt_group li = group(r.X(P_LIGHT), r.G(P_LIGHT), r.M(P_LIGHT), r.V(P_LIGHT), 3 * info.NL, FR_GROUP_LIGHT,
                                    LR_LIGHT, step);
            li.w_prior = W1;
            li.w_box = W_BOX;
            li.aux2 = r.stage_geo ? r.X(P_STAGE) : light_da;     // the kernel forms d^2 / a
            out.push_back(li);
            if (r.stage_geo) {
                fr_opt_group o = group(r.X(P_STAGE), r.G(P_STAGE), r.M(P_STAGE), r.V(P_STAGE), 4 * info.NL,
                                       FR_GROUP_STAGE, LR_LIGHT, step);
                o.aux = r.X(P_LIGHT);
                o.w_prior = W1;
                o.w_box = W_BOX;
                o.clamp_lo = STAGE_LO;
                o.clamp_hi = STAGE_HI;
                out.push_back(o);
            }
            if (info.have_albedo) {
                const int kab[2] = {info.k_diffuse, info.k_specular};
                const float w[2] = {W_C, W_S};
                for (int q = 0; q < 2; ++q) {
                    if (kab[q] <= 0) continue;
                    fr_opt_group o = group(r.ab[q][0], r.ab[q][1], r.ab[q][2], r.ab[q][3], kab[q], FR_GROUP_COEF,
                                           LR_ALBEDO, step);
                    o.n_prior = kab[q];
                    o.w_prior = w[q];
                    out.push_back(o);
                }
            }
            return;
        }
        const int step = r.it - r.n_init - r.s1 + 1;
        const int M = info.tex;
        fr_opt_group d = group(r.X(P_DIFFUSE), r.G(P_DIFFUSE), r.M(P_DIFFUSE), r.V(P_DIFFUSE), 3 * M * M,
                               FR_GROUP_TEX_RGB, LR_TEXTURE, step);
        d.aux = r.ref_d; d.width = M; d.w_sym = W2; d.w_chroma = W3; d.w_smooth = W4;
        out.push_back(d);
        fr_opt_group s = group(r.X(P_SPECULAR), r.G(P_SPECULAR), r.M(P_SPECULAR), r.V(P_SPECULAR), 3 * M * M,
                               FR_GROUP_TEX_RGB, LR_TEXTURE, step);
        s.aux = r.ref_s; s.width = M; s.w_sym = W2; s.w_chroma = W3; s.w_smooth = W4; s.w_box = W_BOX;
        out.push_back(s);
        fr_opt_group o = group(r.X(P_ROUGH), r.G(P_ROUGH), r.M(P_ROUGH), r.V(P_ROUGH), M * M, FR_GROUP_TEX_MONO,
                               LR_TEXTURE, step);
        o.width = M; o.w_smooth = W4; o.w_box = W_BOX; o.clamp_lo = ROUGH_LO; o.clamp_hi = ROUGH_HI;
        out.push_back(o);
    }

    fr_item item(Request& r, fr_grads* g, uint32_t iteration, int spp, uint32_t flags) const {
        fr_item it{};
        it.width = r.W; it.height = r.H; it.spp = spp; it.edge_spp = cfg.edge_spp;
        it.flags = flags; it.iteration = iteration; it.face_id = (uint32_t)r.id;
        it.params = params(r);
        it.target = r.d_target; it.image = r.image; it.loss = r.loss; it.grads = g;
        return it;
    }

    // Start of a request's iteration: zero its gradients, restart the pose
    // and coefficient moments when Stage I follows the landmark
    // initialisation, take the Stage II albedo references.
    bool begin_step(Request& r) {
        bool ok = true;
        if (r.stage() == 1 && r.it == r.n_init && r.n_init > 0)
            for (int k : {P_ROT, P_TRANS, P_COEF}) {
                ok = ok && cudaMemsetAsync(r.M(k), 0, sizeof(float) * r.seg[k], stream) == cudaSuccess;
                ok = ok && cudaMemsetAsync(r.V(k), 0, sizeof(float) * r.seg[k], stream) == cudaSuccess;
            }
        if (r.stage() == 2 && !r.refs_taken) {
            const size_t n = sizeof(float) * r.seg[P_DIFFUSE];
            ok = ok && cudaMemcpyAsync(r.ref_d, r.X(P_DIFFUSE), n, cudaMemcpyDeviceToDevice, stream) == cudaSuccess;
            ok = ok && cudaMemcpyAsync(r.ref_s, r.X(P_SPECULAR), n, cudaMemcpyDeviceToDevice, stream) == cudaSuccess;
            r.refs_taken = true;
        }
        ok = ok && cudaMemsetAsync(r.g, 0, sizeof(float) * r.n_par, stream) == cudaSuccess;
        if (info.have_albedo)
            for (int q = 0; q < 2; ++q)
                ok = ok && cudaMemsetAsync(r.ab[q][1], 0, sizeof(float) * std::max(q ? info.k_specular : info.k_diffuse, 1),
                                           stream) == cudaSuccess;
        return ok;
    }

    // One iteration of every admitted request.  Returns "" or what failed.
    std::string step() {
        std::vector<Request*> run;                      // requests with iterations left
        {
            std::lock_guard<std::mutex> lk(mu);
            for (Request* r : active)
                if (!r->done() && !r->cancel) run.push_back(r);
        }
        for (Request* r : run)
            if (!begin_step(*r)) return "enqueueing the start of a step failed";
        std::vector<Request*> rend, stat;
        for (Request* r : run)
            if (r->stage() > 0) {
                rend.push_back(r);
                if (r->stage() == 1 && info.have_albedo) stat.push_back(r);
            }
        void* st = static_cast<void*>(stream);
        if (!stat.empty()) {
            std::vector<const float*> b, c;
            std::vector<float*> dif, spe;
            for (Request* r : stat) {
                b.push_back(r->ab[0][0]); c.push_back(r->ab[1][0]);
                dif.push_back(r->X(P_DIFFUSE)); spe.push_back(r->X(P_SPECULAR));
            }
            if (fr_albedo_morph(ctx, (int)stat.size(), b.data(), c.data(), dif.data(), spe.data(), st) != FR_OK)
                return std::string("albedo morph: ") + fr_last_error(ctx);
        }
        if (!rend.empty()) {
            std::vector<fr_grads> gs(rend.size());
            std::vector<fr_item> items;
            for (size_t k = 0; k < rend.size(); ++k) {
                Request& r = *rend[k];
                gs[k] = grads(r);
                items.push_back(item(r, &gs[k], (uint32_t)r.it, r.spp,
                                     cfg.item_flags | (r.stage() == 2 ? STAGE2_FLAGS : 0u)));
            }
            if (fr_render_batch(ctx, items.data(), (int)items.size(), st) != FR_OK)
                return std::string("render: ") + fr_last_error(ctx);
        }
        if (!stat.empty()) {
            std::vector<const float*> gd, gsp;
            std::vector<float*> gb, gc;
            for (Request* r : stat) {
                gd.push_back(r->G(P_DIFFUSE)); gsp.push_back(r->G(P_SPECULAR));
                gb.push_back(r->ab[0][1]); gc.push_back(r->ab[1][1]);
            }
            if (fr_albedo_adjoint(ctx, (int)stat.size(), gd.data(), gsp.data(), gb.data(), gc.data(), st) != FR_OK)
                return std::string("albedo adjoint: ") + fr_last_error(ctx);
        }
        for (Request* r : run)
            if (r->landmarks && r->stage() <= 1) {
                const fr_params p = params(*r);
                fr_grads g = grads(*r);
                if (fr_landmark_loss(ctx, &p, r->W, r->H, r->d_lm, ALPHA1, r->land_loss, &g, nullptr, st) != FR_OK)
                    return std::string("landmark loss: ") + fr_last_error(ctx);
            }
        std::vector<fr_opt_group> gr;
        for (Request* r : run) groups(*r, gr);
        for (size_t k = 0; k < gr.size(); k += FR_MAX_OPT_GROUPS) {
            const int n = (int)std::min<size_t>(FR_MAX_OPT_GROUPS, gr.size() - k);
            if (fr_adam(gr.data() + k, n, 1, ADAM_B1, ADAM_B2, ADAM_EPS, nullptr, st) != FR_OK)
                return "optimiser step rejected its groups";
        }
        const fr_status s = fr_sync_status(ctx, st);
        if (s != FR_OK) return std::string("device status after a step: ") + fr_last_error(ctx);
        std::lock_guard<std::mutex> lk(mu);
        for (Request* r : run) r->it++;
        if (!run.empty()) {
            stats.steps++;
            stats.item_steps += (int64_t)run.size();
        }
        return "";
    }

    // Final loss of the finished requests (one batched forward), results, release.
    std::string retire() {
        std::vector<Request*> fin, cancelled;
        {
            std::lock_guard<std::mutex> lk(mu);
            for (Request* r : active) {
                if (r->cancel) cancelled.push_back(r);
                else if (r->done()) fin.push_back(r);
            }
        }
        // cancelled requests leave at the step boundary without an evaluation
        for (Request* r : cancelled) {
            release(*r);
            std::lock_guard<std::mutex> lk(mu);
            r->state = FR_REQ_FAILED;
            r->err = "cancelled";
            r->t_finish = now_s(t0);
            used -= r->bytes;
            finished++;
        }
        if (!cancelled.empty()) {
            active.erase(std::remove_if(active.begin(), active.end(),
                                        [](Request* r) { return r->state == FR_REQ_FAILED; }),
                         active.end());
            idle.notify_all();
        }
        if (fin.empty()) return "";
        std::vector<fr_item> items;
        for (Request* r : fin)
            items.push_back(item(*r, nullptr, cfg.eval_iteration, cfg.eval_spp > 0 ? cfg.eval_spp : r->spp,
                                 cfg.item_flags | STAGE2_FLAGS));
        void* st = static_cast<void*>(stream);
        if (fr_render_batch(ctx, items.data(), (int)items.size(), st) != FR_OK)
            return std::string("final evaluation: ") + fr_last_error(ctx);
        if (fr_sync_status(ctx, st) != FR_OK) return std::string("device status after evaluation: ") + fr_last_error(ctx);
        // a failed read stops the loop; the requests retired before it leave
        // `active` here, so the caller's fail_active handles only the others
        std::string err;
        for (Request* r : fin) {
            double loss = 0.0;
            if (!read_back(&loss, r->loss, sizeof(double))) {
                err = "reading a final loss failed";
                break;
            }
            // the final parameters are read back to check them (and kept if asked)
            std::vector<float> keep(r->n_par);
            if (!read_back(keep.data(), r->x, sizeof(float) * r->n_par)) {
                err = "reading final parameters failed";
                break;
            }
            bool finite = std::isfinite(loss);
            for (size_t i = 0; finite && i < keep.size(); ++i) finite = std::isfinite(keep[i]);
            if (!cfg.keep_params || !finite) keep.clear();
            release(*r);
            std::lock_guard<std::mutex> lk(mu);
            r->final_loss = loss;
            r->out.swap(keep);
            if (finite) {
                r->state = FR_REQ_DONE;
            } else {
                r->state = FR_REQ_FAILED;
                r->err = "the final loss or parameters are not finite";
            }
            r->t_finish = now_s(t0);
            used -= r->bytes;
            finished++;
        }
        active.erase(std::remove_if(active.begin(), active.end(),
                                    [](Request* r) { return r->state == FR_REQ_DONE || r->state == FR_REQ_FAILED; }),
                     active.end());
        idle.notify_all();
        return err;
    }

    // Device-to-host read of a result.  A test can make the n-th read from now
    // fail on the host (fr_server_inject_read_failure) to exercise the error
    // path without a device fault.
    bool read_back(void* dst, const void* src, size_t bytes) {
        int n = inject_read_fail.load();
        while (n >= 0 && !inject_read_fail.compare_exchange_weak(n, n - 1)) {
        }
        if (n == 0) return false;
        return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    }

    void fail_active(const std::string& why) {
        for (Request* r : active) release(*r);
        std::lock_guard<std::mutex> lk(mu);
        for (Request* r : active) {
            if (r->state == FR_REQ_DONE || r->state == FR_REQ_FAILED) continue;   // already accounted for
            r->state = FR_REQ_FAILED;
            r->err = why;
            r->t_finish = now_s(t0);
            used -= r->bytes;
            finished++;
        }
        active.clear();
        idle.notify_all();
    }

    void run() {
        cudaSetDevice(device);
        for (;;) {
            std::vector<Request*> admit;
            {
                std::unique_lock<std::mutex> lk(mu);
                wake.wait(lk, [&] { return stop || !queue.empty() || !active.empty(); });
                if (stop) return;
                // FIFO admission by slots and memory (the head waits for memory to free up)
                size_t planned = used;
                while (!queue.empty() && active.size() + admit.size() < (size_t)cfg.max_slots) {
                    Request* r = queue.front();
                    const size_t b = layout(*r);
                    if (!(active.empty() && admit.empty()) && planned + b > cfg.mem_cap_bytes) break;
                    queue.pop_front();
                    r->state = FR_REQ_RUNNING;          // from here fr_cancel flags it instead
                    planned += b;
                    admit.push_back(r);
                }
            }
            for (Request* r : admit) {
                const bool ok = admit_one(*r);
                std::lock_guard<std::mutex> lk(mu);
                if (ok) {
                    r->t_admit = now_s(t0);
                    used += r->bytes;
                    stats.peak_bytes = std::max<uint64_t>(stats.peak_bytes, used);
                    active.push_back(r);
                } else {
                    r->state = FR_REQ_FAILED;
                    r->t_finish = now_s(t0);
                    finished++;
                    idle.notify_all();
                }
            }
            {
                std::lock_guard<std::mutex> lk(mu);
                stats.max_active = std::max<int32_t>(stats.max_active, (int32_t)active.size());
            }
            if (active.empty()) continue;
            std::string e = step();
            if (e.empty()) e = retire();
            if (!e.empty()) fail_active(e);
        }
    }
};

extern "C" {

fr_status fr_server_create(fr_server** out, fr_ctx* ctx, const fr_server_config* cfg) {
    if (!out || !ctx || !cfg) return FR_EINVAL;
    *out = nullptr;
    std::unique_ptr<fr_server> s(new fr_server());
    s->ctx = ctx;
    s->cfg = *cfg;
    ctx_info(ctx, s->info);
    const CtxInfo& I = s->info;
    if (!I.ready) return FR_EINVAL;
    if (I.env_size > 0) return FR_EINVAL;          // requests carry no environment map
    if (cfg->max_slots < 1 || cfg->max_slots > I.max_batch) return FR_EINVAL;
    if (cfg->n_identity < 0 || cfg->n_identity > I.K) return FR_EINVAL;
    if (cfg->edge_spp < 0 || cfg->edge_spp > 64) return FR_EINVAL;
    if (cfg->eval_spp != 0 && (!pow2(cfg->eval_spp) || cfg->eval_spp > I.spp)) return FR_EINVAL;
    if (cudaGetDevice(&s->device) != cudaSuccess) return FR_ECUDA;
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return FR_ECUDA;
    if (cudaMalloc(&s->light_da, sizeof(float) * std::max(2 * I.NL, 1)) != cudaSuccess ||
        cudaMemcpy(s->light_da, I.light_da.data(), sizeof(float) * 2 * I.NL, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        if (s->light_da) cudaFree(s->light_da);
        cudaStreamDestroy(s->stream);
        return FR_ECUDA;
    }
    s->t0 = std::chrono::steady_clock::now();
    fr_server* raw = s.get();
    s->worker = std::thread([raw] { raw->run(); });
    *out = s.release();
    return FR_OK;
}

fr_status fr_submit(fr_server* s, const fr_request* q, uint64_t* id) {
    if (!s || !q || !id || !q->target) return FR_EINVAL;
    const fr_params& P = q->init;
    if (!P.coef || !P.rot || !P.trans || !P.focal || !P.light_i || !P.diffuse || !P.specular || !P.roughness)
        return FR_EINVAL;
    const CtxInfo& I = s->info;
    std::unique_ptr<Request> r(new Request());
    r->W = q->width; r->H = q->height; r->spp = q->spp;
    r->s1 = q->stage1_iters; r->s2 = q->stage2_iters;
    r->landmarks = q->landmarks != nullptr;
    r->n_init = r->landmarks ? q->init_iters : 0;
    const int geo = (P.light_d != nullptr) + (P.light_a != nullptr) + (P.light_p != nullptr);
    r->stage_geo = geo == 3;
    if (r->W < 1 || r->H < 1 || (long)r->W * r->H > (long)I.width * I.height)
        r->err = "image larger than the server's context";
    else if (!pow2(r->spp) || r->spp > I.spp)
        r->err = "spp must be a power of two no larger than the context's";
    else if (q->init_iters < 0 || q->stage1_iters < 0 || q->stage2_iters < 0)
        r->err = "negative iteration count";
    else if (geo != 0 && geo != 3)
        r->err = "light_d, light_a and light_p must be given together";
    else if (r->stage_geo && !I.have_stage)
        r->err = "light geometry given but the context has no light stage";
    else if (r->landmarks && (I.n_landmarks < 1 || q->n_landmarks != I.n_landmarks))
        r->err = "landmark count does not match the context's landmark vertices";
    if (r->err.empty()) {
        r->target.assign(q->target, q->target + 3 * (size_t)r->W * r->H);
        if (r->landmarks) r->lm.assign(q->landmarks, q->landmarks + 2 * (size_t)I.n_landmarks);
        const float* src[P_COUNT] = {P.coef, P.rot, P.trans, P.focal, P.light_i, P.diffuse, P.specular, P.roughness,
                                     nullptr};
        for (int k = 0; k < P_STAGE; ++k) r->init[k].assign(src[k], src[k] + s->seg_size(k, false));
        if (r->stage_geo) {
            std::vector<float>& a = r->init[P_STAGE];
            a.assign(P.light_d, P.light_d + I.NL);
            a.insert(a.end(), P.light_a, P.light_a + I.NL);
            a.insert(a.end(), P.light_p, P.light_p + 2 * I.NL);
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->all.size();
    r->t_submit = now_s(s->t0);
    *id = r->id;
    Request* raw = r.get();
    s->all.push_back(std::move(r));
    if (!raw->err.empty()) {
        raw->state = FR_REQ_FAILED;
        raw->t_finish = raw->t_submit;
        s->finished++;
        s->idle.notify_all();
    } else {
        s->queue.push_back(raw);
        s->wake.notify_one();
    }
    return FR_OK;
}

fr_status fr_poll(fr_server* s, uint64_t id, fr_result* out, const fr_grads* params_out) {
    if (!s || !out) return FR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= s->all.size()) return FR_EINVAL;
    const Request& r = *s->all[id];
    std::memset(out, 0, sizeof(*out));
    out->state = r.state;
    out->iterations = r.it;
    out->final_loss = r.final_loss;
    out->submit_s = r.t_submit;
    out->admit_s = r.t_admit;
    out->finish_s = r.t_finish;
    std::snprintf(out->error, sizeof(out->error), "%s", r.err.c_str());
    if (r.state != FR_REQ_DONE && r.state != FR_REQ_FAILED) return FR_EAGAIN;
    if (params_out && r.state == FR_REQ_DONE && !r.out.empty()) {
        const CtxInfo& I = s->info;
        float* dst[P_COUNT] = {params_out->coef, params_out->rot, params_out->trans, params_out->focal,
                               params_out->light_i, params_out->diffuse, params_out->specular, params_out->roughness,
                               nullptr};
        for (int k = 0; k < P_STAGE; ++k)
            if (dst[k]) std::memcpy(dst[k], r.out.data() + r.off[k], sizeof(float) * r.seg[k]);
        if (r.stage_geo) {
            const float* g = r.out.data() + r.off[P_STAGE];
            if (params_out->light_d) std::memcpy(params_out->light_d, g, sizeof(float) * I.NL);
            if (params_out->light_a) std::memcpy(params_out->light_a, g + I.NL, sizeof(float) * I.NL);
            if (params_out->light_p) std::memcpy(params_out->light_p, g + 2 * I.NL, sizeof(float) * 2 * I.NL);
        }
    }
    return FR_OK;
}

fr_status fr_cancel(fr_server* s, uint64_t id) {
    if (!s) return FR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (id >= s->all.size()) return FR_EINVAL;
    Request* r = s->all[id].get();
    if (r->state == FR_REQ_DONE || r->state == FR_REQ_FAILED) return FR_EINVAL;
    if (r->state == FR_REQ_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
        r->state = FR_REQ_FAILED;
        r->err = "cancelled";
        r->t_finish = now_s(s->t0);
        s->finished++;
        s->idle.notify_all();
    } else {
        r->cancel = true;                              // the worker retires it at the next step boundary
    }
    return FR_OK;
}

fr_status fr_server_wait(fr_server* s, double timeout_s) {
    if (!s) return FR_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->idle.wait_for(lk, std::chrono::duration<double>(std::max(timeout_s, 0.0)),
                                     [&] { return s->finished == s->all.size(); });
    return ok ? FR_OK : FR_ETIMEOUT;
}

fr_status fr_server_inject_read_failure(fr_server* s, int32_t n) {
    if (!s || n < 0) return FR_EINVAL;
    s->inject_read_fail.store(n);
    return FR_OK;
}

fr_status fr_server_get_stats(fr_server* s, fr_server_stats* out) {
    if (!s || !out) return FR_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->queued = (int32_t)s->queue.size();
    int32_t running = 0;
    for (const auto& r : s->all) running += r->state == FR_REQ_RUNNING;
    out->active = running;
    out->used_bytes = s->used;
    out->finished = s->finished;
    return FR_OK;
}

void fr_server_destroy(fr_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->wake.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaStreamSynchronize(s->stream);
    for (auto& r : s->all) s->release(*r);
    cudaFree(s->light_da);
    cudaStreamDestroy(s->stream);
    delete s;
}

}  // extern "C"
