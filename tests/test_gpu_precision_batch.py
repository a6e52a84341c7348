"""The batched precision configuration: 64 faces through one batched call
with the morph as one BF16 x BF16 -> FP32 tensor-core GEMM over the whole
batch (MMA width 64), FP32 tracing and shading, against the FP64 oracle per
result.  Faces of the 2,562-vertex face (K = 20) and of the 35,709-vertex
face (basis 107,127 x 144).  Per face: the morphed vertices within the BF16
rounding bound, and the rendered image at sampled pixels; targets are renders
of random ground-truth parameters plus N(0, 0.01) pixel noise, and the loss
and gradient of the batched call equal those of FP32-morph single calls up to
the BF16 morph's own effect.  The served form's gradient is also pinned
exactly: it must equal the oracle's gradient taken at the geometry the BF16
morph produced (within the FP32 path's 1e-3, per element)."""
import numpy as np
import pytest

import oracle
from paper_2101_05356_gb300 import synth
from tests.parity import compare_grads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_FACES = 64


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _batch(r, sc, prs, targets, grads=True):
    items = []
    for k, pr in enumerate(prs):
        dp = r.device_params(pr)
        items.append(dict(width=sc.width, height=sc.height, spp=sc.spp, edge_spp=1, flags=0, iteration=3, face_id=k,
                          params=dp, target=targets[k], image=torch.zeros((sc.height, sc.width, 3), device="cuda"),
                          loss=torch.zeros(1, dtype=torch.float64, device="cuda"),
                          grads=r.zero_grads(dp) if grads else None))
    return items


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_64_face_batch_per_result_error(name):
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene(name)
    if name == "c2":                         # the large basis on the small image configuration
        import dataclasses
        sc = dataclasses.replace(sc, width=64, height=64, spp=4)
    rng = np.random.default_rng(7)
    prs = [synth.random_params(sc, 300 + k) for k in range(N_FACES)]
    r = facert.Renderer(sc, flags=facert.FLAG_MORPH_BF16, max_batch=N_FACES)
    gen = facert.Renderer(sc)
    targets = []
    for k in range(N_FACES):
        gt = gen.forward(gen.device_params(synth.random_params(sc, 900 + k)), iteration=10 ** 7, face_id=k)
        targets.append((gt + torch.as_tensor(rng.normal(0.0, 0.01, gt.shape), dtype=torch.float32).cuda()).contiguous())
    # morph: per element within the BF16 bound, every face of the 64-wide GEMM
    out = torch.empty((N_FACES, sc.n_vertices, 3), device="cuda")
    facert.fr_debug_morph(r.ctx, [r.device_params(p) for p in prs], out)
    items = _batch(r, sc, prs, targets)
    facert.fr_render_batch(r.ctx, items)
    torch.cuda.synchronize()
    assert r.status() == 0
    B = sc.basis.astype(np.float64)
    worst = 0.0
    for k, pr in enumerate(prs):
        q = pr.copy()
        q.rot[:] = 0.0
        q.trans[:] = 0.0
        v, _ = oracle.geometry(sc, q)
        bound = 2.0 ** -7 * np.tensordot(np.abs(pr.coef.astype(np.float64)), np.abs(B), axes=1) + 1e-6
        ratio = float(np.max(np.abs(out[k].cpu().numpy() - v) / bound))
        assert ratio <= 1.0, (k, ratio)
        worst = max(worst, ratio)
    # image: sampled pixels of every face against the FP64 oracle (FP64 morph)
    px = rng.choice(sc.width * sc.height, size=24, replace=False).astype(np.int32)
    rel = []
    for k in range(0, N_FACES, 8):
        o = oracle.render(sc, prs[k], iteration=3, face_id=k, pixels=px).reshape(-1, 3)[px]
        g = items[k]["image"].cpu().numpy().reshape(-1, 3)[px]
        lit = o.sum(axis=1) > 0.0                       # pixels that see the face
        rel.append((np.abs(g - o) / np.maximum(np.abs(o), 1e-2 * max(o.mean(), 1e-6)))[lit])
    rel = np.concatenate(rel).ravel()
    # the batched BF16 call against FP32-morph single calls: losses and gradients
    ref = facert.Renderer(sc)
    dl, dg = [], []
    for k in (0, N_FACES // 2, N_FACES - 1):
        dp = ref.device_params(prs[k])
        img, loss, g = ref.render(dp, targets[k], iteration=3, face_id=k)
        dl.append(abs(items[k]["loss"].item() - loss.item()) / loss.item())
        a, b = items[k]["grads"]["coef"].cpu().numpy(), g["coef"].cpu().numpy()
        dg.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
    print("%s x %d: morph worst error / BF16 bound %.3f; image rel. error vs FP64 oracle on face pixels: median %.2e, "
          "99th pct %.2e; loss vs FP32 morph %.2e; coef gradient vs FP32 morph %.2e"
          % (name, N_FACES, worst, np.median(rel), np.percentile(rel, 99), max(dl), max(dg)))
    # the BF16 morph moves every vertex by up to 2^-7 sum_k |c_k||B_ki| (pinned above), so the image
    # differs from the FP64-morph oracle by more than the FP32 path's 1e-4: report it, bound it loosely;
    # the gradient against the FP32 morph (dg) is reported only: where a silhouette edge changes
    # classification between the two geometries the edge samples pick other edges
    assert np.median(rel) <= 1e-3
    assert max(dl) <= 1e-3
    if name == "c1":
        # exact pin of the served form: the oracle on a face whose mean shape is the vertices the
        # BF16 morph produced (coefficients 0, same basis, pose and everything else) has the same
        # geometry, so its coefficient, pose, focal and light gradients must match the batched
        # call's (textures are compared per element by the masked-adjoint parity tests: with this
        # unmasked loss adjoint one sample whose FP32 and FP64 hits differ moves its texel taps)
        import dataclasses
        for k in (1, N_FACES - 2):
            sk = dataclasses.replace(sc, mean=out[k].cpu().numpy().astype(np.float32))
            qk = prs[k].copy()
            qk.coef = np.zeros_like(qk.coef)
            _, _, ado = oracle.loss(items[k]["image"].cpu().numpy().astype(np.float64),
                                    targets[k].cpu().numpy())
            go = oracle.grad(sk, qk, ado, iteration=3, face_id=k)
            compare_grads(items[k]["grads"], go, ["coef", "rot", "trans", "focal", "light_i"])
