"""Statistical albedo model (Sec. 3.2) on the GPU against the FP64 oracle:
the texture-space morph in FP32 and as the BF16 tensor-core GEMM (batched,
ragged texel counts), its transpose, the chain from the rendered loss to beta
and gamma, and a Stage I reconstruction that optimises them."""
import numpy as np
import pytest

import oracle
from oracle import albedo as oalb
from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _scene(name):
    if name == "c1":
        return synth.make_scene("c1", albedo_k=80)
    # 15 x 15 texels: 675 rows, neither a multiple of 4 nor of 128
    return synth.make_scene("tiny", tex_size=15, albedo_k=7)


def _coefs(sc, n, seed):
    rng = np.random.default_rng(seed)
    a = sc.albedo
    return ([rng.normal(size=a.k_diffuse).astype(np.float32) for _ in range(n)],
            [rng.normal(size=a.k_specular).astype(np.float32) for _ in range(n)])


@pytest.mark.parametrize("name", ["c1", "ragged"])
@pytest.mark.parametrize("bf16", [False, True])
def test_albedo_morph_matches_oracle(name, bf16):
    from paper_2101_05356_gb300 import facert
    sc = _scene(name)
    n = 3
    r = facert.Renderer(sc, flags=facert.FLAG_MORPH_BF16 if bf16 else 0, max_batch=n)
    betas, gammas = _coefs(sc, n, 1)
    M = sc.tex_size
    d = [torch.empty((M, M, 3), device="cuda") for _ in range(n)]
    s = [torch.empty((M, M, 3), device="cuda") for _ in range(n)]
    facert.fr_albedo_morph(r.ctx, [torch.as_tensor(b).cuda() for b in betas],
                           [torch.as_tensor(g).cuda() for g in gammas], d, s)
    torch.cuda.synchronize()
    a = sc.albedo
    for b in range(n):
        for got, mean, basis, c in ((d[b], a.mean_diffuse, a.basis_diffuse, betas[b]),
                                    (s[b], a.mean_specular, a.basis_specular, gammas[b])):
            want = oalb.morph(mean, basis, c)
            scale = np.tensordot(np.abs(c.astype(np.float64)), np.abs(basis.astype(np.float64)), axes=(0, 0))
            err = np.abs(got.cpu().numpy() - want)
            if bf16:
                # BF16 unit roundoff 2^-8 on basis and coefficient: 2^-7 per product
                assert np.all(err <= 2.0 ** -7 * scale + 1e-6), float(np.max(err / (scale + 1e-12)))
            else:
                assert np.all(err <= 1e-6 * (np.abs(mean) + scale) + 1e-7), float(np.max(err))
    assert r.status() == 0


@pytest.mark.parametrize("name", ["c1", "ragged"])
def test_albedo_adjoint_matches_oracle(name):
    from paper_2101_05356_gb300 import facert
    sc = _scene(name)
    n = 2
    r = facert.Renderer(sc, max_batch=n)
    rng = np.random.default_rng(2)
    M = sc.tex_size
    gd = [rng.normal(size=(M, M, 3)).astype(np.float32) for _ in range(n)]
    gs = [rng.normal(size=(M, M, 3)).astype(np.float32) for _ in range(n)]
    a = sc.albedo
    ob = [torch.full((a.k_diffuse,), 0.25, device="cuda") for _ in range(n)]   # added into
    og = [torch.full((a.k_specular,), -0.5, device="cuda") for _ in range(n)]
    facert.fr_albedo_adjoint(r.ctx, [torch.as_tensor(x).cuda() for x in gd], [torch.as_tensor(x).cuda() for x in gs],
                             ob, og)
    torch.cuda.synchronize()
    for b in range(n):
        for got, base, basis, g in ((ob[b], 0.25, a.basis_diffuse, gd[b]), (og[b], -0.5, a.basis_specular, gs[b])):
            want = base + oalb.adjoint(basis, g)
            tol = 1e-5 * np.abs(np.tensordot(np.abs(basis.astype(np.float64)), np.abs(g), axes=([1, 2, 3], [0, 1, 2])))
            assert np.all(np.abs(got.cpu().numpy() - want) <= tol + 1e-6)


def test_loss_gradient_reaches_beta_and_gamma():
    """render -> texture gradients -> transpose equals the oracle's texture
    gradient mapped by the oracle's transpose (interior term)."""
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene("c1", albedo_k=16)
    pr = synth.random_params(sc, 3)
    r = facert.Renderer(sc, flags=facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE |
                         facert.FLAG_NO_SPECULAR_EDGE)
    betas, gammas = _coefs(sc, 1, 4)
    dp = r.device_params(pr)
    facert.fr_albedo_morph(r.ctx, [torch.as_tensor(betas[0]).cuda()], [torch.as_tensor(gammas[0]).cuda()],
                           [dp["diffuse"]], [dp["specular"]])
    # the oracle renders with the GPU's float32 textures (FP32 morph vs FP64 differ by 1e-7)
    q = pr.copy()
    q.diffuse = dp["diffuse"].cpu().numpy()
    q.specular = dp["specular"].cpu().numpy()
    img, tri, mask = r.records(dp, iteration=1)
    oi, ot, om = oracle.render(sc, q, records=True, iteration=1)
    ok = ((tri.cpu().numpy() == ot) & (mask.cpu().numpy().view(np.uint64) == om).all(axis=1)).reshape(-1, sc.spp).all(axis=1)
    adj = np.random.default_rng(6).uniform(0.2, 1.0, (sc.height, sc.width, 3)) * ok.reshape(sc.height, sc.width, 1)
    g = r.backward(dp, torch.as_tensor(adj, dtype=torch.float32).cuda(), iteration=1)
    gb = torch.zeros(16, device="cuda")
    gc = torch.zeros(16, device="cuda")
    facert.fr_albedo_adjoint(r.ctx, [g["diffuse"]], [g["specular"]], [gb], [gc])
    go = oracle.grad(sc, q, adj.astype(np.float32).astype(np.float64), terms=oracle.TERM_INTERIOR, iteration=1)
    for got, basis, gt in ((gb, sc.albedo.basis_diffuse, go["diffuse"]), (gc, sc.albedo.basis_specular, go["specular"])):
        want = oalb.adjoint(basis, gt)
        assert np.linalg.norm(got.cpu().numpy() - want) <= 1e-3 * np.linalg.norm(want)


def test_stage1_optimises_the_statistical_albedo():
    from paper_2101_05356_gb300 import facert, optim
    sc = synth.make_scene("c1", albedo_k=20)
    r = facert.Renderer(sc)
    gt = synth.random_params(sc, 9)
    rng = np.random.default_rng(10)
    gt.diffuse = oalb.morph(sc.albedo.mean_diffuse, sc.albedo.basis_diffuse,
                            rng.normal(size=20) * 1.5).astype(np.float32)
    tgt = r.forward(r.device_params(gt), iteration=10 ** 6)
    rec = optim.Reconstruction(r, tgt, synth.init_params(sc), schedule=optim.Schedule(12, 2))
    losses = []
    for _ in range(12):
        rec.step()
        losses.append(float(rec.loss.item()))
    beta = rec.ab["beta"]["x"].cpu().numpy()
    assert np.abs(beta).max() > 0.0 and np.all(np.isfinite(beta))
    assert min(losses[-3:]) < losses[0]
    # the textures are the statistical albedo of the current coefficients
    want = oalb.morph(sc.albedo.mean_diffuse, sc.albedo.basis_diffuse,
                      beta - 0.0)   # last morph used the pre-step beta; compare loosely
    assert np.abs(rec.p["diffuse"].cpu().numpy() - want).max() < 0.05
    # Stage II starts from the last statistical albedo
    d_before = rec.p["diffuse"].clone()
    rec.step()
    assert torch.equal(rec.ref_diffuse, d_before)
    assert r.status() == 0
