"""Environment-map lighting (lights at infinity, Sec. 7) on the GPU against
the FP64 oracle: the rendered image and its hit and visibility records, and
the gradients of the interior, primary-edge and shadow-boundary terms with
respect to the geometry, the textures and the map's radiance."""
import numpy as np
import pytest

import oracle
import scenes
from paper_2101_05356_gb300 import synth

from tests.parity import compare_grads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _case(name):
    if name == "box":               # occluder shadow on a floor under a bright texel
        return scenes.env_box()
    if name == "mixed":             # area emitters and environment blocks together
        return scenes.mixed_box()
    if name == "tiny12":            # a map side that is not a power of two
        sc = synth.make_scene("tiny", env=(12, 3))
        return sc, synth.random_params(sc, 6)
    sc = synth.make_scene("tiny", env=(8, 2))
    return sc, synth.random_params(sc, 2)


def _records(sc, pr, r, dp, iteration):
    img, tri, mask = r.records(dp, iteration=iteration)
    oi, ot, om = oracle.render(sc, pr, records=True, iteration=iteration)
    agree = (tri.cpu().numpy() == ot) & (mask.cpu().numpy().view(np.uint64) == om).all(axis=1)
    px_ok = agree.reshape(-1, sc.spp).all(axis=1).reshape(sc.height, sc.width)
    return img.cpu().numpy(), oi, agree, px_ok


@pytest.mark.parametrize("name", ["tiny", "box", "mixed", "tiny12"])
def test_env_forward_parity(name):
    """Pixels whose samples agree on hit and visibility match within 1e-4;
    at most a couple of samples (FP32 vs FP64 directions grazing an edge) may
    disagree."""
    from paper_2101_05356_gb300 import facert
    sc, pr = _case(name)
    r = facert.Renderer(sc)
    dp = r.device_params(pr)
    g, o, agree, px_ok = _records(sc, pr, r, dp, 3)
    assert np.sum(~agree) <= max(2, 1e-4 * agree.size), int(np.sum(~agree))
    assert o.max() > 0.05
    err = np.abs(g - o) / np.maximum(np.abs(o), 1e-2 * o.mean())
    assert np.max(err[px_ok]) <= 1e-4, float(np.max(err[px_ok]))
    assert r.status() == 0


def test_env_shadow_lists_match_the_oracle():
    """Per-block shadow-candidate lists (exact range of n . w over the block, FP64)."""
    from paper_2101_05356_gb300 import facert
    sc, pr = _case("tiny")
    r = facert.Renderer(sc)
    E = r.n_edges
    prim = torch.empty(E, dtype=torch.int32, device="cuda")
    npr = torch.empty(1, dtype=torch.int32, device="cuda")
    per = torch.empty((sc.n_lights, E), dtype=torch.int32, device="cuda")
    cnt = torch.empty(sc.n_lights, dtype=torch.int32, device="cuda")
    facert.fr_debug_silhouettes(r.ctx, r.device_params(pr), prim, npr, per, cnt)
    po, lo = oracle.silhouettes(sc, pr)
    assert np.array_equal(prim.cpu().numpy()[: int(npr.item())], po)
    c = cnt.cpu().numpy()
    per = per.cpu().numpy()
    for j in range(sc.n_lights):
        assert 0 < c[j] < E, j
        assert np.array_equal(per[j, : c[j]], lo[j]), j


def _compare(gg, go, groups, rtol=1e-3):
    """Group norm and per element (entries >= 1e-2 of the group's largest) at
    rtol, every group with a non-zero oracle gradient."""
    for k in groups:
        assert np.linalg.norm(np.asarray(go[k], np.float64)) > 0.0, k
    compare_grads(gg, go, groups, rtol)


@pytest.mark.parametrize("name,term", [("tiny", "interior"), ("box", "interior"), ("box", "shadow"),
                                       ("box", "primary"), ("tiny", "primary"), ("tiny", "all"), ("box", "all"),
                                       ("mixed", "interior"), ("mixed", "shadow"), ("mixed", "all"),
                                       ("tiny12", "interior"), ("tiny12", "all")])
def test_env_gradient_parity(name, term):
    from paper_2101_05356_gb300 import facert
    sc, pr = _case(name)
    nse = facert.FLAG_NO_SPECULAR_EDGE
    flags = {"interior": facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE | nse,
             "shadow": facert.FLAG_NO_INTERIOR | facert.FLAG_NO_PRIMARY_EDGE | nse,
             "primary": facert.FLAG_NO_INTERIOR | facert.FLAG_NO_SHADOW_EDGE | nse, "all": 0}[term]
    terms = {"interior": oracle.TERM_INTERIOR, "shadow": oracle.TERM_SHADOW, "primary": oracle.TERM_PRIMARY,
             "all": oracle.TERM_ALL}[term]
    r = facert.Renderer(sc, flags=flags)
    dp = r.device_params(pr)
    _, _, _, px_ok = _records(sc, pr, r, dp, 0)
    adj = np.random.default_rng(11).uniform(0.2, 1.0, (sc.height, sc.width, 3)) * px_ok[..., None]
    gg = r.backward(dp, torch.as_tensor(adj, dtype=torch.float32).cuda())
    go = oracle.grad(sc, pr, adj.astype(np.float32).astype(np.float64), terms=terms)
    groups = {"interior": ["env", "coef", "rot", "trans", "focal", "diffuse", "roughness"],
              "shadow": ["coef", "rot"], "primary": ["coef", "focal"],
              "all": ["env", "coef", "rot", "trans", "diffuse"]}[term]
    if name == "mixed" and term != "shadow":
        groups = groups + ["light_i"]
    _compare(gg, go, groups)
    env_lights = sc.lights[:, 0] == synth.LIGHT_ENV
    assert np.all(gg["light_i"].cpu().numpy()[env_lights] == 0.0)
    assert r.status() == 0


def test_env_blocks_are_validated():
    from paper_2101_05356_gb300 import facert
    sc, pr = _case("tiny")
    ctx = facert.fr_create(sc.width, sc.height, sc.spp, sc.tex_size, 1, 0, 0, 1)
    try:
        facert.fr_set_mesh(ctx, sc.mean, sc.basis, sc.faces, sc.uv)
        bad = sc.lights.copy()
        bad[0, 2] = 9                  # row range past the 8 x 8 map
        with pytest.raises(facert.FacertError):
            facert.fr_set_lights(ctx, bad, sc.light_d, sc.light_a, None, 8)
        with pytest.raises(facert.FacertError):   # env_size missing
            facert.fr_set_lights(ctx, sc.lights, sc.light_d, sc.light_a, None, 0)
        facert.fr_set_lights(ctx, sc.lights, sc.light_d, sc.light_a, None, 8)
    finally:
        facert.fr_destroy(ctx)


def test_env_stage1_reconstruction_lowers_the_loss():
    """Stage I under an environment map: the map's texels are optimised (with
    the light prior and box) together with shape and pose; the loss falls,
    the map moves and stays finite."""
    from paper_2101_05356_gb300 import facert, optim
    sc = synth.make_scene("tiny", env=(8, 2))
    r = facert.Renderer(sc)
    gt = synth.random_params(sc, 3, coef_scale=0.5)
    target = r.forward(r.device_params(gt), iteration=10 ** 6)
    init = synth.init_params(sc)
    rec = optim.Reconstruction(r, target, init, schedule=optim.Schedule(30, 0))
    e0 = optim.photometric_loss(r, rec.p, target)
    env0 = rec.p["env"].cpu().numpy().copy()
    rec.run()
    e1 = optim.photometric_loss(r, rec.p, target)
    env1 = rec.p["env"].cpu().numpy()
    assert r.status() == 0
    assert e1 < e0, (e0, e1)
    assert not np.array_equal(env0, env1)
    assert np.all(np.isfinite(env1))


def test_native_server_rejects_environment_contexts():
    from paper_2101_05356_gb300 import facert
    sc, _ = _case("tiny")
    r = facert.Renderer(sc, max_batch=2)
    with pytest.raises(facert.FacertError):
        facert.fr_server_create(r.ctx, max_slots=2)


def test_env_batch_matches_single_renders():
    """fr_render_batch over faces of mixed size and spp under an environment
    map: every face gets the image, loss and gradients of its single render."""
    import dataclasses
    from paper_2101_05356_gb300 import facert
    base = synth.make_scene("tiny", env=(8, 2))
    cases = [(24, 24, 2, 1, 0, 0), (16, 20, 4, 2, 5, 1), (8, 8, 8, 4, 2, 2)]
    big = facert.Renderer(base, max_batch=len(cases))
    items, expect = [], []
    for (w, h, spp, seed, it, face) in cases:
        sc = dataclasses.replace(base, width=w, height=h, spp=spp)
        prm = synth.random_params(sc, seed)
        tgt = torch.as_tensor(np.random.default_rng(seed).uniform(0, 0.1, (h, w, 3)), dtype=torch.float32).cuda()
        solo = facert.Renderer(sc)
        dp = solo.device_params(prm)
        img, loss, g = solo.render(dp, tgt, iteration=it, face_id=face)
        expect.append((img.cpu().numpy(), loss.item(), {k: v.cpu().numpy() for k, v in g.items()}))
        solo.close()
        dpb = big.device_params(prm)
        items.append(dict(width=w, height=h, spp=spp, edge_spp=1, flags=0, iteration=it, face_id=face, params=dpb,
                          target=tgt, image=torch.zeros((h, w, 3), device="cuda"),
                          loss=torch.zeros(1, dtype=torch.float64, device="cuda"), grads=big.zero_grads(dpb)))
    facert.fr_render_batch(big.ctx, items)
    torch.cuda.synchronize()
    assert big.status() == 0
    for it, (img, loss, g) in zip(items, expect):
        assert np.array_equal(it["image"].cpu().numpy(), img)
        assert it["loss"].item() == pytest.approx(loss, rel=1e-12)
        assert np.abs(g["env"]).max() > 0.0
        for k in g:
            a = it["grads"][k].cpu().numpy()
            assert np.allclose(a, g[k], rtol=1e-4, atol=1e-5 * max(np.abs(g[k]).max(), 1e-12)), k


def test_env_autograd_function_gives_the_map_gradient():
    """RenderFn carries the environment map: its gradient through autograd
    equals the adjoint call's for the same samples."""
    from paper_2101_05356_gb300 import autograd, facert
    sc, pr = _case("box")
    r = facert.Renderer(sc)
    dp = r.device_params(pr)
    adj = torch.as_tensor(np.random.default_rng(2).uniform(0.2, 1.0, (sc.height, sc.width, 3)),
                          dtype=torch.float32).cuda()
    want = r.backward(dp, adj, iteration=4)
    p = {k: v.clone().requires_grad_(k in ("env", "coef")) for k, v in dp.items()}
    img = autograd.render(r, p, iteration=4)
    (img * adj).sum().backward()
    assert torch.equal(p["env"].grad, want["env"])
    assert torch.equal(p["coef"].grad, want["coef"])
