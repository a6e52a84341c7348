"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Both sides draw the same Philox samples, so the comparison is per sample:
hit triangles and shadow masks must agree except for rare FP32/FP64 flips at
edges; radiance and gradients are compared where the records agree.
Tolerances: radiance 1e-4 relative (per pixel, floor 1e-2 x mean), gradients
1e-3 relative per parameter group (norm) and per element on the entries of
at least 1e-2 of the group's largest, as fixed for the FP32 path, for every
term (interior, primary-visibility and shadow-boundary) and the fused step."""
import numpy as np
import pytest

import oracle
from paper_2101_05356_gb300 import synth
from tests import scenes
from tests.parity import compare_grads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_05356_gb300 import facert
    facert.lib()


def _renderer(sc, **kw):
    from paper_2101_05356_gb300 import facert
    return facert.Renderer(sc, **kw)


SCENES = {
    "tiny": lambda: (synth.make_scene("tiny"), None),
    "c1": lambda: (synth.make_scene("c1"), None),
    "ragged": lambda: (synth.make_scene("tiny", width=37, height=29, spp=8), None),
    "box": lambda: scenes.shadow_box(),
    # 80 lights: two 64-light visibility chunks
    "many": lambda: (synth.make_scene("tiny", n_lights=80), None),
    # the paper's icosahedral virtual light stage (20 triangular lights) and
    # its 80-face sphere variant
    "ico": lambda: (synth.make_scene("tiny", light_stage="ico"), None),
    "sphere80": lambda: (synth.make_scene("c1", light_stage="sphere80"), None),
    # scenes where shadow boundaries are sampled often: the shadow box under 80
    # small quads (the second visibility word in use) and under the icosahedral stage
    "many_box": lambda: scenes.many_box(),
    "ico_box": lambda: scenes.ico_box(),
    # a coarse prism whose silhouette-adjacent faces carry the curve n_s . o = 0
    # under a strong specular lobe
    "tube": lambda: scenes.tube(),
}


def _scene(name, seed=0):
    sc, pr = SCENES[name]()
    if pr is None:
        pr = synth.random_params(sc, seed)
    return sc, pr


def test_philox_bit_exact():
    from paper_2101_05356_gb300 import facert
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, size=(2048, 4), dtype=np.uint64).astype(np.uint32)
    k0, k1 = 0x12345678, 0x9abcdef0
    dc = torch.as_tensor(ctr.view(np.int32)).cuda()
    out = torch.empty_like(dc)
    facert.fr_philox(k0, k1, dc, out)
    got = out.cpu().numpy().view(np.uint32)
    for i in range(0, 2048, 7):
        assert list(got[i]) == list(oracle.philox(k0, k1, *[int(x) for x in ctr[i]]))


@pytest.mark.parametrize("name", ["tiny", "c1", "box"])
def test_geometry_matches_oracle(name):
    sc, pr = _scene(name)
    r = _renderer(sc)
    dp = r.device_params(pr)
    v = torch.empty((sc.n_vertices, 3), device="cuda")
    n = torch.empty((sc.n_vertices, 3), device="cuda")
    from paper_2101_05356_gb300 import facert
    facert.fr_debug_geometry(r.ctx, dp, v, n)
    vo, no = oracle.geometry(sc, pr)
    assert np.max(np.abs(v.cpu().numpy() - vo)) <= 1e-5 * max(1.0, np.abs(vo).max())
    assert np.max(np.abs(n.cpu().numpy() - no)) <= 2e-5


@pytest.mark.parametrize("name", ["tiny", "c1", "c2"])
@pytest.mark.parametrize("rebuild", [False, True])
def test_bvh_is_valid(name, rebuild):
    """The refitted static SAH topology (default) and the per-call LBVH."""
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene(name) if name == "c2" else _scene(name)[0]
    pr = synth.random_params(sc, 0)
    r = _renderer(sc, flags=facert.FLAG_LBVH if rebuild else 0)
    from paper_2101_05356_gb300 import facert
    out = torch.zeros(3, dtype=torch.int32, device="cuda")
    facert.fr_debug_bvh(r.ctx, r.device_params(pr), out)
    leaves, bad, depth = out.cpu().tolist()
    assert leaves == sc.n_triangles
    assert bad == 0
    assert depth <= 64
    assert r.status() == 0


@pytest.mark.parametrize("name", ["tiny", "c1"])
def test_closest_hit_matches_brute_force(name):
    sc, pr = _scene(name)
    r = _renderer(sc)
    rng = np.random.default_rng(3)
    n = 4096
    tgt = np.stack([rng.uniform(-1.0, 1.0, n), rng.uniform(-1.2, 1.2, n), np.full(n, -4.5)], 1)
    org = np.zeros((n, 3))
    org[: n // 2] = rng.uniform(-0.2, 0.2, (n // 2, 3))
    dirs = tgt - org
    from paper_2101_05356_gb300 import facert
    tri = torch.empty(n, dtype=torch.int32, device="cuda")
    t = torch.empty(n, dtype=torch.float32, device="cuda")
    facert.fr_debug_trace(r.ctx, r.device_params(pr), torch.as_tensor(org, dtype=torch.float32).cuda(),
                          torch.as_tensor(dirs, dtype=torch.float32).cuda(), tri, t)
    tri_o, t_o = oracle.closest_hit(sc, pr, org.astype(np.float32).astype(np.float64),
                                    dirs.astype(np.float32).astype(np.float64))
    tri_g = tri.cpu().numpy()
    same = tri_g == tri_o
    assert np.mean(~same) <= 1e-3, np.sum(~same)
    hit = same & (tri_o >= 0)
    assert np.mean(tri_o >= 0) > 0.2
    assert np.allclose(t.cpu().numpy()[hit], t_o[hit], rtol=1e-5)


def _records_and_image(sc, pr, r, dp, iteration=0):
    img, tri, mask = r.records(dp, iteration=iteration)
    oi, ot, om = oracle.render(sc, pr, records=True, iteration=iteration)
    tri_g = tri.cpu().numpy()
    mask_g = mask.cpu().numpy().view(np.uint64)
    agree = (tri_g == ot) & (mask_g == om).all(axis=1)     # both visibility words
    px_ok = agree.reshape(-1, sc.spp).all(axis=1).reshape(sc.height, sc.width)
    return img.cpu().numpy(), oi, agree, px_ok


@pytest.mark.parametrize("name", ["tiny", "c1", "ragged", "box", "many", "ico", "sphere80", "many_box", "ico_box"])
def test_forward_parity(name):
    sc, pr = _scene(name)
    r = _renderer(sc)
    dp = r.device_params(pr)
    g, o, agree, px_ok = _records_and_image(sc, pr, r, dp, iteration=3)
    assert np.mean(~agree) <= 1e-4, int(np.sum(~agree))
    scale = 1e-2 * o.mean()
    err = np.abs(g - o) / np.maximum(np.abs(o), scale)
    assert np.max(err[px_ok]) <= 1e-4, np.max(err[px_ok])
    assert r.status() == 0


@pytest.mark.parametrize("name", ["c1", "box"])
def test_forward_parity_with_lbvh_rebuild(name):
    """The same records and radiance with the per-call LBVH instead of the
    refitted topology (the closest hit and any hit do not depend on the tree)."""
    from paper_2101_05356_gb300 import facert
    sc, pr = _scene(name)
    r = _renderer(sc, flags=facert.FLAG_LBVH)
    dp = r.device_params(pr)
    g, o, agree, px_ok = _records_and_image(sc, pr, r, dp, iteration=3)
    assert np.mean(~agree) <= 1e-4, int(np.sum(~agree))
    scale = 1e-2 * o.mean()
    err = np.abs(g - o) / np.maximum(np.abs(o), scale)
    assert np.max(err[px_ok]) <= 1e-4, np.max(err[px_ok])
    ref = _renderer(sc)
    assert torch.equal(ref.forward(dp, iteration=3), r.forward(dp, iteration=3))
    assert r.status() == 0


@pytest.mark.parametrize("flags", [oracle.GGX, oracle.SCHLICK_LINEAR, oracle.FLAT, oracle.VIEW_CUTOFF])
def test_forward_parity_modes(flags):
    sc, pr = _scene("tiny")
    r = _renderer(sc, flags=flags)       # library flag bits equal the oracle's
    dp = r.device_params(pr)
    img, tri, mask = r.records(dp)
    oi, ot, om = oracle.render(sc, pr, records=True, flags=flags)
    agree = (tri.cpu().numpy() == ot) & (mask.cpu().numpy().view(np.uint64) == om).all(axis=1)
    px_ok = agree.reshape(-1, sc.spp).all(axis=1).reshape(sc.height, sc.width)
    g = img.cpu().numpy()
    err = np.abs(g - oi) / np.maximum(np.abs(oi), 1e-2 * oi.mean())
    assert np.max(err[px_ok]) <= 1e-4


def test_silhouette_lists_match():
    sc, pr = _scene("c1")
    r = _renderer(sc)
    from paper_2101_05356_gb300 import facert
    E = r.n_edges
    prim = torch.empty(E, dtype=torch.int32, device="cuda")
    npr = torch.empty(1, dtype=torch.int32, device="cuda")
    per = torch.empty((sc.n_lights, E), dtype=torch.int32, device="cuda")
    cnt = torch.empty(sc.n_lights, dtype=torch.int32, device="cuda")
    facert.fr_debug_silhouettes(r.ctx, r.device_params(pr), prim, npr, per, cnt)
    po, lo = oracle.silhouettes(sc, pr)
    ev, _ = oracle.edges(sc)
    assert E == len(ev)
    assert np.array_equal(prim.cpu().numpy()[: int(npr.item())], po)
    c = cnt.cpu().numpy()
    per = per.cpu().numpy()
    for j in range(sc.n_lights):
        assert np.array_equal(per[j, : c[j]], lo[j])


def test_loss_parity():
    sc, pr = _scene("c1")
    r = _renderer(sc)
    dp = r.device_params(pr)
    img = r.forward(dp)
    tgt = oracle.render(sc, synth.random_params(sc, 5)).astype(np.float32)
    loss, adj, bl = r.loss(img, torch.as_tensor(tgt).cuda())
    lo, blo, ado = oracle.loss(img.cpu().numpy().astype(np.float64), tgt)
    assert loss.item() == pytest.approx(lo, rel=1e-6)
    assert np.max(np.abs(bl.cpu().numpy() - blo)) <= 1e-6
    # signs can only differ where the blurred residual is ~0 in float32
    d = np.abs(adj.cpu().numpy() - ado)
    assert np.mean(d > 1e-5) < 1e-3


def _masked_adjoint(sc, pr, r, dp, seed=11):
    adj = np.random.default_rng(seed).uniform(0.2, 1.0, (sc.height, sc.width, 3))
    _, _, _, px_ok = _records_and_image(sc, pr, r, dp)
    return adj * px_ok[..., None]


GROUPS = ["coef", "rot", "trans", "focal", "light_i", "diffuse", "specular", "roughness"]


def _compare_grads(gg, go, groups, rtol=1e-3):
    compare_grads(gg, go, groups, rtol)


@pytest.mark.parametrize("name", ["tiny", "c1", "box", "many", "ico", "many_box"])
def test_interior_gradient_parity(name):
    from paper_2101_05356_gb300 import facert
    sc, pr = _scene(name)
    r = _renderer(sc, flags=facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE | facert.FLAG_NO_SPECULAR_EDGE)
    dp = r.device_params(pr)
    adj = _masked_adjoint(sc, pr, r, dp)
    gg = r.backward(dp, torch.as_tensor(adj, dtype=torch.float32).cuda())
    go = oracle.grad(sc, pr, adj.astype(np.float32).astype(np.float64), terms=oracle.TERM_INTERIOR)
    _compare_grads(gg, go, GROUPS)


@pytest.mark.parametrize("name", ["tiny", "c1", "box"])
def test_primary_edge_gradient_parity(name):
    from paper_2101_05356_gb300 import facert
    sc, pr = _scene(name)
    r = _renderer(sc, edge_spp=2, flags=facert.FLAG_NO_INTERIOR | facert.FLAG_NO_SHADOW_EDGE |
                  facert.FLAG_NO_SPECULAR_EDGE)
    dp = r.device_params(pr)
    adj = _masked_adjoint(sc, pr, r, dp)
    gg = r.backward(dp, torch.as_tensor(adj, dtype=torch.float32).cuda())
    go = oracle.grad(sc, pr, adj.astype(np.float32).astype(np.float64), terms=oracle.TERM_PRIMARY, edge_spp=2)
    _compare_grads(gg, go, ["coef", "rot", "trans", "focal"])


@pytest.mark.parametrize("name", ["box", "many_box", "ico_box"])
def test_shadow_edge_gradient_parity(name):
    """The shadow-boundary term on scenes whose occluder casts shadows from every
    light (on convex meshes and on the small faces it is exactly zero: no
    boundary sample lands on an emitter)."""
    from paper_2101_05356_gb300 import facert
    sc, pr = _scene(name)
    r = _renderer(sc, flags=facert.FLAG_NO_INTERIOR | facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SPECULAR_EDGE)
    dp = r.device_params(pr)
    adj = _masked_adjoint(sc, pr, r, dp)
    gg = r.backward(dp, torch.as_tensor(adj, dtype=torch.float32).cuda())
    go = oracle.grad(sc, pr, adj.astype(np.float32).astype(np.float64), terms=oracle.TERM_SHADOW)
    assert np.linalg.norm(go["coef"]) > 0.0
    _compare_grads(gg, go, ["coef", "rot", "trans", "focal"])


@pytest.mark.parametrize("name,edge_spp,mode", [("tube", 1, ""), ("tube", 2, ""), ("tiny", 1, ""), ("c1", 2, ""),
                                                ("tube", 1, "ggx"), ("tube", 1, "cutoff")])
def test_specular_boundary_gradient_parity(name, edge_spp, mode):
    """The boundary term of the specular lobe's cutoff inside triangles (the
    curve n_s . o = 0 met along scanlines) against the oracle's, per element;
    also with the GGX lobe (its jump G1(o) / (n . o) -> 2 / alpha) and under
    the reading that cuts every contribution there (the jump is the whole
    radiance)."""
    from paper_2101_05356_gb300 import facert
    sc, pr = _scene(name)
    extra, oflags = {"": (0, 0), "ggx": (facert.FLAG_GGX, oracle.GGX),
                     "cutoff": (facert.FLAG_VIEW_CUTOFF, oracle.VIEW_CUTOFF)}[mode]
    r = _renderer(sc, edge_spp=edge_spp,
                  flags=facert.FLAG_NO_INTERIOR | facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE | extra)
    dp = r.device_params(pr)
    adj = _masked_adjoint(sc, pr, r, dp)
    groups = ["coef", "rot", "trans", "focal"]

    def both(a):
        gg = r.backward(dp, torch.as_tensor(a, dtype=torch.float32).cuda())
        assert r.status() == 0
        return gg, oracle.grad(sc, pr, a.astype(np.float32).astype(np.float64), terms=oracle.TERM_SPECULAR,
                               edge_spp=edge_spp, flags=oflags)

    # every crossing: group norms
    gg, go = both(adj)
    assert abs(go["focal"][0]) > 0.0
    for k in groups:
        a, b = gg[k].cpu().numpy().astype(np.float64).ravel(), np.asarray(go[k], np.float64).ravel()
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), k
    # element by element, without the pixels of crossings on triangles seen within 0.06 degrees of
    # edge-on: kappa = |n_f| |v_0| / |n_f . v_0| > 1000 amplifies the FP32 rounding of the vertex
    # positions in the crossing's position and velocity by about kappa (the C1 face's two such
    # pixels: 1.8e-3 per element with them, 7.4e-4 without)
    v, _ = oracle.geometry(sc, pr)
    for scan in range((sc.width + sc.height) * edge_spp):
        tr, xy = oracle.spec_crossings(sc, pr, scan, edge_spp=edge_spp)
        for (t, _), (x, y) in zip(tr, xy):
            i0, i1, i2 = sc.faces[t]
            nf = np.cross(v[i1] - v[i0], v[i2] - v[i0])
            if np.linalg.norm(nf) * np.linalg.norm(v[i0]) > 1000.0 * abs(np.dot(nf, v[i0])) and \
                    0 <= x < sc.width and 0 <= y < sc.height:
                adj[int(y), int(x)] = 0.0
    gg, go = both(adj)
    _compare_grads(gg, go, groups)


def test_full_gradient_and_render_step_c1():
    """fr_render (forward + loss + adjoint, all terms) against the oracle."""
    sc, pr = _scene("c1")
    r = _renderer(sc)
    dp = r.device_params(pr)
    tgt = oracle.render(sc, synth.random_params(sc, 5)).astype(np.float32)
    img, loss, gg = r.render(dp, torch.as_tensor(tgt).cuda(), iteration=2)
    oi = oracle.render(sc, pr, iteration=2)
    lo, _, ado = oracle.loss(img.cpu().numpy().astype(np.float64), tgt)
    assert loss.item() == pytest.approx(lo, rel=1e-6)
    go = oracle.grad(sc, pr, ado, iteration=2)
    # every term at once, on the unmasked loss adjoint: the same bars as the terms alone
    _compare_grads(gg, go, GROUPS)
    err = np.abs(img.cpu().numpy() - oi) / np.maximum(np.abs(oi), 1e-2 * oi.mean())
    assert np.max(err) <= 1e-4, float(np.max(err))
