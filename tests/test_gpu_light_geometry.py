"""Virtual light stage geometry (Sec. 3.3) on the GPU against the FP64 oracle:
lights built from each light's distance, relative area and barycentric
centre, the rendered image, and the gradients with respect to (d, a, p) from
the interior term and from the moving-emitter shadow-boundary term."""
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


def _case(name="ico", seed=4):
    if name == "box":               # two stage lights casting the occluder's shadow on the floor
        return scenes.stage_box()
    sc = synth.make_scene("tiny", light_stage="ico")
    pr = synth.with_stage_geometry(sc, synth.random_params(sc, 1), seed=seed)
    return sc, pr


def _records(sc, pr, r, dp, iteration):
    img, tri, mask = r.records(dp, iteration=iteration)
    oi, ot, om = oracle.render(sc, pr, records=True, iteration=iteration)
    agree = (tri.cpu().numpy() == ot) & (mask.cpu().numpy().view(np.uint64) == om).all(axis=1)
    px_ok = agree.reshape(-1, sc.spp).all(axis=1).reshape(sc.height, sc.width)
    return img.cpu().numpy(), oi, agree, px_ok


def test_stage_lights_at_the_generator_values_match_the_records():
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene("tiny", light_stage="ico")
    pr = synth.random_params(sc, 1)
    r = facert.Renderer(sc)
    a = r.forward(r.device_params(pr), iteration=2).cpu().numpy()
    b = r.forward(r.device_params(synth.with_stage_geometry(sc, pr)), iteration=2).cpu().numpy()
    assert np.allclose(a, b, rtol=1e-4, atol=1e-6 * a.max())


@pytest.mark.parametrize("name", ["ico", "box"])
def test_forward_parity_with_moved_lights(name):
    from paper_2101_05356_gb300 import facert
    sc, pr = _case(name)
    r = facert.Renderer(sc)
    dp = r.device_params(pr)
    g, o, agree, px_ok = _records(sc, pr, r, dp, 3)
    assert np.mean(~agree) <= 1e-4, int(np.sum(~agree))
    err = np.abs(g - o) / np.maximum(np.abs(o), 1e-2 * o.mean())
    assert np.max(err[px_ok]) <= 1e-4, float(np.max(err[px_ok]))
    assert r.status() == 0


def _compare(gg, go, groups, rtol=1e-3):
    """Group norm and per element (entries >= 1e-2 of the group's largest) at
    rtol, every group with a non-zero oracle gradient."""
    for k in groups:
        assert np.linalg.norm(np.asarray(go[k], np.float64)) > 0.0, k
    compare_grads(gg, go, groups, rtol)


@pytest.mark.parametrize("name,term", [("ico", "interior"), ("box", "interior"), ("box", "shadow"),
                                       ("ico", "all"), ("box", "all")])
def test_light_geometry_gradient_parity(name, term):
    from paper_2101_05356_gb300 import facert
    sc, pr = _case(name)
    nse = facert.FLAG_NO_SPECULAR_EDGE
    flags = {"interior": facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE | nse,
             "shadow": facert.FLAG_NO_INTERIOR | facert.FLAG_NO_PRIMARY_EDGE | nse, "all": 0}[term]
    terms = {"interior": oracle.TERM_INTERIOR, "shadow": oracle.TERM_SHADOW, "all": oracle.TERM_ALL}[term]
    r = facert.Renderer(sc, flags=flags)
    dp = r.device_params(pr)
    _, _, _, px_ok = _records(sc, pr, r, dp, 0)
    adj = np.random.default_rng(11).uniform(0.2, 1.0, (sc.height, sc.width, 3)) * px_ok[..., None]
    gg = r.backward(dp, torch.as_tensor(adj, dtype=torch.float32).cuda())
    go = oracle.grad(sc, pr, adj.astype(np.float32).astype(np.float64), terms=terms)
    groups = ["light_d", "light_a", "light_p"] + (["light_i", "coef", "rot"] if term != "shadow" else [])
    _compare(gg, go, groups)
    assert r.status() == 0
