"""Hit records of a fused step: the adjoint that reads the forward's per-sample
hit triangle and shadow visibility gives the same image, loss and gradients as
the adjoint that re-traces them with the same Philox counters (the gradient
sums are fixed point, so the comparison is exact), and traces no camera or
shadow ray of its own."""
import numpy as np
import pytest

import oracle
from paper_2101_05356_gb300 import synth

from scenes import shadow_box

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = {
    "c1": lambda: synth.make_scene("c1"),
    "box": lambda: shadow_box()[0],
    "many": lambda: synth.make_scene("tiny", n_lights=80),
    "spp64": lambda: synth.make_scene("tiny", width=20, height=12, spp=64),
}


@pytest.mark.parametrize("name", list(CASES))
def test_recorded_adjoint_equals_retraced(name):
    from paper_2101_05356_gb300 import facert
    sc = CASES[name]()
    pr = shadow_box()[1] if name == "box" else synth.random_params(sc, 1)
    tgt = torch.as_tensor(oracle.render(sc, synth.random_params(sc, 5) if name != "box" else pr,
                                        iteration=9).astype(np.float32) * 0.9).cuda()
    out = {}
    for mode, flags in (("records", 0), ("retrace", facert.FLAG_RECOMPUTE)):
        r = facert.Renderer(sc, edge_spp=1, flags=flags)
        dp = r.device_params(pr)
        facert.fr_counters(r.ctx, reset=True)
        img, loss, g = r.render(dp, tgt, iteration=4)
        cnt = facert.fr_counters(r.ctx, reset=True)
        out[mode] = (img.cpu().numpy(), loss.item(), {k: v.cpu().numpy() for k, v in g.items()}, cnt)
        assert r.status() == 0
        r.close()
    ia, la, ga, ca = out["records"]
    ib, lb, gb, cb = out["retrace"]
    assert np.array_equal(ia, ib) and la == lb
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), (k, float(np.max(np.abs(ga[k] - gb[k]))))
    # the recorded adjoint traces only shadow-boundary rays
    assert ca["adjoint"]["rays"] < 0.25 * cb["adjoint"]["rays"]
    assert ca["forward"] == cb["forward"]
