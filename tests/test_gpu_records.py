"""Hit records of a fused step: the adjoint that reads the forward's per-sample
hit triangle and shadow visibility gives the same image, loss and gradients as
the adjoint that re-traces them with the same Philox counters (the gradient
sums are fixed point, so the comparison is exact), and traces no camera or
shadow ray of its own.  Images whose records do not fit the record buffer
recompute them tile by tile (a visibility-only forward pass per tile, then the
recorded adjoint): the same results again, for fused steps, batches and the
stand-alone adjoint."""
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
    # a record holds one visibility word up to 64 lights, two from 65
    "l64": lambda: synth.make_scene("tiny", n_lights=64),
    "l65": lambda: synth.make_scene("tiny", n_lights=65),
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


@pytest.mark.parametrize("name", ["c1", "box", "many", "spp64", "l64", "l65"])
def test_tiled_recomputed_records_equal_retraced(name):
    """Records recomputed in about four tiles per image (the last one partial)
    against the re-tracing adjoint:
    bitwise equal image, loss and gradients, through fr_render and through
    fr_backward (which has no forward records of its own)."""
    from paper_2101_05356_gb300 import facert
    sc = CASES[name]()
    pr = shadow_box()[1] if name == "box" else synth.random_params(sc, 1)
    tgt = torch.as_tensor(oracle.render(sc, synth.random_params(sc, 5) if name != "box" else pr,
                                        iteration=9).astype(np.float32) * 0.9).cuda()
    n = sc.width * sc.height * sc.spp
    unit = max(128, sc.spp)
    tile = unit * max(1, (n // 4) // unit)              # about four tiles, the last one partial
    if n % tile == 0:
        tile += unit
    assert n % tile != 0 and n // tile >= 3
    out = {}
    for mode, flags in (("tiled", 0), ("retrace", facert.FLAG_RECOMPUTE)):
        r = facert.Renderer(sc, edge_spp=1, flags=flags)
        if mode == "tiled":
            facert.fr_debug_record_tile(r.ctx, tile)
        dp = r.device_params(pr)
        img, loss, g = r.render(dp, tgt, iteration=4)
        gb = r.backward(dp, torch.as_tensor(np.random.default_rng(2).uniform(0.1, 1.0, (sc.height, sc.width, 3)),
                                            dtype=torch.float32).cuda(), iteration=6)
        out[mode] = (img.cpu().numpy(), loss.item(), {k: v.cpu().numpy() for k, v in g.items()},
                     {k: v.cpu().numpy() for k, v in gb.items()})
        assert r.status() == 0
        r.close()
    ia, la, ga, ba = out["tiled"]
    ib, lb, gb_, bb = out["retrace"]
    assert np.array_equal(ia, ib) and la == lb
    for k in ga:
        assert np.array_equal(ga[k], gb_[k]), ("render", k, float(np.max(np.abs(ga[k] - gb_[k]))))
        assert np.array_equal(ba[k], bb[k]), ("backward", k, float(np.max(np.abs(ba[k] - bb[k]))))


def test_tiled_records_in_a_mixed_batch():
    """A batch mixing images whose records fit one tile (the forward records
    them) with larger ones (recomputed in tiles) gives each face the result of
    its single call."""
    import dataclasses
    from paper_2101_05356_gb300 import facert
    base = synth.make_scene("tiny", width=32, height=32, spp=4)
    big = facert.Renderer(base, edge_spp=1, max_batch=3)
    facert.fr_debug_record_tile(big.ctx, 1024)                       # 32 x 32 x 4 = 4 tiles
    items, expect = [], []
    for k, (w, h, spp) in enumerate([(32, 32, 4), (16, 12, 4), (24, 20, 2)]):
        sc = dataclasses.replace(base, width=w, height=h, spp=spp)
        pr = synth.random_params(sc, 10 + k)
        tgt = torch.as_tensor(np.random.default_rng(k).uniform(0, 0.2, (h, w, 3)), dtype=torch.float32).cuda()
        solo = facert.Renderer(sc, edge_spp=1, flags=facert.FLAG_RECOMPUTE)
        img, loss, g = solo.render(solo.device_params(pr), tgt, iteration=3, face_id=k)
        expect.append((img.cpu().numpy(), loss.item(), {n: v.cpu().numpy() for n, v in g.items()}))
        solo.close()
        dp = big.device_params(pr)
        items.append(dict(width=w, height=h, spp=spp, edge_spp=1, flags=0, iteration=3, face_id=k, params=dp,
                          target=tgt, image=torch.zeros((h, w, 3), device="cuda"),
                          loss=torch.zeros(1, dtype=torch.float64, device="cuda"), grads=big.zero_grads(dp)))
    facert.fr_render_batch(big.ctx, items)
    torch.cuda.synchronize()
    assert big.status() == 0
    for it, (img, loss, g) in zip(items, expect):
        assert np.array_equal(it["image"].cpu().numpy(), img)
        assert it["loss"].item() == pytest.approx(loss, rel=1e-12)
        for n in g:       # the batched call's tolerance against single calls
            a = it["grads"][n].cpu().numpy()
            assert np.allclose(a, g[n], rtol=1e-4, atol=1e-5 * max(np.abs(g[n]).max(), 1e-12)), n
    big.close()
