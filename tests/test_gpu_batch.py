"""Batched launches: every face of a mixed batch (different image sizes,
sample counts, parameters and Philox streams) gets the same image, loss and
gradients as when it is rendered alone."""
import dataclasses

import numpy as np
import pytest

from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [  # (width, height, spp, param seed, iteration, face id)
    (24, 24, 2, 1, 0, 0),
    (16, 20, 4, 2, 5, 1),
    (24, 24, 1, 3, 9, 7),
    (8, 8, 8, 4, 2, 2),
]


def test_batch_matches_single_renders():
    from paper_2101_05356_gb300 import facert
    base = synth.make_scene("tiny")
    big = facert.Renderer(base, max_batch=len(CASES))
    items, expect = [], []
    for (w, h, spp, seed, it, face) in CASES:
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
                          loss=torch.zeros(1, dtype=torch.float64, device="cuda"),
                          grads=big.zero_grads(dpb)))
    facert.fr_render_batch(big.ctx, items)
    torch.cuda.synchronize()
    assert big.status() == 0
    for it, (img, loss, g) in zip(items, expect):
        assert np.array_equal(it["image"].cpu().numpy(), img)
        assert it["loss"].item() == pytest.approx(loss, rel=1e-12)
        for k in g:
            a = it["grads"][k].cpu().numpy()
            assert np.allclose(a, g[k], rtol=1e-4, atol=1e-5 * max(np.abs(g[k]).max(), 1e-12)), k
