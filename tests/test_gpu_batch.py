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


def test_losses_of_a_64_face_batch_are_stored_not_accumulated():
    """Every item of a batch of 64 (above 32 included) gets its loss stored, not
    added onto what its buffer held: loss buffers pre-filled with a non-zero
    value, the same batch called twice, each loss equal bitwise to the face's
    single fr_render (the loss reduction does not depend on block order)."""
    from paper_2101_05356_gb300 import facert
    base = synth.make_scene("tiny")
    n = 64
    big = facert.Renderer(base, max_batch=n)
    solo = facert.Renderer(base)
    items, expect = [], []
    for k in range(n):
        w, h, spp = (16, 12, 2) if k % 2 else (24, 24, 4)
        sc = dataclasses.replace(base, width=w, height=h, spp=spp)
        prm = synth.random_params(sc, 100 + k)
        tgt = torch.as_tensor(np.random.default_rng(k).uniform(0, 0.1, (h, w, 3)), dtype=torch.float32).cuda()
        one = facert.Renderer(sc)
        _, loss, _ = one.render(one.device_params(prm), tgt, iteration=3, face_id=k, with_grad=False)
        expect.append(loss.item())
        one.close()
        items.append(dict(width=w, height=h, spp=spp, edge_spp=1, flags=0, iteration=3, face_id=k,
                          params=big.device_params(prm), target=tgt, image=torch.zeros((h, w, 3), device="cuda"),
                          loss=torch.full((1,), 1.0e6 + k, dtype=torch.float64, device="cuda")))
    solo.close()
    for call in range(2):
        facert.fr_render_batch(big.ctx, items)
        torch.cuda.synchronize()
        assert big.status() == 0
        got = [it["loss"].item() for it in items]
        assert got == expect, (call, [k for k in range(n) if got[k] != expect[k]])
    big.close()
