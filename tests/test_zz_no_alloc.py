"""The allocation-free loss entry point against the context-based one.

fr_loss_noalloc serves callers that cannot allocate device memory (their host
application owns the device memory pool, or a latency-critical loop cannot
absorb an allocation).  It must give the same loss, blurred image and adjoint
as fr_loss, call after call, although every call reuses one static scratch
array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _loss_both(r, facert, img, tgt):
    ref_loss, ref_adj, ref_bl = r.loss(img, tgt)
    h, w = img.shape[:2]
    loss = torch.full((1,), 123.0, dtype=torch.float64, device="cuda")   # must be overwritten
    adj = torch.full_like(img, 7.0)
    bl = torch.full_like(img, 7.0)
    facert.fr_loss_noalloc(h, w, img, tgt, loss, adj, bl)
    torch.cuda.synchronize()
    return (ref_loss.item(), ref_adj.cpu().numpy(), ref_bl.cpu().numpy()), \
           (loss.item(), adj.cpu().numpy(), bl.cpu().numpy())


def test_noalloc_loss_matches_fr_loss_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_05356_gb300 import facert
    results = []
    # two calls in a row with different sizes and contents: the second call
    # must not see anything left in the shared scratch by the first
    for name, seed in (("c1", 1), ("tiny", 2)):
        sc = synth.make_scene(name)
        r = facert.Renderer(sc)
        img = r.forward(r.device_params(synth.random_params(sc, seed)))
        tgt = r.forward(r.device_params(synth.random_params(sc, seed + 10)))
        ref, got = _loss_both(r, facert, img, tgt)
        results.append((ref, got))
        r.close()
    for ref, got in results:
        assert got[0] == pytest.approx(ref[0], rel=1e-6)
        assert np.allclose(got[2], ref[2], rtol=0, atol=1e-6)
        assert np.allclose(got[1], ref[1], rtol=0, atol=1e-6)


def test_noalloc_rejects_images_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_05356_gb300 import facert
    img = torch.zeros((2, 2, 3), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(facert.FacertError) as e:
        facert.fr_loss_noalloc(1024, 1024, img, img, loss, img, img)
    assert e.value.code == facert.FR_EINVAL
