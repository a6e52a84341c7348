"""The allocation-free loss entry point against the context-based one.

fr_loss_noalloc serves callers that cannot allocate device memory (their host
application owns the device memory pool, or a latency-critical loop cannot
absorb an allocation).  It must give the same loss, blurred image and adjoint
as fr_loss, call after call, although every call reuses one static scratch
array, and it must not change the device's free memory.  This file is
collected last on purpose."""
import dataclasses

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


def _check(ref, got):
    assert got[0] == ref[0]                       # the same fixed-order FP64 sum
    assert np.allclose(got[2], ref[2], rtol=0, atol=1e-6)
    assert np.allclose(got[1], ref[1], rtol=0, atol=1e-6)


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
        _check(ref, got)


def test_noalloc_at_its_size_limit_allocates_nothing():
    """At exactly 512 x 512 pixels (the scratch's limit) the result equals
    fr_loss's, twice in a row, and the device's free memory is the same before
    and after the calls (after one warm-up call, which may load the library's
    module on the device)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_05356_gb300 import facert
    sc = dataclasses.replace(synth.make_scene("tiny"), width=512, height=512)
    r = facert.Renderer(sc)
    rng = np.random.default_rng(4)
    imgs = [torch.as_tensor(rng.uniform(0, 1, (512, 512, 3)), dtype=torch.float32).cuda() for _ in range(3)]
    tgt = torch.as_tensor(rng.uniform(0, 1, (512, 512, 3)), dtype=torch.float32).cuda()
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    adj = torch.empty_like(tgt)
    bl = torch.empty_like(tgt)
    facert.fr_loss_noalloc(512, 512, imgs[0], tgt, loss, adj, bl)      # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for img in imgs[1:]:
        facert.fr_loss_noalloc(512, 512, img, tgt, loss, adj, bl)
        torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for img in imgs[1:]:
        ref, got = _loss_both(r, facert, img, tgt)
        _check(ref, got)
    r.close()


def test_noalloc_rejects_images_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_05356_gb300 import facert
    img = torch.zeros((2, 2, 3), device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    for h, w in ((1024, 1024), (512, 513), (0, 4)):
        with pytest.raises(facert.FacertError) as e:
            facert.fr_loss_noalloc(h, w, img, img, loss, img, img)
        assert e.value.code == facert.FR_EINVAL
