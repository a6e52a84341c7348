"""The batched BF16 tensor-core morph (tcgen05.mma, FP32 accumulate, FP32 mean)
against the FP64 oracle morph, with an error bound derived from BF16 rounding:
basis and coefficients are each rounded to nearest with 8 significant bits
(unit roundoff 2^-8), so each product is off by at most 2^-7 relative, hence
|v_bf16 - v| <= 2^-7 * sum_k |c_k| |B_ki| (+ FP32 accumulation, far smaller)."""
import numpy as np
import pytest

import oracle
from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _exact(sc, pr):
    q = pr.copy()
    q.rot[:] = 0.0
    q.trans[:] = 0.0
    v, _ = oracle.geometry(sc, q)     # v' = v when R = I and T = 0
    return v


@pytest.mark.parametrize("name,nfaces", [("c1", 3), ("c2", 5), ("c1", 32), ("c1", 33), ("c1", 64), ("c2", 64)])
def test_tensor_core_morph_within_bf16_bound(name, nfaces):
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene(name)
    r_tc = facert.Renderer(sc, flags=facert.FLAG_MORPH_BF16, max_batch=nfaces)
    r_32 = facert.Renderer(sc, max_batch=nfaces)
    prs = [synth.random_params(sc, 100 + k) for k in range(nfaces)]
    out_tc = torch.empty((nfaces, sc.n_vertices, 3), device="cuda")
    out_32 = torch.empty((nfaces, sc.n_vertices, 3), device="cuda")
    facert.fr_debug_morph(r_tc.ctx, [r_tc.device_params(p) for p in prs], out_tc)
    facert.fr_debug_morph(r_32.ctx, [r_32.device_params(p) for p in prs], out_32)
    torch.cuda.synchronize()
    assert r_tc.status() == 0
    B = sc.basis.astype(np.float64)                       # [K, N, 3]
    worst = 0.0
    for k, pr in enumerate(prs):
        v = _exact(sc, pr)
        bound = 2.0 ** -7 * np.tensordot(np.abs(pr.coef.astype(np.float64)), np.abs(B), axes=1) + 1e-6
        err_tc = np.abs(out_tc[k].cpu().numpy() - v)
        assert np.all(err_tc <= bound), (k, float(np.max(err_tc / bound)))
        worst = max(worst, float(np.max(err_tc / bound)))
        assert np.allclose(out_32[k].cpu().numpy(), v, rtol=1e-5, atol=1e-6)
    print("worst BF16 error / bound:", worst)


def test_bf16_batch_render_close_to_fp32():
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene("c1")
    n = 4
    outs = {}
    for flags in (0, facert.FLAG_MORPH_BF16):
        r = facert.Renderer(sc, flags=flags, max_batch=n)
        items = []
        for k in range(n):
            dp = r.device_params(synth.random_params(sc, 200 + k))
            items.append(dict(width=sc.width, height=sc.height, spp=sc.spp, edge_spp=1, flags=flags, iteration=1,
                              face_id=k, params=dp, target=torch.zeros((sc.height, sc.width, 3), device="cuda"),
                              image=torch.zeros((sc.height, sc.width, 3), device="cuda"),
                              loss=torch.zeros(1, dtype=torch.float64, device="cuda"), grads=None))
        facert.fr_render_batch(r.ctx, items)
        torch.cuda.synchronize()
        assert r.status() == 0
        outs[flags] = [it["image"].cpu().numpy() for it in items]
    for a, b in zip(outs[0], outs[facert.FLAG_MORPH_BF16]):
        # geometry moves by ~1e-4; images agree except at a few silhouette pixels
        assert np.mean(np.abs(a - b)) < 2e-3 * np.mean(a)
