"""Parity at full size, on outputs the oracle can compute one by one:
per-sample records and radiance at sampled pixels, and the gradient of an
adjoint image that is non-zero on a few pixels only (all terms).  Two
workloads: the paper-scale face (35,709 vertices / 70,789 triangles, K = 144,
256 x 256, 16 spp, 40 lights, 512^2 textures) in the launch configuration the
benchmark times, and the large one (50,002 vertices / 100,000 triangles,
K = 20, 1024 x 1024, 64 spp, 80 lights, 2048^2 textures)."""
import numpy as np
import pytest

import oracle
from paper_2101_05356_gb300 import synth

from tests.parity import compare_grads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


# (config, pixels on the face, pixels anywhere) for the radiance check
SAMPLES = {"c2": (32, 16), "c5": (16, 8)}


@pytest.fixture(scope="module", params=["c2", "c5"])
def c2(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene(request.param)
    pr = synth.random_params(sc, 4)
    r = facert.Renderer(sc, edge_spp=1)
    yield sc, pr, r
    r.close()
    torch.cuda.empty_cache()


def test_records_and_radiance_at_sampled_pixels(c2):
    sc, pr, r = c2
    dp = r.device_params(pr)
    img, tri, mask = r.records(dp, iteration=7)
    rng = np.random.default_rng(0)
    # half the sample on the face, half anywhere
    tri_np = tri.cpu().numpy().reshape(-1, sc.spp)
    on_face = np.nonzero((tri_np >= 0).any(axis=1))[0]
    n_face, n_any = SAMPLES["c5" if sc.width > 512 else "c2"]
    pix = np.unique(np.concatenate([rng.choice(on_face, n_face, replace=False),
                                    rng.choice(sc.width * sc.height, n_any, replace=False)])).astype(np.int32)
    oi, ot, om = oracle.render(sc, pr, iteration=7, pixels=pix, records=True)
    ot = ot.reshape(-1, sc.spp)[pix]
    om = om.reshape(-1, sc.spp, 2)[pix]
    gt = tri_np[pix]
    gm = mask.cpu().numpy().view(np.uint64).reshape(-1, sc.spp, 2)[pix]
    agree = (gt == ot) & (gm == om).all(axis=2)        # both visibility words (lights 0..63, 64..127)
    assert np.mean(~agree) <= 1e-4, int(np.sum(~agree))
    ok = agree.all(axis=1)
    g = img.cpu().numpy().reshape(-1, 3)[pix]
    o = oi.reshape(-1, 3)[pix]
    scale = 1e-2 * max(o.mean(), 1e-6)
    err = np.abs(g - o) / np.maximum(np.abs(o), scale)
    assert np.max(err[ok]) <= 1e-4, float(np.max(err[ok]))


def test_gradients_of_a_sparse_adjoint_image(c2):
    sc, pr, r = c2
    from paper_2101_05356_gb300 import facert
    dp = r.device_params(pr)
    E = r.n_edges
    # the ordered silhouette lists must agree for the edge samples to match
    prim = torch.empty(E, dtype=torch.int32, device="cuda")
    npr = torch.empty(1, dtype=torch.int32, device="cuda")
    facert.fr_debug_silhouettes(r.ctx, dp, prim, npr, None, None)
    po, _ = oracle.silhouettes(sc, pr)
    assert np.array_equal(prim.cpu().numpy()[: int(npr.item())], po)
    img, tri, mask = r.records(dp, iteration=3)
    tri_np = tri.cpu().numpy().reshape(-1, sc.spp)
    on_face = np.nonzero((tri_np >= 0).all(axis=1))[0]
    pix = np.random.default_rng(1).choice(on_face, 12, replace=False)
    # keep pixels whose records agree with the oracle
    _, ot, om = oracle.render(sc, pr, iteration=3, pixels=pix.astype(np.int32), records=True)
    gm = mask.cpu().numpy().view(np.uint64).reshape(-1, sc.spp, 2)
    keep = [p for p in pix if np.array_equal(tri_np[p], ot.reshape(-1, sc.spp)[p])
            and np.array_equal(gm[p], om.reshape(-1, sc.spp, 2)[p])]
    assert len(keep) >= 10
    adj = np.zeros((sc.height, sc.width, 3))
    adj.reshape(-1, 3)[keep] = np.random.default_rng(2).uniform(0.3, 1.0, (len(keep), 3))
    adj32 = adj.astype(np.float32)
    gg = r.backward(dp, torch.as_tensor(adj32).cuda(), iteration=3)
    go = oracle.grad(sc, pr, adj32.astype(np.float64), iteration=3, edge_spp=1)
    compare_grads(gg, go, ("coef", "rot", "trans", "focal", "light_i", "diffuse", "specular", "roughness"), 1e-3)
