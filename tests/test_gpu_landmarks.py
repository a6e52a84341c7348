"""Sparse landmark loss (Sec. 4, Eq. landmark) on the GPU against the FP64
oracle: projections, energy and gradients (coefficients, Euler angles,
translation, focal), accumulation into existing gradients, and the
landmark-only pose/expression initialisation that precedes Stage I."""
import numpy as np
import pytest

from oracle import landmarks as olm
from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name", ["c1", "c2"])
def test_landmark_loss_matches_oracle(name):
    from paper_2101_05356_gb300 import facert
    sc = synth.make_scene(name)
    r = facert.Renderer(sc)
    pr = synth.random_params(sc, 7)
    idx = sc.landmarks
    z = olm.project(sc, synth.random_params(sc, 8), idx, sc.width, sc.height).astype(np.float32)
    dp = r.device_params(pr)
    g = r.zero_grads(dp)
    for k in g:                                  # gradients are added into
        g[k].fill_(0.5)
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    proj = torch.zeros((len(idx), 2), device="cuda")
    w = 0.75
    facert.fr_landmark_loss(r.ctx, dp, sc.width, sc.height, torch.as_tensor(z).cuda(), w, loss, g, proj)
    torch.cuda.synchronize()
    assert np.allclose(proj.cpu().numpy(), olm.project(sc, pr, idx, sc.width, sc.height), rtol=0, atol=1e-3)
    e = olm.energy(sc, pr, idx, z, sc.width, sc.height)
    assert loss.item() == pytest.approx(w * e, rel=1e-9)
    go = olm.grad(sc, pr, idx, z, sc.width, sc.height)
    for k in ("coef", "rot", "trans", "focal"):
        got = g[k].cpu().numpy().astype(np.float64) - 0.5
        want = w * go[k]
        assert np.allclose(got, want, rtol=1e-5, atol=1e-6 * np.abs(want).max()), k
    # untouched groups stay as they were
    assert torch.all(g["light_i"] == 0.5) and torch.all(g["diffuse"] == 0.5)


def test_landmark_initialisation_fits_pose_and_expression():
    from paper_2101_05356_gb300 import facert, optim
    sc = synth.make_scene("c2")
    r = facert.Renderer(sc)
    gt = synth.random_params(sc, 11)
    z = olm.project(sc, gt, sc.landmarks, sc.width, sc.height)
    tgt = r.forward(r.device_params(gt), iteration=10 ** 6)
    rec = optim.Reconstruction(r, tgt, synth.init_params(sc), schedule=optim.Schedule(stage1=2, stage2=0, init=40),
                               landmarks=z)
    e0 = olm.energy(sc, synth.init_params(sc), sc.landmarks, z, sc.width, sc.height)
    seen = []
    while rec.stage == 0:
        rec.step()
        seen.append(float(rec.land_loss.item()))
    assert seen[0] == pytest.approx(e0, rel=1e-6)
    assert seen[-1] < 0.3 * seen[0]
    # Stage I adds the photometric term and keeps alpha_1 E_land
    rec.step()
    assert rec.stage == 1 and float(rec.loss.item()) > 0.0 and float(rec.land_loss.item()) > 0.0
    assert r.status() == 0
