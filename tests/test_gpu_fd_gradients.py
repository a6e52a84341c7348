"""The autograd.Function's gradients (interior + primary-visibility +
shadow-boundary terms + the boundary term of the specular lobe's cutoff
inside triangles, through the hand-written adjoint) against central
finite differences of the GPU's own rendered image with common random
numbers: the derivative of the expected image, so the two must agree within
their combined Monte Carlo error over repeated Philox iterations, while the
interior term alone must not where a visibility boundary moves.  Geometry,
pose and camera on the 2,562-vertex face; the virtual light stage's distance,
relative area and barycentric centre on the stage-lit shadow box."""
import dataclasses

import numpy as np
import pytest

import scenes
from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_ITER = 48
_MEANS = {}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _weights(sc):
    yy, xx = np.mgrid[0:sc.height, 0:sc.width]
    w = 1.0 + 0.5 * np.sin(xx / 3.0)[..., None] * np.cos(yy / 4.0)[..., None] * np.array([1.0, 0.7, -0.4])
    return torch.as_tensor(w, dtype=torch.float64).cuda()


def _z_scores(sc, pr, fields):
    from paper_2101_05356_gb300 import autograd, facert
    W = _weights(sc)
    out = {}
    for interior_only in (False, True):
        flags = (facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE |
                 facert.FLAG_NO_SPECULAR_EDGE) if interior_only else 0
        r = facert.Renderer(sc, flags=flags)
        dp = r.device_params(pr)
        grads = {f: [] for f in fields}
        fds = {f: [] for f in fields}
        for it in range(N_ITER):
            leaves = {k: v.clone().requires_grad_(True) for k, v in dp.items()}
            img = autograd.render(r, leaves, iteration=500 + it)
            (img.double() * W).sum().backward()
            for (name, idx, h) in fields:
                grads[(name, idx, h)].append(float(leaves[name].grad.reshape(-1)[idx]))
                if interior_only:
                    continue
                vals = []
                for sgn in (1.0, -1.0):
                    q = dict(dp)
                    q[name] = dp[name].clone()
                    q[name].view(-1)[idx] += sgn * h
                    vals.append(float((r.forward(q, iteration=500 + it).double() * W).sum()))
                fds[(name, idx, h)].append((vals[0] - vals[1]) / (2.0 * h))
        assert r.status() == 0
        for f in fields:
            g = np.array(grads[f])
            out.setdefault(f, {})["interior" if interior_only else "full"] = g
            if not interior_only:
                out[f]["fd"] = np.array(fds[f])
        r.close()

    def se(a):
        return np.std(a, ddof=1) / np.sqrt(len(a))

    z = {}
    for f, d in out.items():
        z[f] = ((d["full"].mean() - d["fd"].mean()) / np.hypot(se(d["full"]), se(d["fd"])),
                (d["interior"].mean() - d["fd"].mean()) / np.hypot(se(d["interior"]), se(d["fd"])))
        _MEANS[f] = (d["fd"].mean(), d["full"].mean())
        print("%s[%d]: finite difference %.4g +- %.2g, gradient %.4g +- %.2g, interior only %.4g"
              % (f[0], f[1], d["fd"].mean(), se(d["fd"]), d["full"].mean(), se(d["full"]), d["interior"].mean()))
    return z


@pytest.mark.parametrize("case", ["face", "light_stage"])
def test_autograd_gradient_matches_finite_differences(case):
    if case == "face":
        sc = dataclasses.replace(synth.make_scene("c1"), spp=16)
        pr = synth.random_params(sc, 5, coef_scale=0.5)
        fields = [("coef", k, 5e-3) for k in range(4)] + [("rot", k, 1e-3) for k in range(3)] + \
                 [("trans", k, 2e-3) for k in range(3)] + [("focal", 0, 0.2)]
    else:
        sc, pr = scenes.stage_box()
        sc = dataclasses.replace(sc, spp=64)
        fields = [("light_d", 0, 1e-2), ("light_d", 1, 1e-2), ("light_a", 0, 1e-2), ("light_a", 1, 1e-2),
                  ("light_p", 0, 1e-2), ("light_p", 3, 1e-2)]
    z = _z_scores(sc, pr, fields)
    print(case, {"%s[%d]" % (f[0], f[1]): (round(a, 2), round(b, 2)) for f, (a, b) in z.items()})
    for f, (z_full, _) in z.items():
        assert abs(z_full) <= 3.5, (f, z_full)
    assert max(abs(z_int) for _, z_int in z.values()) > 6.0         # the boundary terms matter here
    if case == "face":
        # zooming moves the curve n_s.o = 0 inside the silhouette's front-facing triangles most (the
        # specular lobe jumps there): with its boundary term the focal-length gradient is within 3%
        f = ("focal", 0, 0.2)
        assert abs(_MEANS[f][1] - _MEANS[f][0]) <= 0.03 * abs(_MEANS[f][0]), _MEANS[f]
