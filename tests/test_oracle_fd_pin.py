"""End-to-end pin of the oracle's gradient estimator: the derivative of the
expected image is the interior term plus the primary-visibility and
shadow-boundary terms (Sec. 4, "Edge Sampling"), so their sum must agree with
central finite differences of the rendered image, taken with common random
numbers, within the combined Monte Carlo error, while the interior term alone
must not wherever a visibility boundary moves.

Scenes: the shadow box (shape coefficients move the occluder and a floor
corner: primary silhouettes and soft shadow boundaries) and the same box lit by
a two-light virtual light stage (Sec. 3.3), whose distance, relative area and
barycentric centre move the shadow boundaries across the floor (the
moving-emitter term).  All seeds are fixed, so the outcome is deterministic."""
import dataclasses

import numpy as np
import pytest

import oracle
import scenes

N_ITER = 24


def _z_scores(make, fields, h):
    sc, pr = make()
    sc = dataclasses.replace(sc, spp=64)
    yy, xx = np.mgrid[0:sc.height, 0:sc.width]
    w = 1.0 + 0.5 * np.sin(xx / 3.0)[..., None] * np.cos(yy / 4.0)[..., None] * np.array([1.0, 0.7, -0.4])
    fd = {f: [] for f in fields}
    full = {f: [] for f in fields}
    interior = {f: [] for f in fields}
    for it in range(N_ITER):
        g_all = oracle.grad(sc, pr, w, iteration=1000 + it, edge_spp=4)
        g_int = oracle.grad(sc, pr, w, iteration=1000 + it, terms=oracle.TERM_INTERIOR)
        for name, idx in fields:
            full[(name, idx)].append(np.asarray(g_all[name]).flat[idx])
            interior[(name, idx)].append(np.asarray(g_int[name]).flat[idx])
            pp, pm = pr.copy(), pr.copy()
            getattr(pp, name).flat[idx] += h
            getattr(pm, name).flat[idx] -= h
            d = oracle.render(sc, pp, iteration=it) - oracle.render(sc, pm, iteration=it)
            fd[(name, idx)].append(float(np.sum(w * d)) / (2.0 * h))

    def se(a):
        return np.std(a, ddof=1) / np.sqrt(len(a))

    out = {}
    for k in fields:
        f, g, i = np.array(fd[k]), np.array(full[k]), np.array(interior[k])
        out[k] = ((g.mean() - f.mean()) / np.hypot(se(g), se(f)),
                  (i.mean() - f.mean()) / np.hypot(se(i), se(f)))
    return out


@pytest.mark.parametrize("case", ["shape", "light_stage"])
def test_full_gradient_matches_finite_differences(case):
    if case == "shape":
        z = _z_scores(scenes.shadow_box, [("coef", k) for k in range(4)], 5e-3)
        boundary = [("coef", 0), ("coef", 3)]
    else:
        z = _z_scores(scenes.stage_box, [("light_d", 0), ("light_d", 1), ("light_a", 0), ("light_a", 1),
                                         ("light_p", 0), ("light_p", 3)], 1e-2)
        boundary = [("light_d", 0), ("light_d", 1)]
    for k, (z_full, _) in z.items():
        assert abs(z_full) <= 3.5, (k, z_full)
    for k in boundary:                      # the boundary terms matter here
        assert abs(z[k][1]) > 6.0, (k, z[k][1])
