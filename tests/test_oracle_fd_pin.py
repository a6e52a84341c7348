"""End-to-end pin of the oracle's gradient estimator: the derivative of the
expected image is the interior term plus the primary-visibility and
shadow-boundary terms and the boundary term of the specular lobe's cutoff
inside triangles (Sec. 4, "Edge Sampling"), so their sum must agree with
central finite differences of the rendered image, taken with common random
numbers, within the combined Monte Carlo error, while the interior term alone
must not wherever a visibility boundary moves.

Scenes: the shadow box (shape coefficients move the occluder and a floor
corner: primary silhouettes and soft shadow boundaries) and the same box lit by
a two-light virtual light stage (Sec. 3.3), whose distance, relative area and
barycentric centre move the shadow boundaries across the floor (the
moving-emitter term), the same box under an environment map of lights at
infinity (Sec. 7; the boundary term on the sphere of directions), and the
camera (focal length, translation, rotation) on a small smooth face.  All seeds
are fixed, so the outcome is deterministic."""
import dataclasses

import numpy as np
import pytest

import oracle
import scenes

N_ITER = 24


def _z_scores(make, fields, h, spp=64, flags=0, partial=oracle.TERM_INTERIOR):
    """(z of the full gradient, z of the `partial` terms alone) against central
    finite differences, per field."""
    sc, pr = make()
    sc = dataclasses.replace(sc, spp=spp)
    yy, xx = np.mgrid[0:sc.height, 0:sc.width]
    w = 1.0 + 0.5 * np.sin(xx / 3.0)[..., None] * np.cos(yy / 4.0)[..., None] * np.array([1.0, 0.7, -0.4])
    fd = {f: [] for f in fields}
    full = {f: [] for f in fields}
    interior = {f: [] for f in fields}
    for it in range(N_ITER):
        g_all = oracle.grad(sc, pr, w, iteration=1000 + it, edge_spp=4, flags=flags)
        g_int = oracle.grad(sc, pr, w, iteration=1000 + it, terms=partial, flags=flags, edge_spp=4)
        for name, idx in fields:
            full[(name, idx)].append(np.asarray(g_all[name]).flat[idx])
            interior[(name, idx)].append(np.asarray(g_int[name]).flat[idx])
            pp, pm = pr.copy(), pr.copy()
            hh = h[name] if isinstance(h, dict) else h
            getattr(pp, name).flat[idx] += hh
            getattr(pm, name).flat[idx] -= hh
            d = oracle.render(sc, pp, iteration=it, flags=flags) - oracle.render(sc, pm, iteration=it, flags=flags)
            fd[(name, idx)].append(float(np.sum(w * d)) / (2.0 * hh))

    def se(a):
        return np.std(a, ddof=1) / np.sqrt(len(a))

    out = {}
    for k in fields:
        f, g, i = np.array(fd[k]), np.array(full[k]), np.array(interior[k])
        out[k] = ((g.mean() - f.mean()) / np.hypot(se(g), se(f)),
                  (i.mean() - f.mean()) / np.hypot(se(i), se(f)))
    return out


def _small_face():
    from paper_2101_05356_gb300 import synth
    sc = synth.make_scene("tiny")
    return sc, synth.random_params(sc, 5, coef_scale=0.5)


CAMERA = [("focal", 0), ("trans", 0), ("trans", 1), ("trans", 2), ("rot", 0), ("rot", 1)]
CAMERA_H = {"focal": 0.1, "trans": 2e-3, "rot": 1e-3}


def test_camera_gradient_matches_finite_differences():
    """Pose and focal length on a smooth closed face: its silhouette moves in
    the image, and with interpolated shading normals a band of front-facing
    triangles along it has normals turned away from the camera."""
    z = _z_scores(_small_face, CAMERA, CAMERA_H, spp=16)
    for k, (z_full, _) in z.items():
        assert abs(z_full) <= 3.5, (k, z_full)
    assert max(abs(z_int) for _, z_int in z.values()) > 6.0


def test_view_cutoff_reading_is_sampled():
    """Zeroing every contribution where n_s . o <= 0 (the diffuse term too)
    puts a jump on the curve n_s . o = 0 inside those triangles; the boundary
    term on that curve carries it, and without that term alone the
    focal-length gradient misses the finite-difference derivative by many
    standard errors."""
    z = _z_scores(_small_face, [("focal", 0)], CAMERA_H, spp=16, flags=oracle.VIEW_CUTOFF,
                  partial=oracle.TERM_ALL & ~oracle.TERM_SPECULAR)
    assert abs(z[("focal", 0)][0]) <= 3.5, z
    assert abs(z[("focal", 0)][1]) > 5.0, z


@pytest.mark.parametrize("case", ["shape", "light_stage", "environment"])
def test_full_gradient_matches_finite_differences(case):
    if case == "shape":
        z = _z_scores(scenes.shadow_box, [("coef", k) for k in range(4)], 5e-3)
        boundary = [("coef", 0), ("coef", 3)]
    elif case == "environment":
        # lights at infinity (Sec. 7): without the shadow-boundary term on the
        # sphere of directions, the occluder's coefficients miss
        z = _z_scores(scenes.env_box, [("coef", k) for k in range(4)], 5e-3,
                      partial=oracle.TERM_INTERIOR | oracle.TERM_PRIMARY)
        boundary = [("coef", 0), ("coef", 1)]       # 5.4 and 7.2 standard errors off without it
    else:
        z = _z_scores(scenes.stage_box, [("light_d", 0), ("light_d", 1), ("light_a", 0), ("light_a", 1),
                                         ("light_p", 0), ("light_p", 3)], 1e-2)
        boundary = [("light_d", 0), ("light_d", 1)]
    for k, (z_full, _) in z.items():
        assert abs(z_full) <= 3.5, (k, z_full)
    for k in boundary:                      # the boundary terms matter here
        assert abs(z[k][1]) > (5.0 if case == "environment" else 6.0), (k, z[k][1])
