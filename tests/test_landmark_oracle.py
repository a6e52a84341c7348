"""Pins of the landmark-loss oracle (Sec. 4, Eq. landmark): the projection in
closed form, its agreement with the oracle renderer's camera rays, the energy
of known offsets, and the hand gradient against central finite differences."""
import numpy as np
import pytest

import oracle
from oracle import landmarks as olm
from paper_2101_05356_gb300 import synth


def test_projection_closed_form():
    """R = I, T = 0: v' = v, so x = W/2 + f v_x / (-v_z), y = H/2 - f v_y / (-v_z)."""
    sc = synth.make_scene("tiny")
    sc = synth.Scene(**{**sc.__dict__, "mean": sc.mean - np.array([0, 0, 4.5], np.float32)})
    pr = synth.init_params(sc)
    pr.rot[:] = 0.0
    pr.trans[:] = 0.0
    pr.focal[:] = 50.0
    idx = np.array([0, 5, 17], np.int32)
    v = sc.mean[idx].astype(np.float64)
    want = np.stack([12 + 50 * v[:, 0] / -v[:, 2], 12 - 50 * v[:, 1] / -v[:, 2]], axis=1)
    assert np.allclose(olm.project(sc, pr, idx, 24, 24), want, rtol=0, atol=1e-9)


def test_projection_lies_on_the_camera_ray():
    """The oracle renderer's camera ray through each projected landmark passes
    through the landmark vertex (direction parallel to the camera-space vertex),
    and its closest hit is that vertex for the landmarks the camera sees."""
    sc = synth.make_scene("c1")
    pr = synth.random_params(sc, 3)
    idx = sc.landmarks
    p = olm.project(sc, pr, idx, sc.width, sc.height)
    f = float(pr.focal[0])
    dirs = np.stack([(p[:, 0] - sc.width / 2) / f, -(p[:, 1] - sc.height / 2) / f, -np.ones(len(idx))], axis=1)
    tri, t = oracle.closest_hit(sc, pr, np.zeros_like(dirs), dirs)
    vcam, _ = oracle.geometry(sc, pr)
    hit = dirs * t[:, None]
    d = np.linalg.norm(hit - vcam[idx], axis=1)
    # the others are hidden behind the nose or brows, or graze the silhouette
    on_vertex = (tri >= 0) & (d < 1e-9)
    assert on_vertex.mean() > 0.7
    # the ray direction is parallel to the camera-space vertex for every landmark
    cosang = np.sum(dirs * vcam[idx], axis=1) / np.linalg.norm(dirs, axis=1) / np.linalg.norm(vcam[idx], axis=1)
    assert np.all(cosang > 1 - 1e-12)


def test_energy_of_known_offsets():
    sc = synth.make_scene("c1")
    pr = synth.random_params(sc, 4)
    idx = sc.landmarks
    p = olm.project(sc, pr, idx, sc.width, sc.height)
    assert olm.energy(sc, pr, idx, p, sc.width, sc.height) == pytest.approx(0.0, abs=1e-18)
    assert olm.energy(sc, pr, idx, p + np.array([3.0, -4.0]), sc.width, sc.height) == pytest.approx(
        25.0 * len(idx), rel=1e-12)


@pytest.mark.parametrize("field", ["coef", "rot", "trans", "focal"])
def test_gradient_matches_finite_differences(field):
    sc = synth.make_scene("c1")
    pr = synth.random_params(sc, 5)
    idx = sc.landmarks
    z = olm.project(sc, synth.random_params(sc, 6), idx, sc.width, sc.height)
    g = olm.grad(sc, pr, idx, z, sc.width, sc.height)[field]
    base = np.asarray(getattr(pr, field), np.float64)
    h = 1e-6 * max(1.0, float(np.abs(base).max()))
    for k in range(min(base.size, 6)):
        qp, qm = pr.copy(), pr.copy()
        getattr(qp, field)[k] = base[k] + h
        getattr(qm, field)[k] = base[k] - h
        # parameters are float32 in Params: use the values actually stored
        hp = float(getattr(qp, field)[k]) - base[k]
        hm = base[k] - float(getattr(qm, field)[k])
        fd = (olm.energy(sc, qp, idx, z, sc.width, sc.height) - olm.energy(sc, qm, idx, z, sc.width, sc.height)) / (hp + hm)
        assert fd == pytest.approx(g[k], rel=2e-3, abs=1e-3 * np.abs(g).max())
