"""Pins of the oracle's light-geometry gradients (Sec. 3.3: each light of the
virtual light stage moves with its distance d_j, relative area a_j and
barycentric centre p_j):

* interior term: on an occluder-free scene the render with every sample held
  fixed in the emitter's own parameterisation is smooth in (d, a, p), so the
  interior gradient must equal central finite differences of the oracle's own
  render;
* moving-emitter boundary term: the shadowed irradiance of a point under one
  stage light with an occluder between them, in closed form (Lambert's
  polygon formula on the light triangle minus its intersection with the
  occluder's projection), differentiated by central differences, against the
  oracle's interior + shadow-boundary estimate."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from paper_2101_05356_gb300 import synth

import scenes
from test_oracle_pins import clip_convex, polygon_irradiance


def _stage_light(stage_row, d, a, p0, p1):
    """The light triangle of a stage row for parameters (d, a, p): the
    definition written out (homothetic face, shrunk by sqrt(a) about the
    barycentric point)."""
    C = np.asarray(stage_row[0:3], float)
    A, B, V = (np.asarray(stage_row[k:k + 3], float) for k in (3, 6, 9))
    G = (A + B + V) / 3.0
    P = C + d * (p0 * A + p1 * B + (1.0 - p0 - p1) * V)
    s = math.sqrt(a) * d
    return P + s * (A - G), P + s * (V - G), P + s * (B - G)


def test_stage_lights_match_the_generator():
    """Consistency, not a pin: the oracle's stage lights at the generator's
    parameters are the generator's records (same triangles, area a d^2 F,
    scale d^2 / a), and both equal the definition written out here.  The
    oracle's builder is pinned by the closed-form shadowed irradiance of a
    moving emitter below."""
    sc = synth.make_scene("tiny", light_stage="ico")
    for j in range(sc.n_lights):
        t0, t1, t2 = _stage_light(sc.stage[j], 3.0, 0.25, 1 / 3, 1 / 3)
        rec = sc.lights[j]
        assert np.allclose(t0, rec[1:4], atol=1e-5)
        assert np.allclose(t1 - t0, rec[4:7], atol=1e-5) and np.allclose(t2 - t0, rec[7:10], atol=1e-5)
    pr = synth.random_params(sc, 1)
    img_rec = oracle.render(sc, pr)
    img_geo = oracle.render(sc, synth.with_stage_geometry(sc, pr))
    assert np.allclose(img_rec, img_geo, rtol=1e-5, atol=1e-8)


def _flat_scene():
    """One triangle facing the camera under the icosahedral stage: nothing can
    shadow anything."""
    sc0 = synth.make_scene("tiny", light_stage="ico")
    tri = [[-0.9, -0.7, -4.0], [0.9, -0.6, -4.1], [0.0, 0.9, -3.9]]
    sc, pr = scenes.make(tri, [[0, 1, 2]], np.zeros((1, 3, 3)), sc0.lights, width=12, height=12, spp=2)
    sc = dataclasses.replace(sc, stage=sc0.stage, light_d=sc0.light_d, light_a=sc0.light_a, fov_deg=60.0)
    pr.focal[:] = 10.0
    pr.light_i = np.random.default_rng(3).uniform(0.5, 1.5, (sc.n_lights, 3)).astype(np.float32)
    return sc, synth.with_stage_geometry(sc, pr, seed=4)


@pytest.mark.parametrize("field", ["light_d", "light_a", "light_p"])
def test_interior_light_geometry_gradient_matches_fixed_sample_fd(field):
    sc, pr = _flat_scene()
    adj = np.random.default_rng(5).uniform(0.2, 1.0, (12, 12, 3))
    g = oracle.grad(sc, pr, adj, terms=oracle.TERM_INTERIOR)[field]
    base = np.asarray(getattr(pr, field), np.float64)
    flat = base.reshape(-1)
    checked = 0
    for idx in np.argsort(-np.abs(g.reshape(-1)))[:6]:        # the lights that matter most
        h = 1e-3
        qp, qm = pr.copy(), pr.copy()
        getattr(qp, field).reshape(-1)[idx] = flat[idx] + h
        getattr(qm, field).reshape(-1)[idx] = flat[idx] - h
        hp = float(getattr(qp, field).reshape(-1)[idx]) - flat[idx]
        hm = flat[idx] - float(getattr(qm, field).reshape(-1)[idx])
        fd = (np.sum(adj * oracle.render(sc, qp)) - np.sum(adj * oracle.render(sc, qm))) / (hp + hm)
        assert fd == pytest.approx(g.reshape(-1)[idx], rel=2e-4, abs=1e-9), (field, idx)
        checked += abs(fd) > 1e-6
    assert checked >= 3


def _boundary_setup():
    # one stage light in the plane z = d above the shading point y = 0 (normal +z)
    stage = np.array([[0, 0, 0, -0.6, -0.5, 1.0, 0.7, -0.4, 1.0, 0.0, 0.7, 1.0]], np.float32)
    theta = np.array([2.0, 0.5, 0.3, 0.35])                 # d, a, p0, p1
    t0, t1, t2 = _stage_light(stage[0], *theta)
    rec = scenes.quad_light(t0, t1 - t0, t2 - t0, synth.LIGHT_TRI)
    occ = [[-0.3, -0.35, 1.0], [0.45, -0.2, 1.0], [0.0, 0.4, 1.0]]
    sc, pr = scenes.make(occ, [[0, 1, 2]], np.zeros((1, 3, 3)), [rec], light_i=[(1, 1, 1)])
    sc = dataclasses.replace(sc, stage=stage, light_d=np.array([theta[0]], np.float32),
                             light_a=np.array([theta[1]], np.float32))
    pr.light_d = np.array([theta[0]], np.float32)
    pr.light_a = np.array([theta[1]], np.float32)
    pr.light_p = np.array([theta[2:]], np.float32)
    return sc, pr, stage, np.array(occ), theta


def _shadowed_value(stage, occ, theta):
    """White Lambertian point at 0 (normal +z): (d^2 / a) / pi times Lambert's
    integral over the light triangle minus the occluder's shadow on it."""
    t = _stage_light(stage[0], *theta)
    zc = t[0][2]                                   # the light plane is z = const
    tri = [(p[0], p[1]) for p in t]
    if (tri[1][0] - tri[0][0]) * (tri[2][1] - tri[0][1]) - (tri[1][1] - tri[0][1]) * (tri[2][0] - tri[0][0]) < 0:
        tri = tri[::-1]
    shadow = [(zc * p[0] / p[2], zc * p[1] / p[2]) for p in occ]
    if (shadow[1][0] - shadow[0][0]) * (shadow[2][1] - shadow[0][1]) - \
            (shadow[1][1] - shadow[0][1]) * (shadow[2][0] - shadow[0][0]) < 0:
        shadow = shadow[::-1]
    hole = clip_convex(shadow, tri)
    n = np.array([0, 0, 1.0])
    E = polygon_irradiance([(x, y, zc) for x, y in tri], np.zeros(3), n)
    if len(hole) >= 3:
        E -= polygon_irradiance([(x, y, zc) for x, y in hole], np.zeros(3), n)
    return theta[0] ** 2 / theta[1] * E / math.pi


def test_moving_emitter_boundary_matches_closed_form():
    sc, pr, stage, occ, theta = _boundary_setup()
    val, _, lg = oracle.point_light_grad(sc, pr, np.zeros(3), np.array([0, 0, 1.0]), 1500000)
    assert val[0] == pytest.approx(_shadowed_value(stage, occ, theta), rel=5e-3)
    h = 1e-5
    for q in range(4):
        e = np.zeros(4)
        e[q] = h
        fd = (_shadowed_value(stage, occ, theta + e) - _shadowed_value(stage, occ, theta - e)) / (2 * h)
        assert abs(fd) > 1e-3
        assert lg[0, q] == pytest.approx(fd, rel=2.5e-2), (q, lg[0, q], fd)
