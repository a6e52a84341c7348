"""Pins of the oracle's environment-map emitters (Sec. 7, environment map vs
light stage) against results fixed by the mathematics, not by the oracle:
the furnace identity, the cosine-weighted solid angle of single texels
(numerical quadrature), homogeneity of the image in the map's radiance, and
the shadow-boundary term on the sphere of directions against Lambert's
polygon formula."""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
import scenes
from paper_2101_05356_gb300 import synth

from test_oracle_pins import polygon_irradiance


def _env_scene(records, me, env, verts=None, faces=None, basis=None):
    verts = scenes.FAR_TRIANGLE if verts is None else verts
    faces = [[0, 1, 2]] if faces is None else faces
    basis = np.zeros((1, len(verts), 3)) if basis is None else basis
    recs = np.asarray(records, np.float32).reshape(-1, 11)
    sc, pr = scenes.make(verts, faces, basis, recs)
    sc = dataclasses.replace(sc, env_size=me)
    pr.env = np.asarray(env, np.float32)
    return sc, pr


def _block(i0, i1, j0, j1):
    r = np.zeros(11, np.float32)
    r[:5] = (synth.LIGHT_ENV, i0, i1, j0, j1)
    return r


def test_env_furnace_white_lambert():
    """A constant map L over the whole sphere lights an unoccluded white
    Lambertian point with L * (1/pi) * int_{n.w > 0} n.w dw = L."""
    me = 8
    recs = [_block(0, 4, 0, 4), _block(0, 4, 4, 8), _block(4, 8, 0, 4), _block(4, 8, 4, 8)]
    env = np.full((me, me, 3), 1.0)
    env[..., 1] = 0.5
    sc, pr = _env_scene(recs, me, env)
    n = np.array([0.3, -0.5, 0.8])
    n /= np.linalg.norm(n)
    val, _ = oracle.point_light_grad(sc, pr, np.zeros(3), n, 200000)
    assert val[0] == pytest.approx(1.0, rel=1e-2)
    assert val[1] == pytest.approx(0.5, rel=1e-2)


def _texel_cos_integral(i, j, me, n):
    """int over texel (i, j) of max(0, n . w) dw, w = (sin t sin p, cos t, sin t cos p)."""
    def f(p, t):
        w = np.array([math.sin(t) * math.sin(p), math.cos(t), math.sin(t) * math.cos(p)])
        return max(0.0, float(n @ w)) * math.sin(t)
    v, _ = integrate.dblquad(f, math.pi * i / me, math.pi * (i + 1) / me,
                             2 * math.pi * j / me, 2 * math.pi * (j + 1) / me, epsabs=1e-12, epsrel=1e-9)
    return v


@pytest.mark.parametrize("i,j,me", [(1, 0, 8), (3, 1, 8), (2, 6, 8), (5, 7, 8), (3, 4, 8), (0, 1, 8), (7, 0, 8),
                                    (4, 1, 12), (0, 11, 12)])
def test_env_single_texel_orientation(i, j, me):
    """One texel as its own block: the oracle's estimate of (1/pi) int n.w dw
    over the texel matches quadrature, which fixes the polar axis (+y), the
    azimuth origin (+z) and direction (towards +x) and the texel's solid angle,
    also at the poles and for a map side that is not a power of two.  Texels
    (3, 4) and (7, 0) face away from n (zero)."""
    env = np.zeros((me, me, 3))
    env[i, j] = (2.0, 1.0, 0.5)
    sc, pr = _env_scene([_block(i, i + 1, j, j + 1)], me, env)
    n = np.array([0.35, 0.45, 0.82])
    n /= np.linalg.norm(n)
    val, _ = oracle.point_light_grad(sc, pr, np.zeros(3), n, 60000)
    want = _texel_cos_integral(i, j, me, n) / math.pi
    if want == 0.0:
        assert val[0] == 0.0
    else:
        assert val[0] == pytest.approx(2.0 * want, rel=1e-2)
        assert val[2] == pytest.approx(0.5 * want, rel=1e-2)


def test_env_block_sampling_matches_quadrature():
    """A 3 x 2 block with different texel radiances: the estimator (texel
    chosen uniformly, direction uniform inside it, weight R C Omega) gives
    the sum of the texels' quadratures."""
    me = 8
    rng = np.random.default_rng(4)
    env = np.zeros((me, me, 3))
    env[2:5, 1:3] = rng.uniform(0.5, 2.0, size=(3, 2, 3))
    sc, pr = _env_scene([_block(2, 5, 1, 3)], me, env)
    n = np.array([0.6, 0.2, 0.77])
    n /= np.linalg.norm(n)
    val, _ = oracle.point_light_grad(sc, pr, np.zeros(3), n, 400000)
    want = np.zeros(3)
    for i in range(2, 5):
        for j in range(1, 3):
            want += env[i, j] * _texel_cos_integral(i, j, me, n) / math.pi
    np.testing.assert_allclose(val, want, rtol=1e-2)


def test_env_image_is_homogeneous_in_the_map():
    """With environment blocks only, the image is linear and homogeneous in
    the map's radiance, so sum(g_env * env) = sum(adjoint * image) for the
    interior gradient of the same samples (Euler's identity); this pins the
    texel each sample's radiance gradient lands on and its weight."""
    sc = synth.make_scene("tiny", env=(8, 2))
    pr = synth.random_params(sc)
    img = oracle.render(sc, pr)
    adj = np.random.default_rng(3).normal(size=img.shape)
    g = oracle.grad(sc, pr, adj, terms=oracle.TERM_INTERIOR)
    lhs = float(np.sum(g["env"] * pr.env))
    rhs = float(np.sum(adj * img))
    assert abs(rhs) > 1e-3
    assert lhs == pytest.approx(rhs, rel=1e-9)
    assert np.all(g["light_i"] == 0.0)


def _occluder_scene(coef):
    """A triangle in the plane x = 1 in front of the point y = 0 (normal +x),
    inside one environment block of constant radiance around +x."""
    occ = np.array([[1.0, -0.3, -0.2], [1.0, 0.35, -0.1], [1.0, 0.05, 0.4]])
    basis = np.zeros((2, 3, 3))
    basis[0, 1, 2] = 1.0            # vertex 1 along z (in its plane)
    basis[1, 2, 0] = 1.0            # vertex 2 along x (out of the plane)
    me = 8
    env = np.zeros((me, me, 3))
    env[2:6, 1:3] = (1.5, 1.0, 0.5)   # theta in [pi/4, 3pi/4], phi in [pi/4, 3pi/4]
    sc, pr = _env_scene([_block(2, 6, 1, 3)], me, env, occ, [[0, 1, 2]], basis)
    pr.coef = np.asarray(coef, np.float32)
    return sc, pr, occ, basis


def _occluded_value(coef):
    """(L / pi) [int_block n.w dw - E(occluder)] with E Lambert's polygon
    formula, for an occluder whose directions lie inside the block."""
    _, _, occ, basis = _occluder_scene(coef)
    v = occ + np.tensordot(np.asarray(coef, float), basis, axes=1)
    n = np.array([1.0, 0.0, 0.0])
    # int_{pi/4}^{3pi/4} sin^2 t dt * int_{pi/4}^{3pi/4} sin p dp  (n.w = sin t sin p)
    block = (math.pi / 4 + 0.5) * math.sqrt(2.0)
    return 1.5 * (block - polygon_irradiance(list(v), np.zeros(3), n, 1.0)) / math.pi


def test_env_shadow_boundary_matches_lambert_formula():
    coef = np.array([0.04, 0.1])
    sc, pr, _, _ = _occluder_scene(coef)
    val, g = oracle.point_light_grad(sc, pr, np.zeros(3), np.array([1.0, 0, 0]), 1500000)
    assert val[0] == pytest.approx(_occluded_value(coef), rel=5e-3)
    h = 1e-5
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (_occluded_value(coef + e) - _occluded_value(coef - e)) / (2 * h)
        assert abs(fd) > 1e-3
        assert g[k] == pytest.approx(fd, rel=2.5e-2), (k, g[k], fd)


def test_env_shadow_candidates_are_conservative():
    """Every edge that is a silhouette for some direction of a block (sampled
    densely) is in that block's candidate list, and the exact range of n . w
    over the block still culls edges."""
    sc = synth.make_scene("tiny", env=(8, 2))
    pr = synth.random_params(sc)
    _, lists = oracle.silhouettes(sc, pr)
    v, _ = oracle.geometry(sc, pr)
    ev, ef = oracle.edges(sc)
    f = sc.faces
    nf = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    rng = np.random.default_rng(5)
    me = sc.env_size
    for j, rec in enumerate(sc.lights):
        i0, i1, j0, j1 = (int(x) for x in rec[1:5])
        y = rng.uniform(math.cos(math.pi * i1 / me), math.cos(math.pi * i0 / me), 3000)
        ph = rng.uniform(2 * math.pi * j0 / me, 2 * math.pi * j1 / me, 3000)
        s = np.sqrt(1.0 - y * y)
        w = np.stack([s * np.sin(ph), y, s * np.cos(ph)], 1)
        side = np.sign(nf @ w.T)
        inner = ef[:, 1] >= 0
        sil = np.ones(len(ev), bool)
        sil[inner] = np.any(side[ef[inner, 0]] != side[ef[inner, 1]], axis=1)
        cand = np.zeros(len(ev), bool)
        cand[lists[j]] = True
        assert np.all(cand[sil]), j
        assert cand.sum() < len(ev), j
