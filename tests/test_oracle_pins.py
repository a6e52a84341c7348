"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself: published
known-answer vectors, closed forms (normalisation integrals, Lambert's polygon
irradiance, exact Smith masking, pixel coverage areas), brute-force geometry
with known answers, exact linearity, and finite differences of the oracle's own
values (which use no derivative code)."""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_2101_05356_gb300 import synth
from tests import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# Philox4x32-10: Random123 known-answer vectors
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        c, k, want = v[0:4], v[4:6], v[6:10]
        got = oracle.philox(k[0], k[1], *c)
        assert [int(x) for x in got] == want


# ---------------------------------------------------------------------------
# Reflectance (App. A)
# ---------------------------------------------------------------------------
def _dir(theta, phi):
    return np.array([math.sin(theta) * math.cos(phi), math.sin(theta) * math.sin(phi),
                     math.cos(theta)])


@pytest.mark.parametrize("flags", [0, oracle.GGX])
@pytest.mark.parametrize("r", [0.3, 0.45, 0.6, 0.9])
def test_D_is_normalised(r, flags):
    """Any microfacet distribution integrates to one against (n.h) (App. A, D)."""
    n = np.array([0.0, 0.0, 1.0])

    def f(theta):
        h = _dir(theta, 0.3)
        return oracle.brdf_terms(n, h, h, r, flags)[0] * math.cos(theta) * math.sin(theta)

    val, _ = integrate.quad(f, 0.0, math.pi / 2, limit=200, epsabs=1e-11)
    assert abs(2.0 * math.pi * val - 1.0) < 1e-6


@pytest.mark.parametrize("r", [0.3, 0.5, 0.8])
def test_G1_matches_exact_smith(r):
    """Walter's rational G1 approximates the exact Smith-Beckmann masking
    2 / (1 + erf(a) + exp(-a^2)/(a sqrt(pi))) with a = 1/(r tan theta)."""
    n = np.array([0.0, 0.0, 1.0])
    worst = 0.0
    for cos_t in np.linspace(0.02, 0.999, 200):
        v = _dir(math.acos(cos_t), 0.7)
        g1 = oracle.brdf_terms(n, v, v, r)[1]
        a = cos_t / (r * math.sqrt(1.0 - cos_t * cos_t))
        exact = 2.0 / (1.0 + special.erf(a) + math.exp(-a * a) / (a * math.sqrt(math.pi)))
        worst = max(worst, abs(g1 - exact))
    assert worst < 4e-3


def test_G1_visibility_step():
    """Delta(h.v / n.v) = 0 kills a view direction below the microfacet."""
    n = np.array([0.0, 0.0, 1.0])
    l = _dir(1.2, 0.0)
    o = _dir(1.4, math.pi)            # grazing on the other side
    terms = oracle.brdf_terms(n, l, o, 0.5)
    h = (l + o) / np.linalg.norm(l + o)
    assert (h @ o) / (n @ o) > 0 and terms[1] > 0     # sanity: both visible here
    o2 = np.array([0.0, -0.2, -0.98])
    o2 /= np.linalg.norm(o2)
    assert oracle.brdf_terms(n, l, o2, 0.5)[1] == 0.0


def test_schlick_weight():
    n = np.array([0.0, 0.0, 1.0])
    l = o = _dir(0.4, 0.1)
    assert oracle.brdf_terms(n, l, o, 0.5)[3] == pytest.approx(0.0, abs=1e-15)
    # o.h = 1/2: l and o 120 degrees apart, h bisects them
    l = _dir(math.pi / 3, 0.0)
    o = _dir(math.pi / 3, math.pi)
    w = oracle.brdf_terms(n, l, o, 0.5)[3]
    assert w == pytest.approx(0.5 ** 5, rel=1e-12)
    assert oracle.brdf_terms(n, l, o, 0.5, oracle.SCHLICK_LINEAR)[3] == pytest.approx(0.5, rel=1e-12)


@pytest.mark.parametrize("r", [0.3, 0.6])
def test_specular_peak_normal_incidence(r):
    """n = l = o: h = n, D = 1/(pi r), G = 1, F = s, so f_s = s / (4 pi r)."""
    n = np.array([0.0, 0.0, 1.0])
    s = np.array([0.05, 0.3, 1.0])
    f = oracle.brdf(n, n, n, np.zeros(3), s, r)
    assert np.allclose(f, s / (4.0 * math.pi * r), rtol=1e-12)


def test_lambert_term_and_reciprocity():
    n = np.array([0.0, 0.0, 1.0])
    c = np.array([0.2, 0.5, 0.8])
    l = _dir(0.7, 0.4)
    # l = o makes o.h = 1, so F = s = 0 and only c/pi remains
    assert np.allclose(oracle.brdf(n, l, l, c, np.zeros(3), 0.4), c / math.pi, rtol=1e-13)
    rng = np.random.default_rng(3)
    for _ in range(50):
        l = _dir(rng.uniform(0, 1.5), rng.uniform(0, 6.28))
        o = _dir(rng.uniform(0, 1.5), rng.uniform(0, 6.28))
        s = rng.uniform(0, 1, 3)
        r = rng.uniform(0.2, 0.9)
        a = oracle.brdf(n, l, o, c, s, r)
        b = oracle.brdf(n, o, l, c, s, r)
        assert np.allclose(a, b, rtol=1e-12)                  # Helmholtz reciprocity
    assert np.all(oracle.brdf(n, _dir(1.7, 0), l, c, s, 0.5) == 0.0)   # below the horizon


def _specular_albedo(o, r, flags, m=100):
    n = np.array([0.0, 0.0, 1.0])
    tot = 0.0
    for i in range(m):
        th = (i + 0.5) / m * (math.pi / 2)
        for j in range(2 * m):
            ph = (j + 0.5) / (2 * m) * 2 * math.pi
            f = oracle.brdf(n, _dir(th, ph), o, np.zeros(3), np.ones(3), r, flags)[0]
            tot += f * math.cos(th) * math.sin(th)
    return tot * (math.pi / 2 / m) * (2 * math.pi / (2 * m))


@pytest.mark.parametrize("r", [0.3, 0.6])
def test_specular_directional_albedo_bounded(r):
    """Energy (s = 1): at normal view G1(o) = 1 and the normalised D bound the
    albedo by one; the GGX mode (matched D and G) stays below one at every
    angle.  The paper's Blinn-Phong D with Walter's G1 on the same r is not
    energy conserving at grazing view (albedo ~1.13 at 75 degrees), which is a
    property of the printed model, so no bound is asserted there."""
    assert 0.3 < _specular_albedo(_dir(0.0, 0.0), r, 0) <= 1.0
    for th_o in (0.0, 0.8, 1.3):
        assert 0.3 < _specular_albedo(_dir(th_o, 0.0), r, oracle.GGX) <= 1.0


# ---------------------------------------------------------------------------
# Emitters: Lambert's polygon formula and the disk closed form (Sec. 3.3)
# ---------------------------------------------------------------------------
def polygon_irradiance(poly, y, n, radiance=1.0):
    """Lambert's formula: E = L/2 |sum_k Theta_k (n . unit(p_k x p_k+1))|."""
    p = [np.asarray(q, float) - y for q in poly]
    tot = 0.0
    for k in range(len(p)):
        a, b = p[k], p[(k + 1) % len(p)]
        cr = np.cross(a, b)
        ang = math.acos(np.clip(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)), -1, 1))
        tot += ang * (n @ cr) / np.linalg.norm(cr)
    return 0.5 * radiance * abs(tot)


def test_polygon_formula_matches_disk_closed_form():
    """The test's own closed forms agree: a 4000-gon vs pi L R^2/(R^2 + h^2)."""
    R, h = 0.7, 1.3
    poly = [(R * math.cos(t), R * math.sin(t), h) for t in np.linspace(0, 2 * math.pi, 4000, endpoint=False)]
    E = polygon_irradiance(poly, np.zeros(3), np.array([0, 0, 1.0]))
    assert E == pytest.approx(math.pi * R * R / (R * R + h * h), rel=1e-6)


def _point_value(light_rec, y, n, intensity=(1.0, 0.8, 0.5), samples=400000):
    sc, pr = scenes.make(scenes.FAR_TRIANGLE, [[0, 1, 2]], np.zeros((1, 3, 3)), [light_rec],
                         light_i=[intensity])
    val, _ = oracle.point_light_grad(sc, pr, y, n, samples)
    return val


@pytest.mark.parametrize("case", range(3))
def test_quad_irradiance_matches_polygon_formula(case):
    rng = np.random.default_rng(10 + case)
    c = np.array([0.3, -0.2, 1.5]) + rng.uniform(-0.3, 0.3, 3)
    e1 = np.array([0.8, 0.1, 0.2])
    e2 = np.array([-0.1, -0.6, 0.3])
    if np.cross(e1, e2) @ (np.zeros(3) - c) < 0:        # emit towards the point
        e1, e2 = e2, e1
    n = np.array([0.2, -0.1, 1.0])
    n /= np.linalg.norm(n)
    inten = np.array([1.0, 0.8, 0.5])
    val = _point_value(scenes.quad_light(c, e1, e2), np.zeros(3), n, inten)
    corners = [c - e1 / 2 - e2 / 2, c + e1 / 2 - e2 / 2, c + e1 / 2 + e2 / 2, c - e1 / 2 + e2 / 2]
    want = polygon_irradiance(corners, np.zeros(3), n) / math.pi * inten
    assert np.allclose(val, want, rtol=6e-3)


def test_disk_irradiance_on_axis():
    """Lambertian point on the axis of a disk light: E = pi L R^2 / (R^2 + h^2)."""
    R, h = 0.6, 1.1
    rec = scenes.quad_light([0, 0, h], [R, 0, 0], [0, -R, 0], synth.LIGHT_DISK)
    val = _point_value(rec, np.zeros(3), np.array([0, 0, 1.0]), (1, 1, 1))
    assert np.allclose(val, R * R / (R * R + h * h), rtol=5e-3)


def test_white_furnace_limit():
    """A Lambertian white point under a disk that fills almost the whole
    hemisphere reflects almost exactly the emitted radiance."""
    R, h = 4.0, 0.5          # 98.5% of the cosine-weighted hemisphere
    rec = scenes.quad_light([0, 0, h], [R, 0, 0], [0, -R, 0], synth.LIGHT_DISK)
    val = _point_value(rec, np.zeros(3), np.array([0, 0, 1.0]), (1, 1, 1), samples=2000000)
    # area sampling: per-sample relative std ~4.6, so 2e6 samples give ~0.33%
    assert np.allclose(val, R * R / (R * R + h * h), rtol=1.5e-2)


def test_triangle_emitter_matches_polygon_formula():
    c = np.array([-0.4, -0.3, 1.2])
    e1 = np.array([0.9, 0.0, 0.1])
    e2 = np.array([0.2, 0.8, 0.0])
    if np.cross(e1, e2) @ (np.zeros(3) - c) < 0:
        e1, e2 = e2, e1
    n = np.array([0.0, 0.0, 1.0])
    val = _point_value(scenes.quad_light(c, e1, e2, synth.LIGHT_TRI), np.zeros(3), n, (1, 1, 1))
    want = polygon_irradiance([c, c + e1, c + e2], np.zeros(3), n) / math.pi
    assert np.allclose(val, want, rtol=6e-3)


# ---------------------------------------------------------------------------
# Shadow-boundary term (edge sampling, Sec. 4) vs the closed form of the
# shadowed irradiance: E(quad) - E(quad intersected with the occluder's shadow)
# ---------------------------------------------------------------------------
def clip_convex(poly, clip):
    """Sutherland-Hodgman clipping of a 2D polygon by a convex CCW polygon."""
    out = [np.asarray(p, float) for p in poly]
    for i in range(len(clip)):
        a, b = np.asarray(clip[i], float), np.asarray(clip[(i + 1) % len(clip)], float)
        inp, out = out, []
        if not inp:
            break

        def side(p):
            return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])

        for k in range(len(inp)):
            p, q = inp[k], inp[(k + 1) % len(inp)]
            sp, sq = side(p), side(q)
            if sp >= 0:
                out.append(p)
            if (sp >= 0) != (sq >= 0):
                out.append(p + (q - p) * (sp / (sp - sq)))
    return out


def _shadow_scene(coef):
    occ = np.array([[-0.1, -0.3, 1.0], [0.6, -0.1, 1.0], [0.05, 0.5, 1.0]])
    basis = np.zeros((2, 3, 3))
    basis[0, 1, 0] = 1.0            # moves occluder vertex 1 along x
    basis[1, 2, 2] = 1.0            # moves occluder vertex 2 along z
    light = scenes.quad_light([0, 0, 2.0], [1.0, 0, 0], [0, -1.0, 0])
    sc, pr = scenes.make(occ, [[0, 1, 2]], basis, [light], light_i=[(1, 1, 1)])
    pr.coef = np.asarray(coef, np.float32)
    return sc, pr, occ, basis


def _shadowed_value(coef):
    _, _, occ, basis = _shadow_scene(coef)
    v = occ + np.tensordot(np.asarray(coef, float), basis, axes=1)
    quad = [(-0.5, -0.5), (0.5, -0.5), (0.5, 0.5), (-0.5, 0.5)]
    # central projection from y = 0 onto the plane z = 2
    proj = [(2.0 * p[0] / p[2], 2.0 * p[1] / p[2]) for p in v]
    area2 = (proj[1][0] - proj[0][0]) * (proj[2][1] - proj[0][1]) - \
            (proj[1][1] - proj[0][1]) * (proj[2][0] - proj[0][0])
    if area2 < 0:
        proj = proj[::-1]
    hole = clip_convex(proj, quad)
    n = np.array([0, 0, 1.0])
    E = polygon_irradiance([(x, y, 2.0) for x, y in quad], np.zeros(3), n)
    if len(hole) >= 3:
        E -= polygon_irradiance([(x, y, 2.0) for x, y in hole], np.zeros(3), n)
    return E / math.pi


def test_shadow_edge_term_matches_closed_form():
    coef = np.array([0.05, 0.1])
    sc, pr, _, _ = _shadow_scene(coef)
    val, g = oracle.point_light_grad(sc, pr, np.zeros(3), np.array([0, 0, 1.0]), 1500000)
    assert val[0] == pytest.approx(_shadowed_value(coef), rel=5e-3)
    h = 1e-5
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (_shadowed_value(coef + e) - _shadowed_value(coef - e)) / (2 * h)
        assert abs(fd) > 1e-3
        assert g[k] == pytest.approx(fd, rel=2.5e-2), (k, g[k], fd)


# ---------------------------------------------------------------------------
# Primary-visibility boundary term vs analytic pixel coverage (flat shading)
# ---------------------------------------------------------------------------
def _coverage_scene():
    tri = np.array([[-0.9, -0.8, -3.0], [1.2, -0.3, -3.0], [0.1, 1.1, -3.5]])
    basis = np.zeros((2, 3, 3))
    basis[0, 0, 0] = 1.0
    basis[1, 2, 1] = 0.6
    basis[1, 2, 2] = 0.8
    light = scenes.quad_light([0, 0, 5.0], [1, 0, 0], [0, 1, 0])
    sc, pr = scenes.make(tri, [[0, 1, 2]], basis, [light])
    return sc, pr, tri, basis


def _coverage_objective(theta, weights):
    """sum_p A_p . c area(projected triangle n pixel p), theta = (coef0, coef1, f)."""
    _, pr, tri, basis = _coverage_scene()
    v = tri + theta[0] * basis[0] + theta[1] * basis[1]
    f = theta[2]
    pts = [(8.0 + f * p[0] / -p[2], 8.0 - f * p[1] / -p[2]) for p in v]
    area2 = (pts[1][0] - pts[0][0]) * (pts[2][1] - pts[0][1]) - (pts[1][1] - pts[0][1]) * (pts[2][0] - pts[0][0])
    if area2 < 0:
        pts = pts[::-1]
    c = np.array([0.7, 0.5, 0.3])
    tot = 0.0
    for py in range(16):
        for px in range(16):
            box = [(px, py), (px + 1, py), (px + 1, py + 1), (px, py + 1)]
            poly = clip_convex(pts, box)
            if len(poly) < 3:
                continue
            a = 0.0
            for k in range(len(poly)):
                x0, y0 = poly[k]
                x1, y1 = poly[(k + 1) % len(poly)]
                a += x0 * y1 - x1 * y0
            tot += abs(0.5 * a) * (weights[py, px] @ c)
    return tot


def test_primary_edge_term_matches_coverage_derivative():
    sc, pr, _, _ = _coverage_scene()
    yy, xx = np.mgrid[0:16, 0:16]
    w = 1.0 + 0.5 * np.sin(xx / 3.0)[..., None] * np.cos(yy / 4.0)[..., None] * np.array([1.0, 0.7, -0.4])
    g = oracle.grad(sc, pr, w, terms=oracle.TERM_PRIMARY, flags=oracle.FLAT, edge_spp=256)
    theta = np.array([0.0, 0.0, 16.0])
    h = 1e-5
    fd = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        fd.append((_coverage_objective(theta + e, w) - _coverage_objective(theta - e, w)) / (2 * h))
    got = [g["coef"][0], g["coef"][1], g["focal"][0]]
    for k in range(3):
        assert got[k] == pytest.approx(fd[k], rel=2e-2), (k, got[k], fd[k])
    # flat shading with a uniform texture has no interior term
    gi = oracle.grad(sc, pr, w, terms=oracle.TERM_INTERIOR, flags=oracle.FLAT)
    assert np.all(np.abs(gi["coef"]) < 1e-12)


# ---------------------------------------------------------------------------
# Brute-force intersection with known answers
# ---------------------------------------------------------------------------
def test_closest_hit_known_square():
    verts = [[-1, -1, -5], [1, -1, -5], [1, 1, -5], [-1, 1, -5], [-1, -1, -7], [1, -1, -7], [0, 1, -7]]
    faces = [[0, 1, 2], [0, 2, 3], [4, 5, 6]]
    sc, pr = scenes.make(verts, faces, np.zeros((1, 7, 3)), [scenes.quad_light([0, 0, 3], [1, 0, 0], [0, 1, 0])])
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1.2, 1.2, size=(400, 2))
    dirs = np.concatenate([pts, np.full((400, 1), -5.0)], 1)
    tri, t = oracle.closest_hit(sc, pr, np.zeros((400, 3)), dirs)
    for (x, y), k, tt in zip(pts, tri, t):
        if abs(x) <= 1 and abs(y) <= 1:
            assert k == (0 if x >= y else 1) and tt == pytest.approx(1.0, abs=1e-14)
        else:
            # behind the square only the far triangle can be hit
            assert k in (-1, 2)
    # exactly on the shared diagonal: the tie goes to the lower index
    tri, _ = oracle.closest_hit(sc, pr, np.zeros((1, 3)), np.array([[0.25, 0.25, -5.0]]))
    assert tri[0] == 0


def test_render_records_agree_with_brute_force():
    """Every camera sample's recorded hit triangle equals an independent
    brute-force closest hit: the morphed mesh posed with scipy's R = Rz Ry Rx,
    the jittered camera ray of the sample (Philox dims 0, 1), and a vectorised
    Moller-Trumbore test against all 320 triangles (ties to the lower index)."""
    from scipy.spatial.transform import Rotation
    sc = synth.make_scene("tiny", width=12, height=12, spp=2)
    pr = synth.random_params(sc, 1)
    img, tri, _ = oracle.render(sc, pr, records=True)
    assert img.shape == (12, 12, 3) and np.all(img >= 0)
    v = sc.mean.astype(np.float64) + np.tensordot(pr.coef.astype(np.float64), sc.basis.astype(np.float64), axes=1)
    R = Rotation.from_euler("xyz", pr.rot.astype(np.float64)).as_matrix()
    v = (v - pr.trans.astype(np.float64)) @ R                     # rows of R^T (v - T)
    F = np.asarray(sc.faces)
    v0, e1, e2 = v[F[:, 0]], v[F[:, 1]] - v[F[:, 0]], v[F[:, 2]] - v[F[:, 0]]
    W, H, f = sc.width, sc.height, float(pr.focal[0])
    want = np.empty_like(tri)
    for q in range(W * H * sc.spp):
        p, s_ = divmod(q, sc.spp)
        w = oracle.philox(0, 0, p, s_ << 16, 0, 0)
        sx = p % W + (int(w[0]) >> 8) / 16777216.0
        sy = p // W + (int(w[1]) >> 8) / 16777216.0
        d = np.array([(sx - 0.5 * W) / f, -(sy - 0.5 * H) / f, -1.0])
        pv = np.cross(d, e2)
        det = np.einsum("ij,ij->i", e1, pv)
        sv = -v0
        with np.errstate(divide="ignore", invalid="ignore"):
            b1 = np.einsum("ij,ij->i", sv, pv) / det
            qv = np.cross(sv, e1)
            b2 = (qv @ d) / det
            t = np.einsum("ij,ij->i", e2, qv) / det
        ok = (det != 0) & (b1 >= 0) & (b2 >= 0) & (b1 + b2 <= 1) & (t > 0)
        want[q] = int(np.flatnonzero(ok)[np.argmin(t[ok])]) if ok.any() else -1
    assert 0.2 < np.mean(tri >= 0) < 0.9
    assert np.array_equal(tri, want), int(np.sum(tri != want))


# ---------------------------------------------------------------------------
# Blur and L1 loss (Sec. 4)
# ---------------------------------------------------------------------------
def test_blur_weights_and_loss_gradient():
    h = w = 9
    img = np.zeros((h, w, 3))
    img[4, 4, :] = 1.0
    _, bl, _ = oracle.loss(img, np.zeros((h, w, 3), np.float32))
    z = 1 + 4 * math.exp(-0.5) + 4 * math.exp(-1.0)
    assert bl[4, 4, 0] == pytest.approx(1 / z, rel=1e-14)
    assert bl[3, 4, 0] == pytest.approx(math.exp(-0.5) / z, rel=1e-14)
    assert bl[3, 3, 0] == pytest.approx(math.exp(-1.0) / z, rel=1e-14)
    const = np.full((h, w, 3), 0.37)
    _, bl, _ = oracle.loss(const, np.zeros((h, w, 3), np.float32))
    assert np.allclose(bl, 0.37, rtol=1e-14)
    rng = np.random.default_rng(5)
    img = rng.uniform(0, 1, (h, w, 3))
    tgt = rng.uniform(0, 1, (h, w, 3)).astype(np.float32)
    val, _, adj = oracle.loss(img, tgt)
    d = rng.normal(size=img.shape)
    eps = 1e-7
    fd = (oracle.loss(img + eps * d, tgt)[0] - oracle.loss(img - eps * d, tgt)[0]) / (2 * eps)
    assert fd == pytest.approx(np.sum(adj * d), rel=1e-6)


# ---------------------------------------------------------------------------
# Interior gradients: exact linearity and finite differences with the samples
# held fixed
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny():
    sc = synth.make_scene("tiny", width=16, height=16, spp=2)
    pr = synth.random_params(sc, 2)
    adj = np.random.default_rng(9).uniform(0.2, 1.0, (16, 16, 3))
    return sc, pr, adj


def _J(sc, pr, adj, **kw):
    return float(np.sum(adj * oracle.render(sc, pr, **kw)))


def test_light_gradient_is_single_light_image(tiny):
    sc, pr, adj = tiny
    g = oracle.grad(sc, pr, adj, terms=oracle.TERM_INTERIOR)
    for j in range(sc.n_lights):
        q = pr.copy()
        q.light_i[:] = 0.0
        q.light_i[j] = 1.0
        img = oracle.render(sc, q)
        want = np.sum(adj * img, axis=(0, 1))
        assert np.allclose(g["light_i"][j], want, rtol=1e-10, atol=1e-14)
    # linearity: the sum of single-light images is the full image
    tot = np.zeros((16, 16, 3))
    for j in range(sc.n_lights):
        q = pr.copy()
        q.light_i[:] = 0.0
        q.light_i[j] = pr.light_i[j]
        tot += oracle.render(sc, q)
    assert np.allclose(tot, oracle.render(sc, pr), rtol=1e-12, atol=1e-15)


def test_light_gradient_beyond_64_lights():
    """80 lights (the large light stage): the intensity gradient of lights past
    the 64th is still the single-light image, and the lights sum to the image."""
    sc = synth.make_scene("tiny", width=12, height=12, spp=2, n_lights=80)
    pr = synth.random_params(sc, 3)
    adj = np.random.default_rng(4).uniform(0.2, 1.0, (12, 12, 3))
    g = oracle.grad(sc, pr, adj, terms=oracle.TERM_INTERIOR)
    tot = np.zeros((12, 12, 3))
    for j in range(sc.n_lights):
        q = pr.copy()
        q.light_i[:] = 0.0
        q.light_i[j] = 1.0
        img = oracle.render(sc, q)
        assert np.allclose(g["light_i"][j], np.sum(adj * img, axis=(0, 1)), rtol=1e-10, atol=1e-14), j
        tot += img * pr.light_i[j]
    assert np.abs(g["light_i"][64:]).sum() > 0.0
    assert np.allclose(tot, oracle.render(sc, pr), rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("name", ["diffuse", "specular"])
def test_texture_gradient_exact_by_linearity(tiny, name):
    sc, pr, adj = tiny
    g = oracle.grad(sc, pr, adj, terms=oracle.TERM_INTERIOR)[name]
    d = np.random.default_rng(4).normal(size=g.shape).astype(np.float32) * 0.05
    qp, qm = pr.copy(), pr.copy()
    getattr(qp, name)[...] += d
    getattr(qm, name)[...] -= d
    # the float32 perturbations actually applied
    step = (getattr(qp, name).astype(np.float64) - getattr(qm, name)) / 2.0
    fd = (_J(sc, qp, adj) - _J(sc, qm, adj)) / 2.0
    assert fd == pytest.approx(np.sum(g * step), rel=1e-9)


def _fd_fixed_samples(sc, pr, adj, field, index, h):
    """Central difference of sum(A * image) w.r.t. one float32 parameter with
    every sample's hit triangle and shadow mask held fixed.

    The base point is moved onto a grid of power-of-two step >= h so that the
    float32 parameters represent theta +- step exactly.  Pixels whose records
    change under the step are masked out of A.  Returns (fd, masked A, base)."""
    hh = 2.0 ** round(math.log2(h))
    base = pr.copy()
    arr = getattr(base, field)
    x = float(arr.flat[index])
    step = max(hh, float(np.spacing(np.float32(abs(x) + 4 * hh))))
    x = round(x / step) * step
    arr.flat[index] = np.float32(x)

    def shifted(sign):
        q = base.copy()
        getattr(q, field).flat[index] = np.float32(x + sign * step)
        assert float(getattr(q, field).flat[index]) == x + sign * step
        return q

    b0 = oracle.render(sc, base, records=True)
    up = oracle.render(sc, shifted(+1), records=True)
    dn = oracle.render(sc, shifted(-1), records=True)
    same = (b0[1] == up[1]) & (b0[1] == dn[1]) & (b0[2] == up[2]).all(axis=1) & (b0[2] == dn[2]).all(axis=1)
    keep = same.reshape(-1, sc.spp).all(axis=1).reshape(sc.height, sc.width)
    a = adj * keep[..., None]
    fd = (np.sum(a * up[0]) - np.sum(a * dn[0])) / (2 * step)
    return fd, a, base


@pytest.mark.parametrize("field,index", [("coef", 0), ("coef", 4), ("rot", 1), ("trans", 0),
                                         ("trans", 2), ("focal", 0), ("roughness", 37)])
def test_interior_gradient_matches_fixed_sample_fd(tiny, field, index):
    sc, pr, adj = tiny
    h = 1e-6 if field != "roughness" else 1e-5
    fd, a, base = _fd_fixed_samples(sc, pr, adj, field, index, h)
    g = oracle.grad(sc, base, a, terms=oracle.TERM_INTERIOR)
    got = np.asarray(g[field]).flat[index]
    assert abs(got - fd) <= 1e-5 * max(abs(fd), 1e-3), (got, fd)
