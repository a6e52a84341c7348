"""Pins of the oracle's pose, normals and texture lookup through its full render.

Each render pin recomputes the oracle's image sample by sample from closed-form
geometry: the camera sample positions and emitter sample points come from the
published Philox4x32-10 stream (pinned by its known-answer vectors), then

* Euler pose (Sec. 3.1, R = Rz Ry Rx, v' = R^T (v - T)): rotations from scipy
  (composed) and from the textbook single-axis matrices; the rendered texture
  of a posed plane follows from intersecting each camera ray with the plane in
  closed form and mapping the hit back to model space;
* vertex and shading normals (App. A): on a regular octahedron the vertex
  normals are radial by symmetry, so the barycentric blend of a face's vertex
  normals at a hit point y is parallel to y - centre (its vertices have equal
  radius); on a flat mesh every normal is the plane's; the area-weighted vertex
  normal of a fan equals the vector area of its one-ring, wherever the apex is;
* bilinear texel lookup (Sec. 3.2, texel centres at u M - 1/2, clamp to edge):
  scipy's order-1 map_coordinates with edge replication.

A mistake in any of them (a transposed or reordered rotation, a flipped or
unweighted normal, a shifted texel centre, a wrapped edge) changes the image by
far more than the tolerances."""
import math

import numpy as np
import pytest
from scipy import ndimage
from scipy.spatial.transform import Rotation

import oracle
from paper_2101_05356_gb300 import synth
from tests import scenes


def _u24(x):
    return float(int(x) >> 8) / 16777216.0


def _sample_dims(pixel, s, seed=0, iteration=0, face=0):
    """Camera jitter (dims 0, 1) and the first light's sample (dims 2, 3) of
    camera sample s of `pixel`: Philox key (seed, 0), counter
    (pixel, s << 16 | 0, iteration, face), u = (x >> 8) 2^-24."""
    w = oracle.philox(seed, 0, pixel, (s << 16) | 0, iteration, face)
    return _u24(w[0]), _u24(w[1]), _u24(w[2]), _u24(w[3])


def _camera_dir(sx, sy, W, H, f):
    return np.array([(sx - 0.5 * W) / f, -(sy - 0.5 * H) / f, -1.0])


def _per_pixel(W, H, spp, value):
    """Mean over each pixel's camera samples of value(pixel, s, dims)."""
    img = np.zeros((H, W, 3))
    for p in range(W * H):
        acc = np.zeros(3)
        for s in range(spp):
            acc += value(p, s, _sample_dims(p, s))
        img[p // W, p % W] = acc / spp
    return img


# ---------------------------------------------------------------------------
# Euler pose (Sec. 3.1)
# ---------------------------------------------------------------------------
def _rx(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _ry(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def _rz(t):
    c, s = math.cos(t), math.sin(t)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def _posed_scene(rot, trans, n=9):
    rng = np.random.default_rng(3)
    verts = rng.uniform(-1, 1, (n, 3))
    faces = [[0, 1, 2], [3, 4, 5], [6, 7, 8]]
    sc, pr = scenes.make(verts, faces, np.zeros((1, n, 3)), [scenes.quad_light([0, 0, 3], [1, 0, 0], [0, 1, 0])])
    pr.rot = np.asarray(rot, np.float32)
    pr.trans = np.asarray(trans, np.float32)
    return sc, pr


@pytest.mark.parametrize("axis", range(3))
def test_single_axis_rotation_matches_its_matrix(axis):
    """A rotation about one axis poses vertices with the textbook matrix of that
    axis, transposed: v' = R^T (v - T)."""
    theta = [0.7, -1.1, 2.3][axis]
    rot = np.zeros(3)
    rot[axis] = theta
    trans = np.array([0.3, -0.2, 0.9])
    sc, pr = _posed_scene(rot, trans)
    v, _ = oracle.geometry(sc, pr)
    R = [_rx, _ry, _rz][axis](float(np.float32(theta)))
    want = (sc.mean.astype(np.float64) - pr.trans.astype(np.float64)) @ R      # rows: (R^T (v - T))^T
    assert np.allclose(v, want, rtol=0, atol=1e-12)
    # the other sense of rotation is far off
    assert not np.allclose(v, (sc.mean - pr.trans) @ R.T, atol=1e-3)


def test_composed_euler_rotation_matches_scipy():
    """R = Rz(tz) Ry(ty) Rx(tx): scipy's extrinsic x-y-z rotation; the reversed
    order (Rx Ry Rz) is far off."""
    rot = np.array([0.4, -0.9, 1.3], np.float32)
    sc, pr = _posed_scene(rot, [0.1, 0.2, -0.3])
    v, _ = oracle.geometry(sc, pr)
    R = Rotation.from_euler("xyz", rot.astype(np.float64)).as_matrix()
    assert np.allclose(R, _rz(rot[2]) @ _ry(rot[1]) @ _rx(rot[0]), atol=1e-14)
    d = sc.mean.astype(np.float64) - pr.trans.astype(np.float64)
    assert np.allclose(v, d @ R, rtol=0, atol=1e-12)
    R_rev = _rx(rot[0]) @ _ry(rot[1]) @ _rz(rot[2])
    assert not np.allclose(v, d @ R_rev, atol=1e-2)


# ---------------------------------------------------------------------------
# Textured planes through the render (flat mode: radiance = diffuse texture)
# ---------------------------------------------------------------------------
def _bilinear_clamped(tex, u, v):
    """Texel (i, j) centred at ((j + 1/2)/M, (i + 1/2)/M), edges replicated."""
    M = tex.shape[0]
    return np.array([ndimage.map_coordinates(tex[..., k].astype(np.float64), [[v * M - 0.5], [u * M - 0.5]],
                                             order=1, mode="nearest")[0] for k in range(3)])


def _textured_plane(half, z, M, seed):
    """Two triangles spanning [-half, half]^2 at depth z (model space), facing
    +z, with u = (x + half)/(2 half) - 0.05 and v = (half - y)/(2 half) - 0.05
    scaled past [0, 1] so that clamped edges are sampled too."""
    verts = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]], np.float32)
    faces = [[0, 1, 2], [0, 2, 3]]
    sc, pr = scenes.make(verts, faces, np.zeros((1, 4, 3)), [scenes.quad_light([0, 0, 3], [1, 0, 0], [0, 1, 0])],
                         width=12, height=10, spp=4, tex=M)
    s = 1.1 / (2 * half)
    uv = np.stack([(verts[:, 0] + half) * s - 0.05, (half - verts[:, 1]) * s - 0.05], 1).astype(np.float32)
    sc.uv = uv
    pr.diffuse = np.random.default_rng(seed).uniform(0, 1, (M, M, 3)).astype(np.float32)
    return sc, pr, s


def test_bilinear_texel_lookup_through_the_render():
    """A fronto-parallel textured plane filling the view: each camera sample's
    radiance is the bilinear, edge-clamped lookup at its uv (a 5 x 5 texture,
    uv running from -0.05 to 1.05 across the plane)."""
    half, z, M = 2.6, -4.0, 5
    sc, pr, s = _textured_plane(half, z, M, seed=1)
    W, H, f = sc.width, sc.height, 11.0
    pr.focal = np.array([f], np.float32)
    img = oracle.render(sc, pr, flags=oracle.FLAT)

    def lookup(du, tex):
        def value(p, k, dims):
            d = _camera_dir(p % W + dims[0], p // W + dims[1], W, H, f)
            y = d * (z / d[2])
            return tex((y[0] + half) * s - 0.05 + du, (half - y[1]) * s - 0.05)
        return value

    want = _per_pixel(W, H, sc.spp, lookup(0.0, lambda u, v: _bilinear_clamped(pr.diffuse, u, v)))
    assert np.allclose(img, want, rtol=0, atol=2e-6), float(np.abs(img - want).max())
    # the texels are sampled across the whole map, clamped edges included
    assert want.min() < 0.15 and want.max() > 0.85
    # texel centres shifted by half a texel, or a wrapped instead of clamped edge, are far off
    shifted = _per_pixel(W, H, sc.spp, lookup(0.5 / M, lambda u, v: _bilinear_clamped(pr.diffuse, u, v)))
    assert np.abs(img - shifted).max() > 0.05
    wrapped = _per_pixel(W, H, sc.spp, lookup(0.0, lambda u, v: np.array([ndimage.map_coordinates(
        pr.diffuse[..., k].astype(np.float64), [[v * M - 0.5], [u * M - 0.5]], order=1, mode="grid-wrap")[0]
        for k in range(3)])))
    assert np.abs(img - wrapped).max() > 0.05


def test_posed_plane_through_the_render():
    """The textured plane at the model origin, posed by R = Rz Ry Rx (scipy) and
    T: each camera ray meets the posed plane at t = (n'.p0') / (n'.d) with
    n' = R^T e_z and p0' = -R^T T; its model-space point R y' + T gives the uv
    whose bilinear texel the flat render shows."""
    half, M = 3.0, 6
    sc, pr, s = _textured_plane(half, 0.0, M, seed=2)
    rot = np.array([0.25, -0.2, 0.35], np.float32)
    # T = R (0.1, -0.05, 4): the plane's centre lands near (-0.1, 0.05, -4), in view
    trans = (Rotation.from_euler("xyz", rot.astype(np.float64)).as_matrix() @ [0.1, -0.05, 4.0]).astype(np.float32)
    pr.rot, pr.trans = rot, trans
    W, H, f = sc.width, sc.height, 15.0
    pr.focal = np.array([f], np.float32)
    img = oracle.render(sc, pr, flags=oracle.FLAT)
    T = trans.astype(np.float64)

    def posed(R, inside=False):
        n_c = R.T @ np.array([0.0, 0.0, 1.0])
        p0 = -R.T @ T

        def value(p, k, dims):
            d = _camera_dir(p % W + dims[0], p // W + dims[1], W, H, f)
            y_cam = d * ((n_c @ p0) / (n_c @ d))
            v_model = R @ y_cam + T
            assert abs(v_model[2]) < 1e-9 and (not inside or max(abs(v_model[0]), abs(v_model[1])) < half)
            return _bilinear_clamped(pr.diffuse, (v_model[0] + half) * s - 0.05, (half - v_model[1]) * s - 0.05)
        return _per_pixel(W, H, sc.spp, value)

    R = Rotation.from_euler("xyz", rot.astype(np.float64)).as_matrix()
    want = posed(R, inside=True)
    assert np.allclose(img, want, rtol=0, atol=2e-6), float(np.abs(img - want).max())
    # v' = R (v - T) instead of R^T (v - T), or the rotations composed the other
    # way round (Rx Ry Rz), render a different image
    assert np.abs(img - posed(R.T)).max() > 0.05
    assert np.abs(img - posed(_rx(rot[0]) @ _ry(rot[1]) @ _rz(rot[2]))).max() > 0.02


# ---------------------------------------------------------------------------
# Vertex normals and the interpolated shading normal (App. A)
# ---------------------------------------------------------------------------
OCTA_V = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
# outward (counter-clockwise seen from outside) faces of the octahedron |x|+|y|+|z| = 1
OCTA_F = [[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]]


def test_vertex_normals_closed_forms():
    light = [scenes.quad_light([0, 0, 3], [1, 0, 0], [0, 1, 0])]
    # octahedron: radial by symmetry
    sc, pr = scenes.make(OCTA_V, OCTA_F, np.zeros((1, 6, 3)), light)
    _, n = oracle.geometry(sc, pr)
    assert np.allclose(n, np.asarray(OCTA_V, float), atol=1e-14)
    # flat 3 x 3 grid in a tilted plane: every normal is the plane's
    a, b = np.array([1.0, 0.2, -0.3]), np.array([-0.1, 0.8, 0.4])
    grid = np.array([i * a + j * b for j in range(3) for i in range(3)], np.float32)
    faces = []
    for j in range(2):
        for i in range(2):
            q = 3 * j + i
            faces += [[q, q + 1, q + 4], [q, q + 4, q + 3]]
    sc, pr = scenes.make(grid, faces, np.zeros((1, 9, 3)), light)
    _, n = oracle.geometry(sc, pr)
    nz = np.cross(a, b)
    assert np.allclose(n, nz / np.linalg.norm(nz), atol=1e-6)
    # a fan: the sum of its faces' cross products is the vector area of the
    # one-ring (independent of the apex), so the area-weighted normal at the apex
    # does not move when the apex does; an angle-weighted or unweighted one would
    ring = np.array([[1.0, 0.0, 0.1], [0.6, 0.9, -0.2], [-0.5, 1.1, 0.3], [-1.2, 0.1, -0.1], [-0.4, -0.9, 0.2],
                     [0.7, -0.8, -0.3]])
    va = 0.5 * sum(np.cross(ring[k], ring[(k + 1) % 6]) for k in range(6))
    fan = [[6, k, (k + 1) % 6] for k in range(6)]
    normals = []
    for apex in ([0.0, 0.0, 0.8], [0.3, -0.2, 0.5], [-0.4, 0.35, 1.4]):
        verts = np.vstack([ring, apex]).astype(np.float32)
        sc, pr = scenes.make(verts, fan, np.zeros((1, 7, 3)), light)
        _, n = oracle.geometry(sc, pr)
        vf = verts.astype(np.float64)
        va32 = 0.5 * sum(np.cross(vf[k], vf[(k + 1) % 6]) for k in range(6))
        assert np.allclose(n[6], va32 / np.linalg.norm(va32), atol=1e-12)
        normals.append(n[6])
    assert np.allclose(normals[0], va / np.linalg.norm(va), atol=1e-6)
    unweighted = sum(np.cross(vf[k] - vf[6], vf[(k + 1) % 6] - vf[6]) /
                     np.linalg.norm(np.cross(vf[k] - vf[6], vf[(k + 1) % 6] - vf[6])) for k in range(6))
    assert np.linalg.norm(normals[2] - unweighted / np.linalg.norm(unweighted)) > 1e-2


def _lit_scene(kind):
    """Lambertian white-ish surface, one quad light near the camera."""
    light = scenes.quad_light([0.3, 0.5, -1.0], [0.5, 0.0, 0.0], [0.0, -0.5, 0.0])
    if kind == "octahedron":
        sc, pr = scenes.make(OCTA_V, OCTA_F, np.zeros((1, 6, 3)), [light], width=14, height=12, spp=4,
                             light_i=[(1.5, 1.2, 0.9)])
        pr.trans = np.array([0.0, 0.0, 3.5], np.float32)        # centre at (0, 0, -3.5)
        pr.focal = np.array([26.0], np.float32)
    else:                                                       # flat fan of 8 triangles, tilted
        # dyadic coordinates: the fan is exactly planar in float32
        a, b = np.array([1.5, 0.25, 0.5]), np.array([-0.25, 1.375, 0.625])
        ctr = np.array([0.0, 0.0, -3.5])
        pts = [ctr + (i - 1) * a + (j - 1) * b for j in range(3) for i in range(3)]
        faces = []
        for j in range(2):
            for i in range(2):
                q = 3 * j + i
                faces += [[q, q + 1, q + 4], [q, q + 4, q + 3]]
        sc, pr = scenes.make(pts, faces, np.zeros((1, 9, 3)), [light], width=14, height=12, spp=4,
                             light_i=[(1.5, 1.2, 0.9)])
        pr.focal = np.array([16.0], np.float32)
    return sc, pr, light


def _octa_hit(d, c):
    """Entry point of the ray t d into |x|+|y|+|z| <= 1 centred at c (None: miss)."""
    t_in, t_out, n_in = -np.inf, np.inf, None
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                sgn = np.array([sx, sy, sz], float)
                den = sgn @ d
                t = (1.0 + sgn @ c) / den
                if den < 0 and t > t_in:
                    t_in, n_in = t, sgn / math.sqrt(3.0)
                elif den > 0:
                    t_out = min(t_out, t)
    return (t_in, n_in) if t_in <= t_out else None


@pytest.mark.parametrize("kind", ["octahedron", "flat"])
def test_shading_normals_through_the_render(kind):
    """Diffuse-only render of a lit octahedron (shading normal (y - c)/|y - c|
    at every hit y) and of a flat fan (the plane normal): every camera sample's
    value (c/pi) L A max(0, n_s.l) max(0, -n_L.l) / |z - y|^2 at its emitter
    sample z, shadowed where the geometric normal faces away from the light (the
    octahedron is convex), averaged per pixel."""
    sc, pr, light = _lit_scene(kind)
    W, H, f = sc.width, sc.height, float(pr.focal[0])
    img = oracle.render(sc, pr, flags=oracle.DIFFUSE_ONLY)
    c_alb = pr.diffuse[0, 0].astype(np.float64)
    Lrad = pr.light_i[0].astype(np.float64)
    lc, e1, e2 = (light[1:4].astype(np.float64), light[4:7].astype(np.float64), light[7:10].astype(np.float64))
    nl = np.cross(e1, e2)
    area = np.linalg.norm(nl)
    nl /= area
    verts = sc.mean.astype(np.float64) - pr.trans.astype(np.float64)
    if kind == "flat":
        ng = np.cross(verts[1] - verts[0], verts[4] - verts[0])
        ng /= np.linalg.norm(ng)

    def value(p, k, dims):
        d = _camera_dir(p % W + dims[0], p // W + dims[1], W, H, f)
        if kind == "octahedron":
            ctr = -pr.trans.astype(np.float64)
            h = _octa_hit(d, ctr)
            if h is None:
                return np.zeros(3)
            y = d * h[0]
            ns, n_geo = (y - ctr) / np.linalg.norm(y - ctr), h[1]
        else:
            t = (ng @ verts[0]) / (ng @ d)
            y = d * t
            q = np.linalg.lstsq(np.stack([verts[2] - verts[0], verts[6] - verts[0]], 1), y - verts[0], rcond=None)[0]
            if not (0 <= q[0] <= 1 and 0 <= q[1] <= 1):
                return np.zeros(3)
            ns = n_geo = ng
        z = lc + (dims[2] - 0.5) * e1 + (dims[3] - 0.5) * e2
        lv = z - y
        d2 = lv @ lv
        l = lv / math.sqrt(d2)
        cs, cl = ns @ l, -(nl @ l)
        if cs <= 0 or cl <= 0 or n_geo @ l <= 0:
            return np.zeros(3)
        return c_alb / math.pi * Lrad * area * cs * cl / d2

    want = _per_pixel(W, H, sc.spp, value)
    assert np.count_nonzero(want[..., 0]) > 0.3 * W * H
    assert np.allclose(img, want, rtol=1e-9, atol=1e-12), float(np.abs(img - want).max())
    if kind == "octahedron":
        # the face normal instead of the blended vertex normals is far off
        assert np.abs(img - _per_pixel(W, H, sc.spp, lambda p, k, dims: _flat_octa(
            p, dims, W, H, f, pr, c_alb, Lrad, lc, e1, e2, nl, area))).max() > 1e-2


def _flat_octa(p, dims, W, H, f, pr, c_alb, Lrad, lc, e1, e2, nl, area):
    d = _camera_dir(p % W + dims[0], p // W + dims[1], W, H, f)
    h = _octa_hit(d, -pr.trans.astype(np.float64))
    if h is None:
        return np.zeros(3)
    y, ns = d * h[0], h[1]
    z = lc + (dims[2] - 0.5) * e1 + (dims[3] - 0.5) * e2
    lv = z - y
    d2 = lv @ lv
    l = lv / math.sqrt(d2)
    cs, cl = ns @ l, -(nl @ l)
    if cs <= 0 or cl <= 0:
        return np.zeros(3)
    return c_alb / math.pi * Lrad * area * cs * cl / d2
