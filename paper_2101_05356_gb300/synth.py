"""Seeded synthetic inputs shaped like the paper's workloads.

The paper (Sec. 3.1-3.3, Sec. 5) works on real photographs, the Basel/AlbedoMM
statistical face models and a landmark detector; none of those is available, so
every input here is synthetic and seeded.  This module draws inputs: a mean
face mesh with its topology and UV layout, shape/expression bases, UV textures,
light-stage emitter geometry, and parameter vectors.  It has no morph, pose,
projection, shading, loss or gradient; the renderer under test and the FP64
oracle both consume exactly these arrays.  One piece of the method's geometry
does live here: `stage_records` places the emitters of a virtual light stage
from its frame and (d, a, p) (Sec. 3.3), as the scene's fixed emitter records.
When the parameters carry (d, a, p) the CUDA library rebuilds the lights from
them itself and the oracle with its own code; neither side reads those records
then, and the oracle's builder is pinned by the closed-form shadowed irradiance
of a moving emitter, not by agreement with this function.

Units: model space is roughly a unit head centred at the origin, looking down +z
(towards the camera); the camera sits at T = (0, 0, 4.5) looking down -z, so the
pose v' = R^-1 (v - T) of Sec. 3.1 puts the face at z' ~ -4.5.

Emitter record (one row per light, float32[11]):
    [type, cx, cy, cz, e1x, e1y, e1z, e2x, e2y, e2z, reserved]
type 0 = quad  : z = c + (u - 1/2) e1 + (v - 1/2) e2
type 1 = tri   : vertices c, c + e1, c + e2
type 2 = disk  : centre c, orthogonal radius vectors e1, e2 (|e1| = |e2| = R)
The emitting side is the one that e1 x e2 points to.  Each light also carries
its distance d_j and relative area a_j of Eq. (lightIntensity).
type 3 = environment block: [3, i0, i1, j0, j1, 0...], texel rows [i0, i1) and
columns [j0, j1) of an M_e x M_e latitude-longitude map of lights at infinity
(the environment-map alternative of Sec. 7): row i spans polar angles
[i, i + 1] pi / M_e from camera-space +y, column j azimuths [j, j + 1] 2 pi / M_e
from +z towards +x; the radiance is the map's texel (Params.env).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

LIGHT_QUAD, LIGHT_TRI, LIGHT_DISK, LIGHT_ENV = 0, 1, 2, 3

# Camera translation that places the head in front of the camera (Sec. 3.1).
DEFAULT_T = (0.0, 0.0, 4.5)
# Light-stage centre in camera space: the nominal head position.
STAGE_CENTRE = (0.0, 0.0, -4.5)


@dataclasses.dataclass
class AlbedoModel:
    """Statistical albedo model of Sec. 3.2 in UV texture space: diffuse
    C = mean_diffuse + sum_k beta_k basis_diffuse[k], specular likewise with
    gamma (synthetic stand-in for the absent AlbedoMM; coefficients ~ N(0, 1),
    the column scale is in the basis)."""
    mean_diffuse: np.ndarray    # float32 [M, M, 3]
    basis_diffuse: np.ndarray   # float32 [K_r, M, M, 3]
    mean_specular: np.ndarray   # float32 [M, M, 3]
    basis_specular: np.ndarray  # float32 [K_b, M, M, 3]

    @property
    def k_diffuse(self) -> int:
        return int(self.basis_diffuse.shape[0])

    @property
    def k_specular(self) -> int:
        return int(self.basis_specular.shape[0])


@dataclasses.dataclass
class Scene:
    """Everything that is fixed for a reconstruction: mesh, bases, lights, image."""
    mean: np.ndarray        # float32 [N, 3] mean shape a_s (model space)
    basis: np.ndarray       # float32 [K, N, 3] columns of [Sigma_s | Sigma_e]
    n_shape: int            # K_s
    n_expr: int             # K_e
    faces: np.ndarray       # int32 [T, 3], counter-clockwise seen from outside
    uv: np.ndarray          # float32 [N, 2] in [0, 1]^2
    lights: np.ndarray      # float32 [N_L, 11] emitter records (module doc)
    light_d: np.ndarray     # float32 [N_L] distance d_j
    light_a: np.ndarray     # float32 [N_L] relative area a_j
    width: int
    height: int
    spp: int
    tex_size: int           # M
    fov_deg: float
    albedo: AlbedoModel | None = None
    landmarks: np.ndarray | None = None   # int32 [L] landmark vertex indices (Eq. landmark)
    stage: np.ndarray | None = None       # float32 [N_L, 12] polyhedral stage: centre, face V0, V1, V2
    env_size: int = 0                     # M_e of an environment map (type-3 records), 0: none

    @property
    def n_vertices(self) -> int:
        return int(self.mean.shape[0])

    @property
    def n_triangles(self) -> int:
        return int(self.faces.shape[0])

    @property
    def n_basis(self) -> int:
        return int(self.basis.shape[0])

    @property
    def n_lights(self) -> int:
        return int(self.lights.shape[0])

    def focal_px(self) -> float:
        """Pinhole focal length in pixels for the horizontal field of view."""
        return 0.5 * self.width / math.tan(math.radians(self.fov_deg) * 0.5)


@dataclasses.dataclass
class Params:
    """The optimised parameter set chi-hat (Sec. 4) for one face."""
    coef: np.ndarray        # float32 [K]  (alpha then delta)
    rot: np.ndarray         # float32 [3]  Euler angles (x, y, z)
    trans: np.ndarray       # float32 [3]  T
    focal: np.ndarray       # float32 [1]  focal length in pixels
    light_i: np.ndarray     # float32 [N_L, 3] perceived intensities i_j
    diffuse: np.ndarray     # float32 [M, M, 3]
    specular: np.ndarray    # float32 [M, M, 3]
    roughness: np.ndarray   # float32 [M, M]
    # virtual light stage geometry (Sec. 3.3), for scenes with a polyhedral stage
    light_d: np.ndarray | None = None   # float32 [N_L]    distance d_j
    light_a: np.ndarray | None = None   # float32 [N_L]    relative area a_j
    light_p: np.ndarray | None = None   # float32 [N_L, 2] barycentric centre (p_j0, p_j1)
    # environment-map radiance, for scenes with environment blocks
    env: np.ndarray | None = None       # float32 [M_e, M_e, 3]

    def copy(self) -> "Params":
        return Params(**{f.name: (None if getattr(self, f.name) is None else getattr(self, f.name).copy())
                         for f in dataclasses.fields(self)})

    def as_dict(self) -> dict:
        return {f.name: getattr(self, f.name) for f in dataclasses.fields(self)}


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def icosphere(level: int):
    """Unit icosphere: 10*4^level + 2 vertices, 20*4^level triangles."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
         (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(p, dtype=np.float64) / np.linalg.norm(p) for p in v]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts), np.array(faces, dtype=np.int32)


def _bump(p, centre, amp, width):
    c = np.asarray(centre, dtype=np.float64)
    c = c / np.linalg.norm(c)
    d2 = np.sum((p - c) ** 2, axis=1)
    return amp * np.exp(-d2 / (2.0 * width * width))


def _face_features(p):
    """Radial relief on the unit sphere: nose, brows, cheekbones, eye sockets."""
    r = np.zeros(p.shape[0])
    r += _bump(p, (0.0, -0.05, 1.0), 0.30, 0.16)            # nose
    for s in (-1.0, 1.0):
        r += _bump(p, (0.35 * s, 0.35, 0.87), 0.10, 0.14)   # brow ridge
        r += _bump(p, (0.50 * s, -0.12, 0.85), 0.08, 0.20)  # cheekbone
        r += _bump(p, (0.30 * s, 0.18, 0.93), -0.09, 0.11)  # eye socket
    r += _bump(p, (0.0, -0.55, 0.83), 0.06, 0.18)           # chin
    return r


def _rbf_columns(rng, unit_pts, normals, k_count, rms0):
    """K smooth displacement fields along the normal (16 Gaussian RBFs each),
    column k scaled to RMS rms0 / (1 + k)."""
    n = unit_pts.shape[0]
    cols = np.zeros((k_count, n, 3))
    for k in range(k_count):
        centres = rng.normal(size=(16, 3))
        centres /= np.linalg.norm(centres, axis=1, keepdims=True)
        amps = rng.normal(size=16)
        widths = rng.uniform(0.3, 0.6, size=16)
        field = np.zeros(n)
        for m in range(16):
            d2 = np.sum((unit_pts - centres[m]) ** 2, axis=1)
            field += amps[m] * np.exp(-d2 / (2.0 * widths[m] ** 2))
        disp = field[:, None] * normals
        rms = np.sqrt(np.mean(np.sum(disp * disp, axis=1)))
        cols[k] = disp * (rms0 / (1.0 + k) / max(rms, 1e-12))
    return cols


def face_icosphere(rng, level=4, n_shape=20, n_expr=0):
    """Closed 'face' mesh: icosphere warped into an ellipsoidal head with relief.

    Level 4 gives 2,562 vertices / 5,120 triangles."""
    p, faces = icosphere(level)
    radial = 1.0 + _face_features(p)
    scale = np.array([0.75, 0.95, 0.70])
    mean = p * radial[:, None] * scale
    uv = np.stack([(p[:, 0] + 1.0) * 0.5, (1.0 - p[:, 1]) * 0.5], axis=1)
    basis = _rbf_columns(rng, p, p, n_shape + n_expr, 0.05)
    return mean, basis, faces, uv


def bisect_edges(p, faces, n_edges, rng):
    """Bisect `n_edges` edges of a closed mesh on the unit sphere, no two of
    them on a common triangle: the new vertex is the edge midpoint pushed back
    onto the sphere, and each of the edge's two triangles splits in two
    (orientation kept), so the mesh gains n_edges vertices and 2 n_edges
    triangles.  Edges are taken in a seeded random order."""
    faces = [tuple(int(x) for x in f) for f in faces]
    owner = {}                                   # directed edge (a, b) -> face
    for fi, (a, b, c) in enumerate(faces):
        owner[(a, b)] = fi
        owner[(b, c)] = fi
        owner[(c, a)] = fi
    undirected = sorted((a, b) for (a, b) in owner if a < b)
    used = np.zeros(len(faces), dtype=bool)
    verts = [q for q in np.asarray(p, dtype=np.float64)]
    done = 0
    for idx in rng.permutation(len(undirected)):
        if done == n_edges:
            break
        a, b = undirected[idx]
        f1, f2 = owner[(a, b)], owner[(b, a)]
        if used[f1] or used[f2]:
            continue
        used[f1] = used[f2] = True
        q = verts[a] + verts[b]
        verts.append(q / np.linalg.norm(q))
        m = len(verts) - 1
        for f, (s, t) in ((f1, (a, b)), (f2, (b, a))):
            tri = faces[f]
            k = tri.index(s)                     # rotate so the triangle reads (s, t, o)
            o = tri[(k + 2) % 3]
            faces[f] = (s, m, o)
            faces.append((m, t, o))
        done += 1
    if done != n_edges:
        raise ValueError("not enough independent edges")
    return np.array(verts), np.array(faces, dtype=np.int32)


def face_subdivided(rng, n_triangles=100_000, level=6, n_shape=20):
    """The level-4 head of face_icosphere refined to `n_triangles`: the
    icosphere is subdivided to `level` (81,920 triangles at level 6), then
    (n_triangles - 20 * 4^level) / 2 independent edges are bisected, and the
    head warp, UVs and shape basis are applied to the refined sphere.
    100,000 triangles give 50,002 vertices."""
    p, faces = icosphere(level)
    extra = n_triangles - faces.shape[0]
    if extra < 0 or extra % 2:
        raise ValueError("n_triangles - 20 * 4^level must be even and >= 0")
    p, faces = bisect_edges(p, faces, extra // 2, rng)
    radial = 1.0 + _face_features(p)
    scale = np.array([0.75, 0.95, 0.70])
    mean = p * radial[:, None] * scale
    uv = np.stack([(p[:, 0] + 1.0) * 0.5, (1.0 - p[:, 1]) * 0.5], axis=1)
    basis = _rbf_columns(rng, p, p, n_shape, 0.05)
    return mean, basis, faces, uv


def _disk_rings(n_vertices, n_boundary):
    """Ring sizes (centre vertex excluded) for a disk mesh with exactly
    n_vertices vertices and n_boundary vertices on the outer ring."""
    target = n_vertices - 1
    sizes = []
    i = 1
    while True:
        s = min(6 * i, n_boundary)
        rest = target - sum(sizes)
        if rest - s < n_boundary:
            break
        sizes.append(s)
        i += 1
    rest = target - sum(sizes)
    # rest >= n_boundary here; close with rings of n_boundary and one filler ring
    fill = rest - n_boundary
    while fill > n_boundary:
        sizes.append(n_boundary)
        fill -= n_boundary
    if fill > 0:
        if fill < 3:            # merge a too-small filler into the previous ring
            sizes[-1] += fill
        else:
            sizes.append(fill)
            sizes.sort()
    sizes.append(n_boundary)
    assert sum(sizes) == target
    return sizes


def face_disk(rng, n_vertices=35709, n_boundary=627, n_shape=80, n_expr=64):
    """Open disk-topology height-field face.

    Concentric rings around a centre vertex, stitched by angle.  With V
    vertices and b boundary vertices a disk triangulation has 2V - b - 2
    triangles, so (35,709, 627) gives 70,789 triangles and, by Euler's formula,
    106,497 edges."""
    sizes = _disk_rings(n_vertices, n_boundary)
    n_rings = len(sizes)
    xs, ys = [0.0], [0.0]
    ring_start = []
    angles = []
    for r, n in enumerate(sizes):
        rad = (r + 1) / n_rings
        phase = 0.5 * (r % 2) * 2.0 * math.pi / n
        a = phase + 2.0 * math.pi * np.arange(n) / n
        ring_start.append(len(xs))
        angles.append(a)
        xs += list(rad * np.cos(a))
        ys += list(rad * np.sin(a))
    X = np.array(xs)
    Y = np.array(ys)
    faces = []
    n1 = sizes[0]
    for j in range(n1):
        faces.append((0, ring_start[0] + j, ring_start[0] + (j + 1) % n1))
    for r in range(n_rings - 1):
        na, nb = sizes[r], sizes[r + 1]
        sa, sb = ring_start[r], ring_start[r + 1]
        pa, pb = angles[r][0], angles[r + 1][0]
        ia = ib = 0
        while ia < na or ib < nb:
            next_a = pa + 2.0 * math.pi * (ia + 1) / na
            next_b = pb + 2.0 * math.pi * (ib + 1) / nb
            if ib >= nb or (ia < na and next_a <= next_b):
                faces.append((sa + ia % na, sb + ib % nb, sa + (ia + 1) % na))
                ia += 1
            else:
                faces.append((sa + ia % na, sb + ib % nb, sb + (ib + 1) % nb))
                ib += 1
    faces = np.array(faces, dtype=np.int32)
    # counter-clockwise seen from +z
    e1 = np.stack([X[faces[:, 1]] - X[faces[:, 0]], Y[faces[:, 1]] - Y[faces[:, 0]]], 1)
    e2 = np.stack([X[faces[:, 2]] - X[faces[:, 0]], Y[faces[:, 2]] - Y[faces[:, 0]]], 1)
    cz = e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0]
    flip = cz < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    # height field: dome plus facial relief
    r2 = X * X + Y * Y
    dome = 0.55 * np.sqrt(np.maximum(1.0 - 0.85 * r2, 0.0))
    unit = np.stack([X, Y, np.sqrt(np.maximum(1.0 - np.minimum(r2, 1.0), 0.0))], 1)
    relief = _face_features(unit)
    Z = dome + 0.9 * relief
    mean = np.stack([0.75 * X, 0.95 * Y, Z], 1)
    uv = np.stack([(X + 1.0) * 0.5, (1.0 - Y) * 0.5], axis=1)
    normals = np.tile(np.array([0.0, 0.0, 1.0]), (X.shape[0], 1))
    basis = _rbf_columns(rng, unit, normals, n_shape + n_expr, 0.05)
    return mean, basis, faces, uv


# --------------------------------------------------------------------------
# lights, textures, parameters
# --------------------------------------------------------------------------

def _fibonacci_dirs(n, hemisphere):
    g = math.pi * (3.0 - math.sqrt(5.0))
    out = []
    for i in range(n):
        z = 1.0 - (i + 0.5) / n if hemisphere else 1.0 - (2.0 * i + 1.0) / n
        r = math.sqrt(max(0.0, 1.0 - z * z))
        out.append((r * math.cos(g * i), r * math.sin(g * i), z))
    return np.array(out)


def light_stage(n_lights, radius=3.0, side=0.5, hemisphere=False,
                centre=STAGE_CENTRE, kind=LIGHT_QUAD):
    """Area lights on a (hemi)sphere around the head, each facing the centre."""
    dirs = _fibonacci_dirs(n_lights, hemisphere)
    c0 = np.asarray(centre, dtype=np.float64)
    rec = np.zeros((n_lights, 11), dtype=np.float32)
    for j, dvec in enumerate(dirs):
        inward = -dvec
        up = np.array([0.0, 1.0, 0.0]) if abs(inward[1]) < 0.9 else np.array([1.0, 0.0, 0.0])
        a1 = np.cross(up, inward)
        a1 /= np.linalg.norm(a1)
        a2 = np.cross(inward, a1)          # a1 x a2 = inward
        c = c0 + radius * dvec
        if kind == LIGHT_QUAD:
            e1, e2 = side * a1, side * a2
        elif kind == LIGHT_DISK:
            e1, e2 = 0.5 * side * a1, 0.5 * side * a2
        else:  # triangle with centroid at c
            e1, e2 = side * a1, side * a2
            c = c - (e1 + e2) / 3.0
        rec[j, 0] = kind
        rec[j, 1:4] = c
        rec[j, 4:7] = e1
        rec[j, 7:10] = e2
    return rec


def env_blocks(env_size=32, block=4):
    """Emitter records splitting an env_size x env_size environment map into
    square blocks of block x block texels (one camera-sample direction per
    block), row-major over the blocks; d = a = 1."""
    if env_size % block:
        raise ValueError("block must divide env_size")
    nb = env_size // block
    rec = np.zeros((nb * nb, 11), np.float32)
    for bi in range(nb):
        for bj in range(nb):
            rec[bi * nb + bj, :5] = (LIGHT_ENV, bi * block, (bi + 1) * block, bj * block, (bj + 1) * block)
    n = rec.shape[0]
    return rec, np.ones(n, np.float32), np.ones(n, np.float32)


def env_map(rng, env_size=32, lo=0.1, hi=0.6, n_suns=2, sun=6.0):
    """Environment radiance [M_e, M_e, 3]: a smooth coloured field in [lo, hi]
    plus n_suns bright texels (sun x a random colour) in the upper front
    quarter of the sphere, so that shadows have sharp edges."""
    env = smooth_field(rng, env_size, 3, env_size / 8.0, lo, hi)
    for _ in range(n_suns):
        i = int(rng.integers(env_size // 8, env_size // 2))
        j = int(rng.integers(0, env_size // 4)) if rng.uniform() < 0.5 else int(rng.integers(3 * env_size // 4, env_size))
        env[i, j] += sun * rng.uniform(0.5, 1.0, size=3)
    return env.astype(np.float32)


def _polyhedron(name):
    """Unit-circumradius convex polyhedra with triangular faces, counter-
    clockwise seen from outside: tetrahedron (4 faces), octahedron (8),
    icosahedron (20) and the icosahedron subdivided once onto the sphere (80)."""
    if name == "tetra":
        v = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], np.float64)
        f = np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], np.int32)
    elif name == "octa":
        v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)
        f = np.array([[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4], [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]],
                     np.int32)
    elif name == "ico":
        v, f = icosphere(0)
    elif name == "sphere80":
        v, f = icosphere(1)
    else:
        raise ValueError(name)
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    # orient every face outwards
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    flip = np.sum(np.cross(b - a, c - a) * (a + b + c), axis=1) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def stage_records(stage, d=3.0, a=0.25, p=None):
    """Emitter records of a virtual light stage (Sec. 3.3) from its frame
    ([N_L, 12]: centre C, face V0, V1, V2 per light) and the lights'
    parameters: light j lies in face j's homothetic copy scaled by d_j about C,
    is that face shrunk by sqrt(a_j) (a_j = relative area in [0, 1]) around
    the point with barycentric coordinates p_j (default the centroid), stays
    parallel to the face and emits towards C.  Returns (records [N_L, 11] of
    type LIGHT_TRI, d [N_L], a [N_L])."""
    stage = np.asarray(stage, np.float64)
    n = stage.shape[0]
    d = np.broadcast_to(np.asarray(d, np.float64), (n,))
    a = np.broadcast_to(np.asarray(a, np.float64), (n,))
    p = np.full((n, 3), 1.0 / 3.0) if p is None else np.asarray(p, np.float64)
    if p.shape[1] == 2:
        p = np.concatenate([p, 1.0 - p.sum(axis=1, keepdims=True)], axis=1)
    rec = np.zeros((n, 11), np.float32)
    for j in range(n):
        c0, A, B, C = stage[j, 0:3], stage[j, 3:6], stage[j, 6:9], stage[j, 9:12]
        G = (A + B + C) / 3.0
        P = c0 + d[j] * (p[j, 0] * A + p[j, 1] * B + p[j, 2] * C)
        s = math.sqrt(a[j]) * d[j]
        # vertices in the order A, C, B so that e1 x e2 points inwards
        t0, t1, t2 = P + s * (A - G), P + s * (C - G), P + s * (B - G)
        rec[j, 0] = LIGHT_TRI
        rec[j, 1:4] = t0
        rec[j, 4:7] = t1 - t0
        rec[j, 7:10] = t2 - t0
    return rec, d.astype(np.float32).copy(), a.astype(np.float32).copy()


def polyhedral_stage(name="ico", d=3.0, a=0.25, p=None, centre=STAGE_CENTRE):
    """The virtual light stage of Sec. 3.3 on a convex polyhedron around the
    head (the paper's icosahedron: 20 lights; also the tetrahedron, octahedron
    and 80-face sphere variants it compares): stage_records of its frame."""
    return stage_records(polyhedral_stage_geometry(name, centre), d, a, p)


def polyhedral_stage_geometry(name="ico", centre=STAGE_CENTRE):
    """[N_L, 12] per light: the stage centre C and the unit-circumradius face
    vertices V0, V1, V2 of its polyhedron face (the frame d_j, a_j and p_j act
    in; see polyhedral_stage)."""
    v, f = _polyhedron(name)
    out = np.zeros((f.shape[0], 12), np.float32)
    out[:, 0:3] = centre
    out[:, 3:6], out[:, 6:9], out[:, 9:12] = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    return out


def smooth_field(rng, m, channels, sigma, lo, hi):
    """White noise blurred by a Gaussian of std `sigma` texels (periodic, FFT),
    rescaled per channel to [lo, hi]."""
    noise = rng.normal(size=(m, m, channels))
    f = np.fft.fftfreq(m)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (f[:, None] ** 2 + f[None, :] ** 2))
    out = np.empty_like(noise)
    for c in range(channels):
        out[:, :, c] = np.real(np.fft.ifft2(np.fft.fft2(noise[:, :, c]) * g))
        mn, mx = out[:, :, c].min(), out[:, :, c].max()
        out[:, :, c] = lo + (hi - lo) * (out[:, :, c] - mn) / max(mx - mn, 1e-12)
    return out


def textures(rng, m):
    diffuse = smooth_field(rng, m, 3, m / 16.0, 0.2, 0.8)
    specular = np.full((m, m, 3), 0.05)
    roughness = rng.uniform(0.3, 0.6, size=(m, m))
    return (diffuse.astype(np.float32), specular.astype(np.float32),
            roughness.astype(np.float32))


def _zero_mean_field(rng, m, sigma):
    """Smooth zero-mean random field [m, m, 3] with unit RMS (periodic blur)."""
    noise = rng.normal(size=(m, m, 3))
    f, fr = np.fft.fftfreq(m), np.fft.rfftfreq(m)
    g = np.exp(-2.0 * (math.pi * sigma) ** 2 * (f[:, None] ** 2 + fr[None, :] ** 2))
    out = np.fft.irfft2(np.fft.rfft2(noise, axes=(0, 1)) * g[:, :, None], s=(m, m), axes=(0, 1))
    out -= out.mean(axis=(0, 1), keepdims=True)
    return out / max(float(np.sqrt(np.mean(out * out))), 1e-12)


def albedo_model(rng, m, k_diffuse=80, k_specular=80):
    """Synthetic statistical albedo model: diffuse mean a smooth field in
    [0.35, 0.65] (skin-like, left-right symmetric), specular mean 0.05; column k
    a smooth zero-mean field of RMS 0.08 / (1 + k) (diffuse) and
    0.01 / (1 + k) (specular), so beta, gamma ~ N(0, 1) stay in range."""
    md = smooth_field(rng, m, 3, m / 16.0, 0.35, 0.65)
    md = 0.5 * (md + md[:, ::-1, :])
    bd = np.empty((k_diffuse, m, m, 3), np.float32)
    for k in range(k_diffuse):
        bd[k] = _zero_mean_field(rng, m, m / 24.0) * (0.08 / (1.0 + k))
    ms = np.full((m, m, 3), 0.05, np.float32)
    bs = np.empty((k_specular, m, m, 3), np.float32)
    for k in range(k_specular):
        bs[k] = _zero_mean_field(rng, m, m / 24.0) * (0.01 / (1.0 + k))
    return AlbedoModel(mean_diffuse=md.astype(np.float32), basis_diffuse=bd,
                       mean_specular=ms, basis_specular=bs)


def landmark_vertices(mean, n=68):
    """L landmark vertices on the front of the face (the paper uses L = 68
    detector landmarks): the frontmost half of the vertices (largest z), then
    farthest-point sampling in the image plane starting next to the centre, so
    they spread over the face like a detector's contour, brow, eye, nose and
    mouth points.  Deterministic."""
    c = np.asarray(mean, np.float64) - np.mean(mean, axis=0)
    front = np.nonzero(c[:, 2] >= np.quantile(c[:, 2], 0.5))[0]
    pts = c[front, :2]
    sel = [int(np.argmin(np.sum(pts * pts, axis=1)))]
    d = np.sum((pts - pts[sel[0]]) ** 2, axis=1)
    for _ in range(min(n, front.size) - 1):
        j = int(np.argmax(d))
        sel.append(j)
        d = np.minimum(d, np.sum((pts - pts[j]) ** 2, axis=1))
    return front[np.array(sel)].astype(np.int32)


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def make_scene(config: str = "c1", seed: int = 0, **over) -> Scene:
    """Scenes shaped like the workloads:

    c1   : 2,562 verts / 5,120 tris, K = 20, 64x64, 4 spp, 8 quads on a
           hemisphere of radius 3, 128^2 textures.
    c2   : 35,709 verts / 70,789 tris, K = 80 + 64, 256x256, 16 spp,
           40 quads on a sphere, 512^2 textures.
    c5   : 50,002 verts / 100,000 tris refined from the c1 head, K = 20,
           1024x1024, 64 spp, 80 quads on a sphere, 2048^2 textures.
    tiny : a small closed mesh for fast CPU tests (162 verts / 320 tris, K = 6,
           24x24, 2 spp, 4 lights).
    Keyword overrides replace width/height/spp/tex_size/n_lights/light kind;
    light_stage = "tetra" | "octa" | "ico" | "sphere80" replaces the lights by
    the polyhedral virtual light stage of Sec. 3.3 (light_area = a_j);
    albedo_k > 0 adds a statistical albedo model with that many columns per
    albedo (Sec. 3.2; the paper's K_r = K_b = 80); env = (M_e, block) replaces
    the lights by an M_e x M_e environment map in blocks of block x block
    texels (Sec. 7; the paper's map is 32 x 32)."""
    rng = np.random.default_rng(seed)
    if config == "c1":
        mean, basis, faces, uv = face_icosphere(rng, 4, 20, 0)
        ks, ke = 20, 0
        w = h = 64
        spp, m, nl, hemi = 4, 128, 8, True
    elif config == "c2":
        mean, basis, faces, uv = face_disk(rng, 35709, 627, 80, 64)
        ks, ke = 80, 64
        w = h = 256
        spp, m, nl, hemi = 16, 512, 40, False
    elif config == "c5":
        mean, basis, faces, uv = face_subdivided(rng, 100_000, 6, 20)
        ks, ke = 20, 0
        w = h = 1024
        spp, m, nl, hemi = 64, 2048, 80, False
    elif config == "tiny":
        mean, basis, faces, uv = face_icosphere(rng, 2, 4, 2)
        ks, ke = 4, 2
        w = h = 24
        spp, m, nl, hemi = 2, 16, 4, True
    else:
        raise ValueError(config)
    w = over.get("width", w)
    h = over.get("height", h)
    spp = over.get("spp", spp)
    m = over.get("tex_size", m)
    nl = over.get("n_lights", nl)
    kind = over.get("light_kind", LIGHT_QUAD)
    side = over.get("light_side", 0.5 if kind != LIGHT_DISK else 1.0)
    stage = over.get("light_stage")
    stage_geo = None
    env = over.get("env")                 # (M_e, block): environment map of lights at infinity
    env_size = 0
    if env is not None:
        env_size = int(env[0])
        lights, light_d, light_a = env_blocks(env_size, int(env[1]))
        nl = lights.shape[0]
    elif stage is not None:                 # polyhedral stage: "tetra", "octa", "ico", "sphere80"
        lights, light_d, light_a = polyhedral_stage(stage, 3.0, over.get("light_area", 0.25))
        stage_geo = polyhedral_stage_geometry(stage)
        nl = lights.shape[0]
    else:
        lights = light_stage(nl, 3.0, side, hemi, STAGE_CENTRE, kind)
        light_d, light_a = np.full(nl, 3.0, np.float32), np.ones(nl, np.float32)
    ka = int(over.get("albedo_k", 0))
    albedo = albedo_model(np.random.default_rng(seed + 31), m, ka, ka) if ka > 0 else None
    return Scene(mean=_f32(mean), basis=_f32(basis), n_shape=ks, n_expr=ke,
                 faces=np.ascontiguousarray(faces.astype(np.int32)), uv=_f32(uv),
                 lights=lights, light_d=light_d, light_a=light_a, width=int(w), height=int(h),
                 spp=int(spp), tex_size=int(m), fov_deg=30.0, albedo=albedo,
                 landmarks=landmark_vertices(mean), stage=stage_geo, env_size=env_size)


def init_params(scene: Scene, seed: int = 0) -> Params:
    """Optimisation start: mean shape, neutral expression, frontal pose,
    uniform lights, flat textures (Sec. 4 initialisation)."""
    rng = np.random.default_rng(seed + 1000)
    m = scene.tex_size
    del rng
    return Params(coef=np.zeros(scene.n_basis, np.float32),
                  rot=np.zeros(3, np.float32),
                  trans=np.array(DEFAULT_T, np.float32),
                  focal=np.array([scene.focal_px()], np.float32),
                  light_i=np.full((scene.n_lights, 3), 0.8, np.float32),
                  diffuse=np.full((m, m, 3), 0.5, np.float32),
                  specular=np.full((m, m, 3), 0.05, np.float32),
                  roughness=np.full((m, m), 0.45, np.float32),
                  env=(np.full((scene.env_size, scene.env_size, 3), 0.3, np.float32)
                       if scene.env_size else None))


def random_params(scene: Scene, seed: int = 0, coef_scale: float = 1.0) -> Params:
    """Ground-truth parameters for a synthetic target image."""
    rng = np.random.default_rng(seed + 7)
    m = scene.tex_size
    coef = np.zeros(scene.n_basis)
    coef[:scene.n_shape] = rng.normal(size=scene.n_shape) * coef_scale
    coef[scene.n_shape:] = rng.uniform(0.0, 0.5, size=scene.n_expr)
    diffuse, specular, roughness = textures(rng, m)
    return Params(coef=_f32(coef),
                  rot=_f32(rng.uniform(-0.04, 0.04, size=3)),
                  trans=_f32(np.array(DEFAULT_T) + rng.normal(0.0, 0.03, size=3)),
                  focal=_f32([scene.focal_px()]),
                  light_i=_f32(rng.uniform(0.2, 1.5, size=(scene.n_lights, 3))),
                  diffuse=diffuse, specular=specular, roughness=roughness,
                  env=(env_map(np.random.default_rng(seed + 53), scene.env_size)
                       if scene.env_size else None))


def with_stage_geometry(scene: Scene, params: Params, seed: int | None = None) -> Params:
    """A copy of params whose lights are built from the virtual light stage's
    parameters (d_j, a_j, p_j): the stage defaults (d 3, a 0.25, centroid), or
    a seeded perturbation of them (d 3 +- 0.3, a in [0.15, 0.45], p inside the
    face)."""
    if scene.stage is None:
        raise ValueError("scene has no polyhedral light stage")
    q = params.copy()
    n = scene.n_lights
    if seed is None:
        q.light_d = np.full(n, 3.0, np.float32)
        q.light_a = np.full(n, 0.25, np.float32)
        q.light_p = np.full((n, 2), 1.0 / 3.0, np.float32)
    else:
        rng = np.random.default_rng(seed + 91)
        q.light_d = _f32(3.0 + rng.uniform(-0.3, 0.3, n))
        q.light_a = _f32(rng.uniform(0.15, 0.45, n))
        q.light_p = _f32(rng.dirichlet([6.0, 6.0, 6.0], size=n)[:, :2])
    return q


def pixel_noise(rng_seed: int, shape, sigma: float = 0.01) -> np.ndarray:
    """N(0, sigma) pixel noise added to synthetic targets."""
    return _f32(np.random.default_rng(rng_seed).normal(0.0, sigma, size=shape))
