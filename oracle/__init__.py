"""FP64 CPU oracle for the differentiable ray-traced face render.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg.  The product path (the CUDA library and
its Python binding) never imports it, and it shares no code with them.

The arithmetic lives in ``oracle.cpp`` (plain C++17, double precision,
brute-force intersection, forward-mode dual numbers); this module compiles it
with g++ on first use and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.cpp")
LIB = os.path.join(HERE, "liboracle.so")

GGX, SCHLICK_LINEAR, FLAT, DIFFUSE_ONLY = 1, 2, 4, 8
VIEW_CUTOFF = 1024      # the literal grazing reading: every contribution zero where n_s . o <= 0
TERM_INTERIOR, TERM_PRIMARY, TERM_SHADOW = 1, 2, 4
TERM_SPECULAR = 8       # boundary of the specular lobe inside triangles (the curve n_s . o = 0)
TERM_ALL = 15

_lock = threading.Lock()
_lib = None

f32p = ctypes.POINTER(ctypes.c_float)
f64p = ctypes.POINTER(ctypes.c_double)
i32p = ctypes.POINTER(ctypes.c_int32)
u64p = ctypes.POINTER(ctypes.c_uint64)
u32p = ctypes.POINTER(ctypes.c_uint32)


class OraScene(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32),
                ("n_basis", ctypes.c_int32), ("mean", f32p), ("basis", f32p),
                ("faces", i32p), ("uv", f32p), ("n_lights", ctypes.c_int32),
                ("lights", f32p), ("light_d", f32p), ("light_a", f32p),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("spp", ctypes.c_int32), ("tex_size", ctypes.c_int32),
                ("edge_spp", ctypes.c_int32), ("seed", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("n_threads", ctypes.c_int32), ("stage", f32p),
                ("env_size", ctypes.c_int32)]


class OraParams(ctypes.Structure):
    _fields_ = [(n, f32p) for n in ("coef", "rot", "trans", "focal", "light_i",
                                    "diffuse", "specular", "roughness", "light_d", "light_a", "light_p",
                                    "env")]


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (g++, -O2)."""
    with _lock:
        if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            tmp = LIB + ".tmp.%d" % os.getpid()
            cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
                   "-o", tmp, SRC]
            subprocess.run(cmd, check=True)
            os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.ora_philox.argtypes = [ctypes.c_uint32] * 6 + [u32p]
        L.ora_ray_count.argtypes = [ctypes.c_int]
        L.ora_ray_count.restype = ctypes.c_ulonglong
        L.ora_geometry.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams), f64p, f64p]
        L.ora_edges.argtypes = [ctypes.POINTER(OraScene), i32p, i32p]
        L.ora_silhouettes.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams),
                                      i32p, i32p, i32p, i32p]
        L.ora_closest_hit.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams),
                                      f64p, f64p, ctypes.c_int32, i32p, f64p]
        L.ora_render.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams),
                                 ctypes.c_uint32, ctypes.c_uint32, i32p, ctypes.c_int32,
                                 f64p, i32p, u64p]
        L.ora_loss.argtypes = [ctypes.c_int32, ctypes.c_int32, f64p, f32p, f64p, f64p]
        L.ora_loss.restype = ctypes.c_double
        L.ora_grad.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams),
                               ctypes.c_uint32, ctypes.c_uint32, f64p, ctypes.c_uint32] + [f64p] * 10
        L.ora_brdf.argtypes = [ctypes.c_uint32, f64p, f64p, f64p, f64p, f64p, ctypes.c_double, f64p]
        L.ora_brdf.restype = ctypes.c_double
        L.ora_brdf_terms.argtypes = [ctypes.c_uint32, f64p, f64p, f64p, ctypes.c_double, f64p]
        L.ora_point_light_grad.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams),
                                           f64p, f64p, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_uint32, f64p, f64p, f64p]
        L.ora_spec_crossings.argtypes = [ctypes.POINTER(OraScene), ctypes.POINTER(OraParams), ctypes.c_uint32,
                                         ctypes.c_uint32, ctypes.c_int32, ctypes.c_int32, i32p, f64p]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _c32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class _Bound:
    """Keeps the numpy arrays behind the ctypes structs alive."""

    def __init__(self, scene, params, flags=0, edge_spp=1, seed=0, n_threads=0):
        self.keep = []

        def f(a):
            a = _c32(a)
            self.keep.append(a)
            return a.ctypes.data_as(f32p)

        faces = np.ascontiguousarray(scene.faces, dtype=np.int32)
        self.keep.append(faces)
        self.scene = OraScene(
            scene.n_vertices, scene.n_triangles, scene.n_basis, f(scene.mean),
            f(scene.basis), faces.ctypes.data_as(i32p), f(scene.uv), scene.n_lights,
            f(scene.lights), f(scene.light_d), f(scene.light_a), scene.width, scene.height,
            scene.spp, scene.tex_size, edge_spp, seed, flags, n_threads,
            f(scene.stage) if getattr(scene, "stage", None) is not None else None,
            int(getattr(scene, "env_size", 0) or 0))
        self.params = None
        if params is not None:
            def opt(name):
                x = getattr(params, name, None)
                return f(x) if x is not None else None
            self.params = OraParams(f(params.coef), f(params.rot), f(params.trans),
                                    f(params.focal), f(params.light_i), f(params.diffuse),
                                    f(params.specular), f(params.roughness), opt("light_d"), opt("light_a"),
                                    opt("light_p"), opt("env"))


def ray_count(reset=False):
    """Rays (camera, shadow and edge) traced by the oracle since the last reset."""
    return int(lib().ora_ray_count(1 if reset else 0))


def philox(k0, k1, c0, c1, c2, c3):
    out = np.zeros(4, np.uint32)
    lib().ora_philox(k0, k1, c0, c1, c2, c3, out.ctypes.data_as(u32p))
    return out


def geometry(scene, params):
    b = _Bound(scene, params)
    v = np.zeros((scene.n_vertices, 3))
    n = np.zeros((scene.n_vertices, 3))
    lib().ora_geometry(ctypes.byref(b.scene), ctypes.byref(b.params), _p(v, f64p), _p(n, f64p))
    return v, n


def edges(scene):
    b = _Bound(scene, None)
    n_e = scene.n_vertices + scene.n_triangles + 2 * scene.n_triangles  # upper bound
    ev = np.zeros((n_e, 2), np.int32)
    ef = np.zeros((n_e, 2), np.int32)
    m = lib().ora_edges(ctypes.byref(b.scene), _p(ev, i32p), _p(ef, i32p))
    return ev[:m].copy(), ef[:m].copy()


def silhouettes(scene, params):
    """Ordered primary silhouette edge list and per-light shadow candidate lists."""
    b = _Bound(scene, params)
    n_e = len(edges(scene)[0])
    prim = np.zeros(n_e, np.int32)
    n_prim = np.zeros(1, np.int32)
    per = np.zeros((scene.n_lights, n_e), np.int32)
    cnt = np.zeros(scene.n_lights, np.int32)
    lib().ora_silhouettes(ctypes.byref(b.scene), ctypes.byref(b.params), _p(prim, i32p),
                          _p(n_prim, i32p), _p(per, i32p), _p(cnt, i32p))
    return prim[:n_prim[0]].copy(), [per[j, :cnt[j]].copy() for j in range(scene.n_lights)]


def closest_hit(scene, params, org, dirs, n_threads=0):
    b = _Bound(scene, params, n_threads=n_threads)
    org = np.ascontiguousarray(org, np.float64)
    dirs = np.ascontiguousarray(dirs, np.float64)
    n = org.shape[0]
    tri = np.zeros(n, np.int32)
    t = np.zeros(n)
    lib().ora_closest_hit(ctypes.byref(b.scene), ctypes.byref(b.params), _p(org, f64p),
                          _p(dirs, f64p), n, _p(tri, i32p), _p(t, f64p))
    return tri, t


def render(scene, params, iteration=0, face_id=0, pixels=None, flags=0, seed=0,
           records=False, n_threads=0):
    """Forward render [H, W, 3] (float64); with records also the per-sample hit
    triangle [H*W*spp] and shadow visibility masks [H*W*spp, 2] (bit j of word
    w: the shadow ray to light 64 w + j was traced and is unoccluded)."""
    b = _Bound(scene, params, flags=flags, seed=seed, n_threads=n_threads)
    img = np.zeros((scene.height, scene.width, 3))
    n_rec = scene.height * scene.width * scene.spp
    tri = np.full(n_rec, -2, np.int32) if records else None
    mask = np.zeros((n_rec, 2), np.uint64) if records else None
    pix = None if pixels is None else np.ascontiguousarray(pixels, np.int32)
    lib().ora_render(ctypes.byref(b.scene), ctypes.byref(b.params), iteration, face_id,
                     _p(pix, i32p), 0 if pix is None else len(pix), _p(img, f64p),
                     _p(tri, i32p), _p(mask, u64p))
    return (img, tri, mask) if records else img


def loss(image, target):
    """(E_ph of the blurred image, blurred image, adjoint image dE/dimage)."""
    image = np.ascontiguousarray(image, np.float64)
    target = _c32(target)
    h, w = image.shape[:2]
    bl = np.zeros_like(image)
    adj = np.zeros_like(image)
    val = lib().ora_loss(h, w, _p(image, f64p), _p(target, f32p), _p(bl, f64p), _p(adj, f64p))
    return val, bl, adj


def grad(scene, params, adjoint, iteration=0, face_id=0, terms=TERM_ALL, flags=0, seed=0,
         edge_spp=1, n_threads=0):
    """Gradient of sum(adjoint * image) w.r.t. every parameter group (float64)."""
    b = _Bound(scene, params, flags=flags, edge_spp=edge_spp, seed=seed, n_threads=n_threads)
    adj = np.ascontiguousarray(adjoint, np.float64)
    m = scene.tex_size
    g = dict(coef=np.zeros(scene.n_basis), rot=np.zeros(3), trans=np.zeros(3),
             focal=np.zeros(1), light_i=np.zeros((scene.n_lights, 3)),
             diffuse=np.zeros((m, m, 3)), specular=np.zeros((m, m, 3)),
             roughness=np.zeros((m, m)))
    geom = getattr(scene, "stage", None) is not None and getattr(params, "light_d", None) is not None
    lg = np.zeros((scene.n_lights, 4))
    me = int(getattr(scene, "env_size", 0) or 0)
    if me:   # environment-map radiance [M_e, M_e, 3]
        g["env"] = np.zeros((me, me, 3))
    rc = lib().ora_grad(ctypes.byref(b.scene), ctypes.byref(b.params), iteration, face_id,
                        _p(adj, f64p), terms, *[_p(g[k], f64p) for k in
                                                ("coef", "rot", "trans", "focal", "light_i",
                                                 "diffuse", "specular", "roughness")],
                        _p(lg, f64p) if geom else None, _p(g.get("env"), f64p))
    if geom:   # d/d(d_j, a_j, p_j0, p_j1) of the virtual light stage
        g["light_d"], g["light_a"], g["light_p"] = lg[:, 0].copy(), lg[:, 1].copy(), lg[:, 2:].copy()
    if rc != 0:
        raise ValueError("oracle gradient: unsupported sizes")
    return g


def spec_crossings(scene, params, scan, iteration=0, face_id=0, edge_spp=1, seed=0, max_count=4096):
    """Crossings of image scanline `scan` (rows first, then columns) with the
    curve n_s . o = 0 inside front-facing triangles: ([n, 2] (triangle, root
    index along the line), [n, 2] screen (x, y))."""
    b = _Bound(scene, params, edge_spp=edge_spp, seed=seed)
    tr = np.zeros((max_count, 2), np.int32)
    xy = np.zeros((max_count, 2))
    n = lib().ora_spec_crossings(ctypes.byref(b.scene), ctypes.byref(b.params), iteration, face_id, scan,
                                 max_count, _p(tr, i32p), _p(xy, f64p))
    if n < 0:
        raise ValueError("scanline out of range")
    return tr[:min(n, max_count)].copy(), xy[:min(n, max_count)].copy()


def brdf(n, l, o, c, s, r, flags=0):
    arrs = [np.ascontiguousarray(x, np.float64) for x in (n, l, o, c, s)]
    out = np.zeros(3)
    lib().ora_brdf(flags, *[_p(a, f64p) for a in arrs], float(r), _p(out, f64p))
    return out


def brdf_terms(n, l, o, r, flags=0):
    """(D, G1(o), G1(l), Schlick weight) of the specular lobe."""
    arrs = [np.ascontiguousarray(x, np.float64) for x in (n, l, o)]
    out = np.zeros(4)
    lib().ora_brdf_terms(flags, *[_p(a, f64p) for a in arrs], float(r), _p(out, f64p))
    return out


def point_light_grad(scene, params, y, n, n_samples, tri_self=-1, stream=7, seed=0,
                     n_threads=0):
    """Light integral of a white Lambertian point and its shadow-boundary
    derivative w.r.t. the shape coefficients (occluder motion)."""
    b = _Bound(scene, params, seed=seed, n_threads=n_threads)
    y = np.ascontiguousarray(y, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    val = np.zeros(3)
    g = np.zeros(scene.n_basis)
    lg = np.zeros((scene.n_lights, 4))
    geom = getattr(scene, "stage", None) is not None and getattr(params, "light_d", None) is not None
    lib().ora_point_light_grad(ctypes.byref(b.scene), ctypes.byref(b.params), _p(y, f64p),
                               _p(n, f64p), tri_self, n_samples, stream, _p(val, f64p),
                               _p(g, f64p), _p(lg, f64p) if geom else None)
    if geom:   # channel-0 derivatives w.r.t. each light's (d, a, p0, p1)
        return val, g, lg
    return val, g
