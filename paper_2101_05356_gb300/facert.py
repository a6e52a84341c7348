"""Thin ctypes binding of libfacert.so (include/facert.h), same call names.

Only argument marshalling lives here: every step of the render, the loss and
the adjoint runs in the library's CUDA kernels.  PyTorch provides device memory
and the current stream.  Importing this module does not need a GPU; loading the
library fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfacert.so")

FR_OK, FR_EINVAL, FR_ENOMEM, FR_ECUDA, FR_EOVERFLOW, FR_ETIMEOUT = 0, 1, 2, 3, 4, 5
FLAG_GGX, FLAG_SCHLICK_LINEAR, FLAG_FLAT = 1, 2, 4
FLAG_NO_INTERIOR, FLAG_NO_PRIMARY_EDGE, FLAG_NO_SHADOW_EDGE = 16, 32, 64
FLAG_NO_SPECULAR_EDGE = 2048
FLAG_MORPH_BF16 = 128
FLAG_RECOMPUTE = 256
FLAG_LBVH = 512
FLAG_VIEW_CUTOFF = 1024
# emitter types of the light records (FR_LIGHT_*)
LIGHT_QUAD, LIGHT_TRI, LIGHT_DISK, LIGHT_ENV = 0, 1, 2, 3
FR_MAX_ENV = 64

_vp = ctypes.c_void_p


class FrConfig(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("spp", ctypes.c_int32),
                ("tex_size", ctypes.c_int32), ("edge_spp", ctypes.c_int32),
                ("flags", ctypes.c_uint32), ("seed", ctypes.c_uint32), ("max_batch", ctypes.c_int32)]


class FrMesh(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32),
                ("n_basis", ctypes.c_int32), ("mean", _vp), ("basis", _vp), ("faces", _vp),
                ("uv", _vp)]


class FrLightStage(ctypes.Structure):
    _fields_ = [("n_lights", ctypes.c_int32), ("records", _vp), ("d", _vp), ("a", _vp), ("stage", _vp),
                ("env_size", ctypes.c_int32)]


class FrAlbedoModel(ctypes.Structure):
    _fields_ = [("k_diffuse", ctypes.c_int32), ("k_specular", ctypes.c_int32), ("mean_diffuse", _vp),
                ("basis_diffuse", _vp), ("mean_specular", _vp), ("basis_specular", _vp)]


PARAM_NAMES = ("coef", "rot", "trans", "focal", "light_i", "diffuse", "specular", "roughness")
# optional light-stage geometry (Sec. 3.3): distance, relative area, barycentric centre
STAGE_NAMES = ("light_d", "light_a", "light_p")
# environment-map radiance [M_e, M_e, 3] (lights at infinity, Sec. 7)
ENV_NAMES = ("env",)
ALL_PARAM_NAMES = PARAM_NAMES + STAGE_NAMES + ENV_NAMES


class FrParams(ctypes.Structure):
    _fields_ = [(n, _vp) for n in ALL_PARAM_NAMES]


class FrGrads(ctypes.Structure):
    _fields_ = [(n, _vp) for n in ALL_PARAM_NAMES]


GROUP_PLAIN, GROUP_COEF, GROUP_LIGHT, GROUP_TEX_RGB, GROUP_TEX_MONO, GROUP_STAGE = 0, 1, 2, 3, 4, 5


class FrOptGroup(ctypes.Structure):
    _fields_ = [("x", _vp), ("g", _vp), ("m", _vp), ("v", _vp), ("aux", _vp), ("aux2", _vp),
                ("n", ctypes.c_int32), ("kind", ctypes.c_int32), ("width", ctypes.c_int32),
                ("n_prior", ctypes.c_int32), ("lr", ctypes.c_float), ("w_prior", ctypes.c_float),
                ("w_box", ctypes.c_float), ("w_sym", ctypes.c_float), ("w_chroma", ctypes.c_float),
                ("w_smooth", ctypes.c_float), ("clamp_lo", ctypes.c_float), ("clamp_hi", ctypes.c_float),
                ("step", ctypes.c_int32)]


class FrItem(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("spp", ctypes.c_int32),
                ("edge_spp", ctypes.c_int32), ("flags", ctypes.c_uint32), ("iteration", ctypes.c_uint32),
                ("face_id", ctypes.c_uint32), ("params", FrParams), ("target", _vp), ("image", _vp),
                ("loss", _vp), ("grads", ctypes.POINTER(FrGrads))]


class FrServerConfig(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int32), ("mem_cap_bytes", ctypes.c_uint64), ("n_identity", ctypes.c_int32),
                ("edge_spp", ctypes.c_int32), ("item_flags", ctypes.c_uint32), ("eval_iteration", ctypes.c_uint32),
                ("eval_spp", ctypes.c_int32), ("keep_params", ctypes.c_int32)]


class FrRequest(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("spp", ctypes.c_int32),
                ("init_iters", ctypes.c_int32), ("stage1_iters", ctypes.c_int32), ("stage2_iters", ctypes.c_int32),
                ("target", _vp), ("init", FrParams), ("landmarks", _vp), ("n_landmarks", ctypes.c_int32)]


class FrResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("iterations", ctypes.c_int32), ("final_loss", ctypes.c_double),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("finish_s", ctypes.c_double),
                ("error", ctypes.c_char * 128)]


class FrServerStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("item_steps", ctypes.c_int64), ("max_active", ctypes.c_int32),
                ("active", ctypes.c_int32), ("queued", ctypes.c_int32), ("peak_bytes", ctypes.c_uint64),
                ("used_bytes", ctypes.c_uint64), ("finished", ctypes.c_uint64)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED = 0, 1, 2, 3
FR_EAGAIN = 6


class FacertError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("facert error %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib():
    """Load libfacert.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfacert.so is missing: build it with __graft_entry__.build() "
                               "(nvcc for sm_103a); there is no fallback path")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        L.fr_create.argtypes = [P(_vp), P(FrConfig)]
        L.fr_set_mesh.argtypes = [_vp, P(FrMesh)]
        L.fr_set_lights.argtypes = [_vp, P(FrLightStage)]
        L.fr_set_albedo.argtypes = [_vp, P(FrAlbedoModel)]
        L.fr_set_landmarks.argtypes = [_vp, ctypes.c_int32, _vp]
        L.fr_landmark_loss.argtypes = [_vp, P(FrParams), ctypes.c_int32, ctypes.c_int32, _vp, ctypes.c_float, _vp,
                                       P(FrGrads), _vp, _vp]
        L.fr_albedo_morph.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]
        L.fr_albedo_adjoint.argtypes = [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp]
        L.fr_forward.argtypes = [_vp, P(FrParams), _vp, ctypes.c_uint32, ctypes.c_uint32, _vp]
        L.fr_backward.argtypes = [_vp, P(FrParams), _vp, P(FrGrads), ctypes.c_uint32, ctypes.c_uint32, _vp]
        L.fr_loss.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp]
        L.fr_render.argtypes = [_vp, P(FrParams), _vp, _vp, _vp, P(FrGrads), ctypes.c_uint32,
                                ctypes.c_uint32, _vp]
        L.fr_sync_status.argtypes = [_vp, _vp]
        L.fr_last_error.argtypes = [_vp]
        L.fr_last_error.restype = ctypes.c_char_p
        L.fr_destroy.argtypes = [_vp]
        L.fr_destroy.restype = None
        L.fr_philox.argtypes = [ctypes.c_uint32, ctypes.c_uint32, _vp, ctypes.c_int32, _vp, _vp]
        L.fr_debug_geometry.argtypes = [_vp, P(FrParams), _vp, _vp, _vp]
        L.fr_debug_trace.argtypes = [_vp, P(FrParams), _vp, _vp, ctypes.c_int32, _vp, _vp, _vp]
        L.fr_debug_records.argtypes = [_vp, P(FrParams), _vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint32, _vp]
        L.fr_debug_silhouettes.argtypes = [_vp, P(FrParams), _vp, _vp, _vp, _vp, _vp]
        L.fr_debug_bvh.argtypes = [_vp, P(FrParams), _vp, _vp]
        L.fr_num_edges.argtypes = [_vp]
        L.fr_num_edges.restype = ctypes.c_int32
        L.fr_counters.argtypes = [_vp, _vp, ctypes.c_int32, _vp]
        L.fr_set_timing.argtypes = [_vp, ctypes.c_int32]
        L.fr_get_timing.argtypes = [_vp, _vp]
        L.fr_kernel_launches.argtypes = []
        L.fr_kernel_launches.restype = ctypes.c_uint64
        L.fr_set_flags.argtypes = [_vp, ctypes.c_uint32]
        L.fr_debug_record_tile.argtypes = [_vp, ctypes.c_int64]
        L.fr_debug_morph.argtypes = [_vp, _vp, ctypes.c_int32, _vp, _vp]
        L.fr_render_batch.argtypes = [_vp, _vp, ctypes.c_int32, _vp]
        L.fr_adam.argtypes = [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, _vp, _vp]
        L.fr_loss_noalloc.argtypes = [ctypes.c_int32, ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp]
        L.fr_loss_noalloc_error.argtypes = []
        L.fr_loss_noalloc_error.restype = ctypes.c_char_p
        L.fr_server_create.argtypes = [P(_vp), _vp, P(FrServerConfig)]
        L.fr_submit.argtypes = [_vp, P(FrRequest), P(ctypes.c_uint64)]
        L.fr_poll.argtypes = [_vp, ctypes.c_uint64, P(FrResult), P(FrGrads)]
        L.fr_server_wait.argtypes = [_vp, ctypes.c_double]
        L.fr_server_get_stats.argtypes = [_vp, P(FrServerStats)]
        L.fr_cancel.argtypes = [_vp, ctypes.c_uint64]
        L.fr_server_inject_read_failure.argtypes = [_vp, ctypes.c_int32]
        L.fr_debug_wait_timeout.argtypes = [_vp, ctypes.c_uint32, _vp]
        L.fr_server_destroy.argtypes = [_vp]
        L.fr_server_destroy.restype = None
        _lib = L
    return _lib


def check(code, ctx=None):
    if code != FR_OK:
        msg = lib().fr_last_error(ctx)
        raise FacertError(code, msg.decode() if msg else "")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


# ---- same-named wrappers -------------------------------------------------

def fr_create(width, height, spp, tex_size, edge_spp=1, flags=0, seed=0, max_batch=1):
    h = ctypes.c_void_p()
    cfg = FrConfig(width, height, spp, tex_size, edge_spp, flags, seed, max_batch)
    check(lib().fr_create(ctypes.byref(h), ctypes.byref(cfg)))
    return h


def fr_set_mesh(ctx, mean, basis, faces, uv):
    mean = np.ascontiguousarray(mean, np.float32)
    basis = np.ascontiguousarray(basis, np.float32)
    faces = np.ascontiguousarray(faces, np.int32)
    uv = np.ascontiguousarray(uv, np.float32)
    m = FrMesh(mean.shape[0], faces.shape[0], basis.shape[0], mean.ctypes.data, basis.ctypes.data,
               faces.ctypes.data, uv.ctypes.data)
    check(lib().fr_set_mesh(ctx, ctypes.byref(m)), ctx)


def fr_set_lights(ctx, records, d, a, stage=None, env_size=0):
    records = np.ascontiguousarray(records, np.float32)
    d = np.ascontiguousarray(d, np.float32)
    a = np.ascontiguousarray(a, np.float32)
    st = None if stage is None else np.ascontiguousarray(stage, np.float32)
    ls = FrLightStage(records.shape[0], records.ctypes.data, d.ctypes.data, a.ctypes.data,
                      None if st is None else st.ctypes.data, int(env_size))
    check(lib().fr_set_lights(ctx, ctypes.byref(ls)), ctx)


def fr_set_albedo(ctx, mean_diffuse, basis_diffuse, mean_specular, basis_specular):
    """Statistical albedo model (host arrays): means [M, M, 3], bases [K, M, M, 3]."""
    md = np.ascontiguousarray(mean_diffuse, np.float32)
    bd = np.ascontiguousarray(basis_diffuse, np.float32)
    ms = np.ascontiguousarray(mean_specular, np.float32)
    bs = np.ascontiguousarray(basis_specular, np.float32)
    m = FrAlbedoModel(bd.shape[0], bs.shape[0], md.ctypes.data, bd.ctypes.data, ms.ctypes.data, bs.ctypes.data)
    check(lib().fr_set_albedo(ctx, ctypes.byref(m)), ctx)


def fr_set_landmarks(ctx, vertex_index):
    idx = np.ascontiguousarray(vertex_index, np.int32)
    check(lib().fr_set_landmarks(ctx, idx.shape[0], idx.ctypes.data), ctx)


def fr_landmark_loss(ctx, params, width, height, z, weight, loss, grads=None, projected=None):
    pp = _params(params)
    gg = _grads(grads) if grads is not None else None
    check(lib().fr_landmark_loss(ctx, ctypes.byref(pp), width, height, _ptr(z), weight, _ptr(loss),
                                 ctypes.byref(gg) if gg is not None else None, _ptr(projected), _stream()), ctx)


def _ptr_array(ts):
    if ts is None:
        return None
    return (ctypes.c_void_p * len(ts))(*[t.data_ptr() if t is not None else None for t in ts])


def fr_albedo_morph(ctx, beta, gamma, diffuse, specular):
    """Lists (one entry per face) of device tensors; diffuse/specular may be None."""
    n = len(diffuse if diffuse is not None else specular)
    check(lib().fr_albedo_morph(ctx, n, _ptr_array(beta), _ptr_array(gamma), _ptr_array(diffuse),
                                _ptr_array(specular), _stream()), ctx)


def fr_albedo_adjoint(ctx, g_diffuse, g_specular, g_beta, g_gamma):
    n = len(g_beta if g_beta is not None else g_gamma)
    check(lib().fr_albedo_adjoint(ctx, n, _ptr_array(g_diffuse), _ptr_array(g_specular), _ptr_array(g_beta),
                                  _ptr_array(g_gamma), _stream()), ctx)


def _params(p):
    return FrParams(*[_ptr(p.get(n)) for n in ALL_PARAM_NAMES])


def _grads(g):
    return FrGrads(*[_ptr(g.get(n)) for n in ALL_PARAM_NAMES])


def fr_forward(ctx, params, image, iteration=0, face_id=0):
    pp = _params(params)
    check(lib().fr_forward(ctx, ctypes.byref(pp), _ptr(image), iteration, face_id, _stream()), ctx)


def fr_backward(ctx, params, adj_image, grads, iteration=0, face_id=0):
    pp, gg = _params(params), _grads(grads)
    check(lib().fr_backward(ctx, ctypes.byref(pp), _ptr(adj_image), ctypes.byref(gg), iteration, face_id,
                            _stream()), ctx)


def fr_loss(ctx, image, target, loss, adj_image=None, blurred=None):
    check(lib().fr_loss(ctx, _ptr(image), _ptr(target), _ptr(loss), _ptr(adj_image), _ptr(blurred),
                        _stream()), ctx)


def fr_render(ctx, params, target, image, loss, grads=None, iteration=0, face_id=0):
    pp = _params(params)
    gg = _grads(grads) if grads is not None else None
    check(lib().fr_render(ctx, ctypes.byref(pp), _ptr(target), _ptr(image), _ptr(loss),
                          ctypes.byref(gg) if gg is not None else None, iteration, face_id, _stream()), ctx)


def fr_render_batch(ctx, items):
    """items: list of dicts with width, height, spp, edge_spp, flags, iteration,
    face_id, params (dict of tensors), target, image, loss, grads (dict or None)."""
    arr = (FrItem * len(items))()
    keep = []
    for k, it in enumerate(items):
        g = None
        if it.get("grads") is not None:
            g = _grads(it["grads"])
            keep.append(g)
        arr[k] = FrItem(it["width"], it["height"], it["spp"], it.get("edge_spp", 1), it.get("flags", 0),
                        it.get("iteration", 0), it.get("face_id", 0), _params(it["params"]),
                        _ptr(it["target"]), _ptr(it["image"]), _ptr(it["loss"]),
                        ctypes.pointer(g) if g is not None else None)
    check(lib().fr_render_batch(ctx, ctypes.cast(arr, _vp), len(items), _stream()), ctx)


def fr_sync_status(ctx):
    return lib().fr_sync_status(ctx, _stream())


def fr_destroy(ctx):
    lib().fr_destroy(ctx)


def fr_philox(k0, k1, counters, out):
    check(lib().fr_philox(k0, k1, _ptr(counters), counters.shape[0], _ptr(out), _stream()))


def fr_debug_geometry(ctx, params, v_cam, n_vert):
    pp = _params(params)
    check(lib().fr_debug_geometry(ctx, ctypes.byref(pp), _ptr(v_cam), _ptr(n_vert), _stream()), ctx)


def fr_debug_trace(ctx, params, org, dirs, tri, t):
    pp = _params(params)
    check(lib().fr_debug_trace(ctx, ctypes.byref(pp), _ptr(org), _ptr(dirs), org.shape[0], _ptr(tri), _ptr(t),
                               _stream()), ctx)


def fr_debug_records(ctx, params, image, tri_rec, mask_rec, iteration=0, face_id=0):
    pp = _params(params)
    check(lib().fr_debug_records(ctx, ctypes.byref(pp), _ptr(image), _ptr(tri_rec), _ptr(mask_rec), iteration,
                                 face_id, _stream()), ctx)


def fr_debug_silhouettes(ctx, params, prim, n_prim, per_light, counts):
    pp = _params(params)
    check(lib().fr_debug_silhouettes(ctx, ctypes.byref(pp), _ptr(prim), _ptr(n_prim), _ptr(per_light),
                                     _ptr(counts), _stream()), ctx)


def fr_debug_morph(ctx, params_list, out):
    arr = (FrParams * len(params_list))(*[_params(p) for p in params_list])
    check(lib().fr_debug_morph(ctx, ctypes.cast(arr, _vp), len(params_list), _ptr(out), _stream()), ctx)


def fr_debug_bvh(ctx, params, out):
    pp = _params(params)
    check(lib().fr_debug_bvh(ctx, ctypes.byref(pp), _ptr(out), _stream()), ctx)


def fr_num_edges(ctx):
    return int(lib().fr_num_edges(ctx))


COUNTER_KERNELS = ("forward", "adjoint", "edge_primary")


def fr_counters(ctx, reset=False):
    """Per-kernel traversal work: {kernel: {rays, nodes, tris}}."""
    out = np.zeros(9, np.uint64)
    check(lib().fr_counters(ctx, out.ctypes.data, 1 if reset else 0, _stream()), ctx)
    return {k: {"rays": int(out[3 * i]), "nodes": int(out[3 * i + 1]), "tris": int(out[3 * i + 2])}
            for i, k in enumerate(COUNTER_KERNELS)}


def fr_set_timing(ctx, on=True):
    check(lib().fr_set_timing(ctx, 1 if on else 0), ctx)


TIMING_STAGES = ("build", "forward", "loss", "classify", "adjoint", "edge_primary", "chain", "total")


def fr_get_timing(ctx):
    out = np.zeros(8, np.float32)
    check(lib().fr_get_timing(ctx, out.ctypes.data), ctx)
    return dict(zip(TIMING_STAGES, [float(x) for x in out]))


def fr_set_flags(ctx, flags):
    check(lib().fr_set_flags(ctx, flags), ctx)


def opt_group(x, m, v, g=None, aux=None, kind=GROUP_PLAIN, lr=1e-3, width=0, n_prior=0, w_prior=0.0,
              w_box=0.0, w_sym=0.0, w_chroma=0.0, w_smooth=0.0, clamp=None, step=0, aux2=None):
    """One fr_opt_group over torch device tensors (views of x/g/m/v share storage)."""
    lo, hi = clamp if clamp is not None else (0.0, 0.0)
    grp = FrOptGroup(_ptr(x), _ptr(g), _ptr(m), _ptr(v), _ptr(aux), _ptr(aux2), x.numel(), kind, width, n_prior,
                     lr, w_prior, w_box, w_sym, w_chroma, w_smooth, lo, hi, step)
    grp._keep = (x, g, m, v, aux, aux2)
    return grp


def fr_adam(groups, step=1, beta1=0.9, beta2=0.999, eps=1e-8, reg_energy=None):
    arr = (FrOptGroup * len(groups))(*groups)
    code = lib().fr_adam(ctypes.cast(arr, _vp), len(groups), step, beta1, beta2, eps, _ptr(reg_energy), _stream())
    if code != FR_OK:
        raise FacertError(code, "fr_adam: invalid parameter groups")


def fr_loss_noalloc(height, width, image, target, loss, adj_image=None, blurred=None):
    """fr_loss without a context and without any device allocation (static
    scratch, images up to 512 x 512); raises FacertError on a rejected call."""
    code = lib().fr_loss_noalloc(height, width, _ptr(image), _ptr(target), _ptr(loss), _ptr(adj_image),
                                 _ptr(blurred), _stream())
    if code != FR_OK:
        msg = lib().fr_loss_noalloc_error()
        raise FacertError(code, msg.decode() if msg else "")


def fr_debug_record_tile(ctx, samples):
    """Test hook: recompute the adjoint's hit records in tiles of `samples`
    camera samples (0: the record buffer's full size)."""
    check(lib().fr_debug_record_tile(ctx, int(samples)), ctx)


def fr_kernel_launches():
    return int(lib().fr_kernel_launches())


# ---- convenience: one context bound to a synthetic scene ------------------

class Grads(dict):
    """Gradient tensors by parameter name, views of one flat FP32 device buffer
    (`flat`) so that one fill clears them all.  An entry rebound to a tensor of
    other storage is cleared on its own."""

    def __init__(self, flat, views):
        super().__init__(views)
        self.flat = flat

    def zero_(self):
        self.flat.zero_()
        base = self.flat.untyped_storage().data_ptr()
        for v in self.values():
            if v.untyped_storage().data_ptr() != base:
                v.zero_()
        return self


class Renderer:
    """A library context for one scene (mesh, light stage, image config),
    with torch device buffers for parameters, images and gradients."""

    def __init__(self, scene, edge_spp=1, flags=0, seed=0, max_batch=1):
        import torch
        self.torch = torch
        self.scene = scene
        self.ctx = fr_create(scene.width, scene.height, scene.spp, scene.tex_size, edge_spp, flags, seed, max_batch)
        fr_set_mesh(self.ctx, scene.mean, scene.basis, scene.faces, scene.uv)
        fr_set_lights(self.ctx, scene.lights, scene.light_d, scene.light_a, getattr(scene, "stage", None),
                      getattr(scene, "env_size", 0))
        self.landmarks = getattr(scene, "landmarks", None)
        if self.landmarks is not None:
            fr_set_landmarks(self.ctx, self.landmarks)
        self.albedo = getattr(scene, "albedo", None)
        if self.albedo is not None:
            a = self.albedo
            fr_set_albedo(self.ctx, a.mean_diffuse, a.basis_diffuse, a.mean_specular, a.basis_specular)
        self.n_edges = fr_num_edges(self.ctx)

    def close(self):
        if self.ctx is not None:
            fr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_params(self, params):
        """Device copies of the parameters (the stage geometry only when set)."""
        t = self.torch
        return {n: t.as_tensor(np.ascontiguousarray(getattr(params, n), np.float32)).cuda()
                for n in ALL_PARAM_NAMES if getattr(params, n, None) is not None}

    def zero_grads(self, dparams):
        """Zeroed gradient buffers shaped like `dparams`, as views of one
        device buffer (each view 256-byte aligned): `.zero_()` clears them all
        with one fill."""
        t = self.torch
        sizes = {n: v.numel() for n, v in dparams.items()}
        offs, total = {}, 0
        for n, k in sizes.items():
            offs[n] = total
            total += (k + 63) // 64 * 64
        flat = t.zeros(max(total, 1), dtype=t.float32, device="cuda")
        return Grads(flat, {n: flat[offs[n]:offs[n] + sizes[n]].view(v.shape) for n, v in dparams.items()})

    def image_buffer(self):
        s = self.scene
        return self.torch.zeros((s.height, s.width, 3), dtype=self.torch.float32, device="cuda")

    def forward(self, dparams, iteration=0, face_id=0):
        img = self.image_buffer()
        fr_forward(self.ctx, dparams, img, iteration, face_id)
        return img

    def backward(self, dparams, adj_image, iteration=0, face_id=0, grads=None):
        g = self.zero_grads(dparams) if grads is None else grads
        fr_backward(self.ctx, dparams, adj_image.contiguous(), g, iteration, face_id)
        return g

    def loss(self, image, target):
        t = self.torch
        loss = t.zeros(1, dtype=t.float64, device="cuda")
        adj = t.empty_like(image)
        bl = t.empty_like(image)
        fr_loss(self.ctx, image, target, loss, adj, bl)
        return loss, adj, bl

    def render(self, dparams, target, iteration=0, face_id=0, grads=None, with_grad=True):
        t = self.torch
        img = self.image_buffer()
        loss = t.zeros(1, dtype=t.float64, device="cuda")
        g = (self.zero_grads(dparams) if grads is None else grads) if with_grad else None
        fr_render(self.ctx, dparams, target, img, loss, g, iteration, face_id)
        return img, loss, g

    def records(self, dparams, iteration=0, face_id=0):
        t = self.torch
        s = self.scene
        n = s.width * s.height * s.spp
        img = self.image_buffer()
        tri = t.empty(n, dtype=t.int32, device="cuda")
        mask = t.empty((n, 2), dtype=t.int64, device="cuda")   # lights 0..63, 64..127
        fr_debug_records(self.ctx, dparams, img, tri, mask, iteration, face_id)
        return img, tri, mask

    def status(self):
        return fr_sync_status(self.ctx)


# ---- native server ------------------------------------------------------

def fr_server_create(ctx, max_slots=8, mem_cap_bytes=8 << 30, n_identity=0, edge_spp=1, item_flags=0,
                     eval_iteration=10 ** 6, eval_spp=0, keep_params=True):
    h = ctypes.c_void_p()
    cfg = FrServerConfig(max_slots, mem_cap_bytes, n_identity, edge_spp, item_flags, eval_iteration, eval_spp,
                         1 if keep_params else 0)
    code = lib().fr_server_create(ctypes.byref(h), ctx, ctypes.byref(cfg))
    if code != FR_OK:
        raise FacertError(code, "fr_server_create rejected its context or configuration")
    return h


def _host_params(params):
    """FrParams of host float32 copies (kept alive by the returned list)."""
    keep, ptrs = [], []
    for n in ALL_PARAM_NAMES:
        v = getattr(params, n, None) if not isinstance(params, dict) else params.get(n)
        if v is None:
            ptrs.append(None)
            continue
        a = np.ascontiguousarray(v, np.float32)
        keep.append(a)
        ptrs.append(a.ctypes.data)
    return FrParams(*ptrs), keep


def fr_submit(srv, target, init, spp, stage1, stage2, init_iters=0, landmarks=None):
    """Queue one request (host arrays; copied): returns its id (= its Philox face id)."""
    tgt = np.ascontiguousarray(target, np.float32)
    pp, keep = _host_params(init)
    lm = None if landmarks is None else np.ascontiguousarray(landmarks, np.float32)
    req = FrRequest(tgt.shape[1], tgt.shape[0], spp, init_iters, stage1, stage2, tgt.ctypes.data, pp,
                    None if lm is None else lm.ctypes.data, 0 if lm is None else lm.shape[0])
    rid = ctypes.c_uint64()
    code = lib().fr_submit(srv, ctypes.byref(req), ctypes.byref(rid))
    if code != FR_OK:
        raise FacertError(code, "fr_submit: null target or initial parameter")
    del keep
    return int(rid.value)


def fr_poll(srv, rid, shapes=None):
    """(finished, result dict, final parameters or None).  `shapes` maps
    parameter names to the host shapes to copy back (None: no copy)."""
    res = FrResult()
    out, gg = None, None
    if shapes:
        out = {n: np.zeros(shp, np.float32) for n, shp in shapes.items()}
        gg = FrGrads(*[None if n not in out else out[n].ctypes.data for n in ALL_PARAM_NAMES])
    code = lib().fr_poll(srv, rid, ctypes.byref(res), None if gg is None else ctypes.byref(gg))
    if code not in (FR_OK, FR_EAGAIN):
        raise FacertError(code, "fr_poll: unknown request id")
    r = {"state": res.state, "iterations": res.iterations, "final_loss": res.final_loss,
         "submit_s": res.submit_s, "admit_s": res.admit_s, "finish_s": res.finish_s,
         "error": res.error.decode()}
    done = code == FR_OK
    return done, r, (out if done and res.state == REQ_DONE else None)


def fr_server_wait(srv, timeout_s=3600.0):
    return lib().fr_server_wait(srv, timeout_s) == FR_OK


def fr_server_get_stats(srv):
    st = FrServerStats()
    check(lib().fr_server_get_stats(srv, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in FrServerStats._fields_}


def fr_server_destroy(srv):
    lib().fr_server_destroy(srv)


def fr_server_inject_read_failure(srv, n):
    """Test hook: the n-th device-to-host result read of the server from now
    fails on the host (no device fault)."""
    check(lib().fr_server_inject_read_failure(srv, n))


def fr_cancel(srv, rid):
    """Cancel a request; False if it had already finished or the id is unknown."""
    return lib().fr_cancel(srv, rid) == FR_OK


def fr_debug_wait_timeout(ctx, polls):
    check(lib().fr_debug_wait_timeout(ctx, polls, _stream()), ctx)

