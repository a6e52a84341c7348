"""Continuous-batching reconstruction server.

Requests (a target image of any size up to the server's maximum, a sample count
and a two-stage schedule, Sec. 4) arrive over time.  At every step boundary the
server admits waiting requests while a slot is free and their device state fits
under the memory cap, then advances every admitted request by one iteration
with ONE batched render/loss/adjoint call (fr_render_batch: each stage of the
hot path is one launch over all admitted faces, whatever their size and spp)
and ONE Adam + regulariser launch pair over all their parameter groups.  A
request's parameters, Adam moments and buffers stay on the device until it
finishes; it then leaves and its slot and memory go to the next request.  Each
request's Philox stream is keyed by its id and its own iteration, so its result
does not depend on what it was batched with.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np

from . import facert, optim
from .optim import FaceState, Schedule


@dataclasses.dataclass
class Request:
    rid: int
    target: np.ndarray              # float32 [H, W, 3] (host)
    spp: int
    schedule: Schedule
    arrival: float = 0.0            # seconds after the server starts
    init: object = None             # synth.Params to start from
    landmarks: np.ndarray = None    # float32 [L][2] landmark pixels (enables E_land and the init stage)
    # filled by the server
    admitted: float = None
    finished: float = None
    final_loss: float = None
    params: dict = None             # host copies of the final parameters
    failed: str = None

    @property
    def width(self):
        return int(self.target.shape[1])

    @property
    def height(self):
        return int(self.target.shape[0])


class Server:
    def __init__(self, scene, max_slots=8, mem_cap_bytes=8 << 30, flags=facert.FLAG_MORPH_BF16,
                 max_width=None, max_height=None, max_spp=None, edge_spp=1, seed=0, eval_iteration=10 ** 6,
                 eval_spp=None, keep_params=True):
        import torch
        self.torch = torch
        sc = dataclasses.replace(scene, width=max_width or scene.width, height=max_height or scene.height,
                                 spp=max_spp or scene.spp)
        self.r = facert.Renderer(sc, edge_spp=edge_spp, flags=flags, seed=seed, max_batch=max_slots)
        self.scene = sc
        self.max_slots = max_slots
        self.mem_cap = mem_cap_bytes
        self.flags = flags
        self.edge_spp = edge_spp
        self.eval_iteration = eval_iteration
        self.eval_spp = eval_spp          # final loss at this spp (None: the request's own)
        self.keep_params = keep_params    # copy each finished request's parameters to the host
        self.queue = []
        self.active = []                # (request, FaceState)
        self.done = []
        self.steps = 0
        self.batch_sizes = []

    # ---- admission -------------------------------------------------------
    def submit(self, req: Request):
        if req.width * req.height > self.scene.width * self.scene.height:
            req.failed = "image larger than the server's maximum"
            self.done.append(req)
            return
        self.queue.append(req)

    def _used(self):
        return sum(self.state_bytes(req) for req, _ in self.active)

    def state_bytes(self, req):
        """Device bytes a request's state will hold (parameters, gradients and two
        Adam moments of every group, image and target, Stage II references)."""
        sc = self.scene
        m2 = sc.tex_size * sc.tex_size
        n_param = sc.n_basis + 3 + 3 + 1 + 3 * sc.n_lights + 7 * m2
        if getattr(sc, "stage", None) is not None:
            n_param += 4 * sc.n_lights          # light-stage geometry d, a, p
        return 4 * (4 * n_param + 2 * 3 * req.width * req.height + 2 * 3 * m2) + 8 * 2

    def _admit(self, now):
        torch = self.torch
        while self.queue and len(self.active) < self.max_slots and self.queue[0].arrival <= now:
            req = self.queue[0]
            if self.active and self._used() + self.state_bytes(req) > self.mem_cap:
                break                   # wait for memory to free up (FIFO order kept)
            self.queue.pop(0)
            tgt = torch.as_tensor(np.ascontiguousarray(req.target, np.float32)).cuda()
            st = FaceState(self.r, tgt, req.init, face_id=req.rid, schedule=req.schedule, flags=0,
                           width=req.width, height=req.height, spp=req.spp, landmarks=req.landmarks)
            req.admitted = now
            self.active.append((req, st))

    # ---- one step for every admitted request ------------------------------
    def _step(self):
        run = [st for _, st in self.active if not st.done]         # requests with iterations left
        for st in run:
            st.begin_step()
        states = [st for st in run if st.stage > 0]                 # stage 0: landmarks only, no render
        if states:
            optim.albedo_morph(self.r, states)
            facert.fr_render_batch(self.r.ctx, [st.item(self.edge_spp) for st in states])
            optim.albedo_adjoint(self.r, states)
        for st in run:
            st.landmark_term(self.r)
        groups = [g for st in run for g in st.groups()]
        for k in range(0, len(groups), facert_max_groups()):
            facert.fr_adam(groups[k:k + facert_max_groups()])
        for st in run:
            st.it += 1
        if run:
            self.steps += 1
            self.batch_sizes.append(len(run))

    def _finish(self, now):
        torch = self.torch
        keep = []
        fin = [(req, st) for req, st in self.active if st.done]
        if fin:
            # final photometric loss with a fixed evaluation stream, one batched forward
            items = []
            for req, st in fin:
                it = st.item(self.edge_spp)
                it["iteration"] = self.eval_iteration
                it["grads"] = None
                if self.eval_spp:
                    it["spp"] = self.eval_spp
                items.append(it)
            facert.fr_render_batch(self.r.ctx, items)
            torch.cuda.synchronize()
            for req, st in fin:
                req.final_loss = float(st.loss.item())
                if self.keep_params:
                    req.params = {k: v.detach().cpu().numpy() for k, v in st.p.items()}
                req.finished = time.perf_counter() - self.t0
                self.done.append(req)
        for req, st in self.active:
            if not st.done:
                keep.append((req, st))
        self.active = keep

    def run(self, requests, sync_every_step=True):
        """Serve `requests` (arrival times relative to now); returns them."""
        for req in sorted(requests, key=lambda r: (r.arrival, r.rid)):
            self.submit(req)
        self.t0 = time.perf_counter()
        while self.queue or self.active:
            now = time.perf_counter() - self.t0
            self._admit(now)
            if not self.active:
                if self.queue:
                    time.sleep(max(0.0, min(0.01, self.queue[0].arrival - now)))
                continue
            self._step()
            if sync_every_step:
                self.torch.cuda.synchronize()
            self._finish(time.perf_counter() - self.t0)
        if self.r.status() != 0:
            raise RuntimeError("device status error while serving")
        self.elapsed = time.perf_counter() - self.t0
        return requests


class NativeServer:
    """The library's own server (fr_server_*: admission, batching, the
    two-stage schedule and its optimiser groups run in a worker thread inside
    libfacert.so) behind the same run() interface as Server.  Requests get ids
    0, 1, ... in submission order, and the id is the request's Philox face id,
    so submitting requests whose rid equals their position reproduces Server's
    results bit for bit."""

    def __init__(self, scene, max_slots=8, mem_cap_bytes=8 << 30, flags=facert.FLAG_MORPH_BF16,
                 max_width=None, max_height=None, max_spp=None, edge_spp=1, seed=0, eval_iteration=10 ** 6,
                 eval_spp=None, keep_params=True):
        sc = dataclasses.replace(scene, width=max_width or scene.width, height=max_height or scene.height,
                                 spp=max_spp or scene.spp)
        self.r = facert.Renderer(sc, edge_spp=edge_spp, flags=flags, seed=seed, max_batch=max_slots)
        self.scene = sc
        self.keep_params = keep_params
        self.srv = facert.fr_server_create(self.r.ctx, max_slots=max_slots, mem_cap_bytes=mem_cap_bytes,
                                           n_identity=sc.n_shape, edge_spp=edge_spp, eval_iteration=eval_iteration,
                                           eval_spp=eval_spp or 0, keep_params=keep_params)
        self.done = []

    def _shapes(self, init):
        sc = self.scene
        m, nl = sc.tex_size, sc.n_lights
        shp = {"coef": (sc.n_basis,), "rot": (3,), "trans": (3,), "focal": (1,), "light_i": (nl, 3),
               "diffuse": (m, m, 3), "specular": (m, m, 3), "roughness": (m, m)}
        if getattr(init, "light_d", None) is not None:
            shp.update(light_d=(nl,), light_a=(nl,), light_p=(nl, 2))
        return shp

    def run(self, requests, timeout_s=24 * 3600.0):
        """Submit `requests` at their arrival times (seconds from now), wait
        for all of them and fill in their results; returns them."""
        order = sorted(requests, key=lambda r: (r.arrival, r.rid))
        t0 = time.perf_counter()
        ids = []
        for req in order:
            wait = req.arrival - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            s = req.schedule
            ids.append(facert.fr_submit(self.srv, req.target, req.init, req.spp, s.stage1, s.stage2,
                                        init_iters=s.init, landmarks=req.landmarks))
        if not facert.fr_server_wait(self.srv, timeout_s):
            raise RuntimeError("native server did not finish in time")
        self.elapsed = time.perf_counter() - t0
        for req, rid in zip(order, ids):
            _, res, params = facert.fr_poll(self.srv, rid, self._shapes(req.init) if self.keep_params else None)
            req.native_id = rid
            if res["state"] == facert.REQ_FAILED:
                req.failed = res["error"]
            else:
                req.final_loss = res["final_loss"]
                req.params = params
                # server clock: latency = finish - submit, reported against the arrival
                req.admitted = req.arrival + (res["admit_s"] - res["submit_s"])
                req.finished = req.arrival + (res["finish_s"] - res["submit_s"])
            self.done.append(req)
        self.stats = facert.fr_server_get_stats(self.srv)
        return requests

    def close(self):
        """Stop the server before its context goes away."""
        if getattr(self, "srv", None) is not None:
            facert.fr_server_destroy(self.srv)
            self.srv = None
        if getattr(self, "r", None) is not None:
            self.r.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def facert_max_groups():
    return 128


def serve_plain(scene, requests, flags=0, edge_spp=1, seed=0, eval_iteration=10 ** 6):
    """Baseline: one face at a time (FIFO), single-face calls, FP32 morph."""
    srv = Server(scene, max_slots=1, flags=flags, edge_spp=edge_spp, seed=seed, eval_iteration=eval_iteration,
                 max_width=max(r.width for r in requests), max_height=max(r.height for r in requests),
                 max_spp=max(r.spp for r in requests))
    srv.run(requests)
    return srv


def latency_stats(requests):
    lat = np.array([r.finished - r.arrival for r in requests if r.finished is not None])
    return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "n": int(lat.size)}
