#!/usr/bin/env python3
"""Throughput of the differentiable ray-traced face render on GB300.

One step = one pass of the hot path over one face: morph, pose + normals, BVH
(refit of the mesh's static SAH topology), camera + shadow rays with
Cook-Torrance shading, blur + L1 loss, and the adjoint (interior term from the
forward's per-sample hit records, shadow-boundary and primary-edge terms, chain
to the parameters).  Headline workload: the paper-scale single face (35,709
vertices / 70,789 triangles, K = 80 + 64 bases, 256 x 256, 16 spp, 40 quad
lights, 512^2 textures), synthetic and seeded.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line.  `value` is rays traced per second over the timed steps
(inputs resident in HBM, L2 flushed between steps; each ray of the step is
traced once, the adjoint reading the forward's hit records); `e2e` is the same
metric with the parameters and target copied in from pinned host memory and
the image, loss and every gradient group copied out inside the timed region.
Keyed legs: `large` (a batch of 8 faces of the 100,000-triangle mesh at
1024^2, 64 spp, 80 lights, 2048^2 textures, adjoint re-tracing, with its own
roofline), `serving_capacity` (requests shaped like the serving workload, all
queued at t = 0: faces/s and latency of the continuous-batching servers against
one face at a time, and their final losses), `retrace` (the headline step with
the adjoint re-tracing), `lbvh_rebuild` (an LBVH rebuilt every call),
`environment_map` (the face under a 32 x 32 environment map), `albedo` (the
statistical albedo morph and its transpose against the HBM roofline) and
`cpu_baseline` (the FP64 oracle on the host cores).
The reference arm times the FP64 CPU oracle on a bounded sample of the same
workload.  Under torchrun each rank renders an independent face (replicas).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s fwd+adjoint"
WORKLOAD = ("paper-scale single face: 35,709 verts / 70,789 tris, K=80+64, 256x256, 16 spp, "
            "40 quad lights, 512^2 textures, 1 primary-edge sample/pixel")
# ALU work per traversal step (algorithmic op counts, FP32 lane operations):
# a node visit tests two child boxes (2 x (6 FMA slab + 10 min/max/compare)),
# a Woop triangle test is ~30 operations (shear 6, edge functions 6, det 2,
# distance 3, compares and the reciprocal ~13).
OPS_PER_NODE = 32
OPS_PER_TRI = 30
# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture of this benchmark's workload, valid while the
# sources that make up the kernel hash to `sources_sha256` (else reported as
# null); the capture command is recorded beside the kernel's profile summary.
TRAFFIC = {"k_forward": {"bytes": 23236864 + 9601280,
                         "sources_sha256": "292936dfbfa4dd07bcb5f6f205eda95c504a32d0849ea664c071a481b62b02fe"}}
KERNEL_SOURCES = {"k_forward": ("render.cu", "trace.cuh", "shade.cuh", "common.cuh")}
# Issue-slot use (smsp__issue_active) of a kernel from its ncu --set full capture,
# valid while its sources hash to `sources_sha256`.
ISSUE = {"k_forward": {"frac": 0.7020,
                       "sources_sha256": "292936dfbfa4dd07bcb5f6f205eda95c504a32d0849ea664c071a481b62b02fe"}}
FP32_LANES_PER_SM = 128


def kernel_sources_sha(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_2101_05356_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def kernel_traffic(kernel):
    t = TRAFFIC.get(kernel)
    if not t or kernel not in KERNEL_SOURCES or kernel_sources_sha(kernel) != t["sources_sha256"]:
        return None
    return t["bytes"]


def kernel_issue(kernel):
    t = ISSUE.get(kernel)
    if not t or kernel not in KERNEL_SOURCES or kernel_sources_sha(kernel) != t["sources_sha256"]:
        return None
    return t["frac"]


def sm_count(dev=0):
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def traversal_roofline(cnt, stage, n_launches, dev=0, kernel=None):
    """ALU roofline of the dominant ray kernel of a step (or of `kernel`):
    algorithmic traversal work (OPS_PER_NODE per node visit, OPS_PER_TRI per
    triangle test, counted by the kernel on the mesh's static binned-SAH
    topology, the reference tree) over its mean CUDA-event time, against SMs x
    128 FP32 lanes x the maximum SM clock.  `stage` holds the per-launch stage
    times (ms) of the launches."""
    pk, src = peaks()
    ms = {k: float(np.mean([st[k] for st in stage])) for k in ("forward", "adjoint", "edge_primary")}
    dom = kernel or max(ms, key=ms.get)
    c = cnt[dom]
    ops_per_launch = (c["nodes"] * OPS_PER_NODE + c["tris"] * OPS_PER_TRI) / n_launches
    sms = sm_count(dev)
    peak_ops = sms * FP32_LANES_PER_SM * pk.get("sm_max_mhz", 2070.0) * 1e6
    achieved = ops_per_launch / (ms[dom] / 1000.0)
    return {"bound": "alu", "kernel": "k_" + dom, "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
            "unit": "Tops/s", "frac": achieved / peak_ops, "traffic": kernel_traffic("k_" + dom),
            "issue_frac": kernel_issue("k_" + dom),
            "peak_source": "derived: %d SMs (device) x %d FP32 lanes x %.0f MHz (%s clocks)"
                           % (sms, FP32_LANES_PER_SM, pk.get("sm_max_mhz", 2070.0), src),
            "work_basis": "node visits and triangle tests on the static binned-SAH topology",
            "ops_per_launch": ops_per_launch, "launch_ms": ms[dom]}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return
        t0 = time.time()                      # the timed region starts once sampling runs
        while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
            time.sleep(0.01)
        self.skip = len(self.lines)           # samples taken before the timed region

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["active", "hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[getattr(self, "skip", 0):]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names[1:], f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def make_workload(face_seed):
    from paper_2101_05356_gb300 import synth
    sc = synth.make_scene("c2")
    target_params = synth.random_params(sc, 100 + face_seed)
    params = synth.init_params(sc)
    return sc, params, target_params


def job_totals(total_ms, units, world, device="cuda"):
    """Whole-job totals of the replicas: the slowest rank's timed milliseconds
    (max over ranks) and the units every rank processed (sum over ranks)."""
    if world <= 1:
        return float(total_ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms), float(units)], dtype=torch.float64, device=device)
    tmax = t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(t[1])


def gpu_arm(args, rank, world):
    import torch
    import torch.distributed as dist

    from paper_2101_05356_gb300 import facert

    dev = rank % max(torch.cuda.device_count(), 1)
    torch.cuda.set_device(dev)
    sc, params, tparams = make_workload(rank)
    r = facert.Renderer(sc, edge_spp=1, seed=rank)
    dp = r.device_params(params)
    dt = r.device_params(tparams)
    # synthetic target: the renderer's own image of the ground-truth parameters + noise
    tgt = r.forward(dt, iteration=10 ** 6)
    tgt = (tgt + torch.as_tensor(np.random.default_rng(7 + rank).normal(0, 0.01, tuple(tgt.shape)),
                                 dtype=torch.float32, device="cuda")).contiguous()
    grads = r.zero_grads(dp)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2
    stream = torch.cuda.current_stream()

    def step_out(it):
        grads.zero_()                                   # one fill: the views share one buffer
        img, loss, _ = r.render(dp, tgt, iteration=it, face_id=rank, grads=grads)
        return img, loss

    def step(it):
        return step_out(it)[1]

    for w in range(args.warmup):
        step(w)
    torch.cuda.synchronize()
    if r.status() != 0:
        raise RuntimeError("device status error during warm-up")

    # ---- device-resident timed region ----
    facert.fr_counters(r.ctx, reset=True)
    facert.fr_set_timing(r.ctx, True)
    launches0 = facert.fr_kernel_launches()
    clocks = ClockSampler(dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, stage = [], []
    for k in range(args.steps):
        flush.zero_()                                   # L2 flush outside the events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(args.warmup + k)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stage.append(facert.fr_get_timing(r.ctx))
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = facert.fr_kernel_launches() - launches0 - 0
    facert.fr_set_timing(r.ctx, False)
    cnt = facert.fr_counters(r.ctx, reset=True)
    status = r.status()
    total_ms = float(np.sum(times))
    rays = sum(v["rays"] for v in cnt.values())
    total_ms_max, rays_all = job_totals(total_ms, rays, world, "cuda")
    value = rays_all / (total_ms_max / 1000.0)

    # ---- dominant kernel roofline ----
    roofline = traversal_roofline(cnt, stage, args.steps, dev)

    # ---- the same step in its alternative forms ----
    def timed_variant(flags, n_steps):
        facert.fr_set_flags(r.ctx, flags)
        for w in range(3):
            step(2 * 10 ** 5 + w)
        facert.fr_counters(r.ctx, reset=True)
        facert.fr_set_timing(r.ctx, True)
        torch.cuda.synchronize()
        rt, rst = [], []
        for k in range(n_steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(3 * 10 ** 5 + k)
            e1.record(stream)
            e1.synchronize()
            rt.append(e0.elapsed_time(e1))
            rst.append(facert.fr_get_timing(r.ctx))
        facert.fr_set_timing(r.ctx, False)
        cnt3 = facert.fr_counters(r.ctx, reset=True)
        facert.fr_set_flags(r.ctx, 0)
        rays3 = sum(v["rays"] for v in cnt3.values())
        return {"ms_per_step": float(np.mean(rt)), "rays_per_step": rays3 / n_steps,
                "rays_per_s": rays3 / (float(np.sum(rt)) / 1000.0), "steps": n_steps,
                "stage_ms": {k: float(np.mean([s_[k] for s_ in rst])) for k in rst[0]}}

    # the adjoint re-tracing every camera and shadow ray (the large-image form)
    retrace = timed_variant(facert.FLAG_RECOMPUTE, args.retrace_steps) if args.retrace_steps > 0 else None
    # an LBVH rebuilt every call instead of refitting the static SAH topology
    lbvh = timed_variant(facert.FLAG_LBVH, args.retrace_steps) if args.retrace_steps > 0 else None

    # the same face under the paper's 32 x 32 environment map (Sec. 7) instead of the light stage
    env = env_variant(sc, params, tparams, args.retrace_steps, flush, stream) if args.retrace_steps > 0 else None

    # ---- end to end through the public API with host buffers ----
    # every step copies the parameters and the target in from pinned host
    # memory and the step's results out: image, loss and every gradient group
    e2e = None
    if args.e2e_steps > 0:
        host = {n: torch.as_tensor(np.ascontiguousarray(getattr(params, n), np.float32)).pin_memory()
                for n in facert.PARAM_NAMES}
        host_tgt = tgt.cpu().pin_memory()
        host_loss = torch.empty(1, dtype=torch.float64).pin_memory()
        host_img = torch.empty(tuple(tgt.shape), dtype=torch.float32).pin_memory()
        host_grads = {n: torch.empty(tuple(g.shape), dtype=g.dtype).pin_memory() for n, g in grads.items()}
        h2d = sum(t.numel() * 4 for t in host.values()) + host_tgt.numel() * 4
        d2h = 8 + host_img.numel() * 4 + sum(t.numel() * t.element_size() for t in host_grads.values())
        facert.fr_counters(r.ctx, reset=True)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = 0.0
        for k in range(args.e2e_steps):
            flush.zero_()
            e0.record(stream)
            for n in facert.PARAM_NAMES:
                dp[n].copy_(host[n], non_blocking=True)
            tgt.copy_(host_tgt, non_blocking=True)
            img, loss = step_out(10 ** 5 + k)
            host_loss.copy_(loss, non_blocking=True)
            host_img.copy_(img, non_blocking=True)
            for n, g in grads.items():
                host_grads[n].copy_(g, non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        cnt2 = facert.fr_counters(r.ctx, reset=True)
        rays2 = sum(v["rays"] for v in cnt2.values())
        e2e = {"value": rays2 / (ms / 1000.0), "unit": "rays/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps}
    out = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "rays_per_step": rays / args.steps,
                   "steps_per_s": 1000.0 * args.steps / total_ms_max,
                   "stage_ms": {k: float(np.mean([s[k] for s in stage])) for k in stage[0]}},
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk, "roofline": roofline,
        "retrace": retrace, "lbvh_rebuild": lbvh, "environment_map": env, "status": int(status),
    }
    return out


def env_variant(sc, params, tparams, n_steps, flush, stream, env_size=32, block=4):
    """Fused steps of the same face and image configuration lit by an
    env_size x env_size environment map of lights at infinity in blocks of
    block x block texels (one direction per block per camera sample) instead
    of the light stage."""
    import dataclasses

    import torch

    from paper_2101_05356_gb300 import facert, synth
    rec, d, a = synth.env_blocks(env_size, block)
    sce = dataclasses.replace(sc, lights=rec, light_d=d, light_a=a, env_size=env_size)
    re_ = facert.Renderer(sce, edge_spp=1)
    p, tp = params.copy(), tparams.copy()
    for q in (p, tp):
        q.light_i = np.ones((rec.shape[0], 3), np.float32)
    p.env = np.full((env_size, env_size, 3), 0.3, np.float32)
    tp.env = synth.env_map(np.random.default_rng(5), env_size)
    dp, dt = re_.device_params(p), re_.device_params(tp)
    tgt = re_.forward(dt, iteration=10 ** 6)
    grads = re_.zero_grads(dp)

    def step(it):
        grads.zero_()                                   # one fill: the views share one buffer
        re_.render(dp, tgt, iteration=it, grads=grads)

    for w in range(3):
        step(w)
    facert.fr_counters(re_.ctx, reset=True)
    facert.fr_set_timing(re_.ctx, True)
    torch.cuda.synchronize()
    rt, rst = [], []
    for k in range(n_steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(100 + k)
        e1.record(stream)
        e1.synchronize()
        rt.append(e0.elapsed_time(e1))
        rst.append(facert.fr_get_timing(re_.ctx))
    facert.fr_set_timing(re_.ctx, False)
    cnt = facert.fr_counters(re_.ctx, reset=True)
    status = re_.status()
    re_.close()
    rays = sum(v["rays"] for v in cnt.values())
    return {"workload": "C2 face, 256^2 x 16 spp, %d x %d environment map in %d blocks of %d x %d texels"
                        % (env_size, env_size, rec.shape[0], block, block),
            "ms_per_step": float(np.mean(rt)), "rays_per_step": rays / n_steps,
            "rays_per_s": rays / (float(np.sum(rt)) / 1000.0), "steps": n_steps, "status": int(status),
            "stage_ms": {k: float(np.mean([s_[k] for s_ in rst])) for k in rst[0]}}


def _serving_summary(serve, srv, reqs):
    lat = serve.latency_stats(reqs)
    if hasattr(srv, "batch_sizes"):
        steps, mean_batch = srv.steps, float(np.mean(srv.batch_sizes))
    else:                                   # the library's native server
        steps = int(srv.stats["steps"])
        mean_batch = srv.stats["item_steps"] / max(steps, 1)
    return dict(faces_per_s=len(reqs) / srv.elapsed, elapsed_s=srv.elapsed, p50_s=lat["p50_s"], p99_s=lat["p99_s"],
                mean_final_loss=float(np.mean([q.final_loss for q in reqs])), mean_batch=mean_batch, steps=steps)


def _close_server(srv):
    if hasattr(srv, "batch_sizes"):
        srv.r.close()
    else:
        srv.close()


def serving_bench(n_requests, iters, rate, seed=0):
    """Served (continuous batching, BF16 tensor-core morph, 8 slots) vs plain (one
    face at a time, FP32 morph) on the same Poisson stream of two-stage
    reconstructions of mixed image size and spp (a reduced form of the serving
    workload: sizes {128,192,256}^2, spp {4,8,16}, iters + iters iterations)."""
    import dataclasses

    import torch

    from paper_2101_05356_gb300 import facert, optim, serve, synth
    sc = synth.make_scene("c2")
    rng = np.random.default_rng(seed)
    sizes = rng.choice([128, 192, 256], size=n_requests)
    spps = rng.choice([4, 8, 16], size=n_requests)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    targets = []
    for k in range(n_requests):
        s2 = dataclasses.replace(sc, width=int(sizes[k]), height=int(sizes[k]), spp=int(spps[k]))
        r = facert.Renderer(s2)
        gt = synth.random_params(s2, 500 + k, coef_scale=0.5)
        targets.append(r.forward(r.device_params(gt), iteration=10 ** 7, face_id=k).cpu().numpy())
        r.close()

    def stream():
        return [serve.Request(rid=k, target=targets[k], spp=int(spps[k]), schedule=optim.Schedule(iters, iters),
                              arrival=float(arrivals[k]), init=synth.init_params(sc)) for k in range(n_requests)]

    out = {}
    for name, mk in (("served", lambda: serve.Server(sc, max_slots=8, max_width=256, max_height=256, max_spp=16)),
                     ("native", lambda: serve.NativeServer(sc, max_slots=8, max_width=256, max_height=256,
                                                           max_spp=16, keep_params=False)),
                     ("plain", lambda: serve.Server(sc, max_slots=1, flags=0, max_width=256, max_height=256,
                                                    max_spp=16))):
        srv = mk()
        reqs = srv.run(stream())
        out[name] = _serving_summary(serve, srv, reqs)
        _close_server(srv)
        torch.cuda.synchronize()
    out["faces_per_s_speedup"] = out["served"]["faces_per_s"] / out["plain"]["faces_per_s"]
    out["native_faces_per_s_speedup"] = out["native"]["faces_per_s"] / out["plain"]["faces_per_s"]
    out["final_loss_ratio"] = out["served"]["mean_final_loss"] / out["plain"]["mean_final_loss"]
    out["workload"] = ("%d Poisson requests (rate %.0f/s), sizes {128,192,256}^2, spp {4,8,16}, %d+%d "
                       "iterations, 35,709-vertex face, 40 lights" % (n_requests, rate, iters, iters))
    return out


def _c4_requests(n_requests, seed=0):
    """Targets of the serving workload: image size uniform in {128, 192, 256,
    384, 512}^2 and spp in {4, 8, 16, 32}, each a render of random
    ground-truth parameters at its own size and spp on the paper-scale face
    (35,709 vertices, 40 lights, 512^2 textures, statistical albedo 80 + 80,
    68 landmarks), with the landmark targets their projections."""
    import torch

    from paper_2101_05356_gb300 import facert, synth
    sc = synth.make_scene("c2", albedo_k=80)
    rng = np.random.default_rng(seed)
    sizes = rng.choice([128, 192, 256, 384, 512], size=n_requests)
    spps = rng.choice([4, 8, 16, 32], size=n_requests)
    gen = facert.Renderer(sc.__class__(**{**sc.__dict__, "width": 512, "height": 512, "spp": 32, "albedo": None}))
    targets, marks = [], []
    zero = torch.zeros((512 * 512 * 3,), device="cuda")
    for k in range(n_requests):
        w, sp = int(sizes[k]), int(spps[k])
        gt = gen.device_params(synth.random_params(sc, 700 + k, coef_scale=0.5))
        img = torch.zeros((w, w, 3), device="cuda")
        loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        facert.fr_render_batch(gen.ctx, [dict(width=w, height=w, spp=sp, edge_spp=1, flags=0, iteration=10 ** 7,
                                              face_id=k, params=gt, target=zero, image=img, loss=loss)])
        proj = torch.zeros((len(sc.landmarks), 2), device="cuda")
        facert.fr_landmark_loss(gen.ctx, gt, w, w, torch.zeros_like(proj), 1.0, loss, None, proj)
        targets.append(img.cpu().numpy())
        marks.append(proj.cpu().numpy())
    gen.close()
    return sc, rng, sizes, spps, targets, marks


def _c4_server(sc, slots, flags, native=False):
    from paper_2101_05356_gb300 import serve
    cls = serve.NativeServer if native else serve.Server
    return cls(sc, max_slots=slots, flags=flags, max_width=512, max_height=512, max_spp=32,
               eval_spp=32, keep_params=False, mem_cap_bytes=64 << 30)


def serving_capacity(n_requests=24, stage1=100, stage2=100, init=20, seed=1, max_slots=8):
    """Closed-loop capacity of the served and plain forms on requests shaped
    like the serving workload (the full size and spp mix, the full landmark +
    Stage I + Stage II schedule), all queued at t = 0: faces/s = requests /
    time to finish all of them; latency = finish time of each request.  Served
    = continuous batching with BF16 tensor-core morphs (the Python server and
    the library's server); plain = one face at a time, FP32 morph.  Final
    losses are evaluated at 32 spp with a fixed evaluation stream."""
    import torch

    from paper_2101_05356_gb300 import facert, optim, serve, synth
    sc, _, sizes, spps, targets, marks = _c4_requests(n_requests, seed)
    sched = optim.Schedule(stage1=stage1, stage2=stage2, init=init)
    out = {"workload": "%d requests queued at t = 0, sizes {128..512}^2 (mean %.0f^2), spp {4,8,16,32} (mean %.1f), "
                       "%d landmark + %d + %d iterations, 35,709-vertex face, 40 lights, statistical albedo 80+80, "
                       "68 landmarks" % (n_requests, float(np.sqrt(np.mean(sizes.astype(float) ** 2))),
                                         float(np.mean(spps)), init, stage1, stage2)}
    for name, slots, flags, native in (("served", max_slots, facert.FLAG_MORPH_BF16, False),
                                       ("native", max_slots, facert.FLAG_MORPH_BF16, True),
                                       ("plain", 1, 0, False)):
        reqs = [serve.Request(rid=k, target=targets[k], spp=int(spps[k]), schedule=sched, arrival=0.0,
                              init=synth.init_params(sc), landmarks=marks[k]) for k in range(n_requests)]
        srv = _c4_server(sc, slots, flags, native)
        done = srv.run(reqs)
        out[name] = _serving_summary(serve, srv, done)
        _close_server(srv)
        torch.cuda.synchronize()
    for name in ("served", "native"):
        out[name + "_capacity_speedup"] = out[name]["faces_per_s"] / out["plain"]["faces_per_s"]
        out[name + "_final_loss_ratio"] = out[name]["mean_final_loss"] / out["plain"]["mean_final_loss"]
    return out


def serving_c4(n_requests=512, stage1=100, stage2=100, init=20, seed=0, max_slots=8,
               forms=("served", "native", "plain")):
    """The serving workload: a Poisson stream of two-stage reconstructions of
    the paper-scale face (35,709 vertices, 40 lights, 512^2 textures, a
    statistical albedo model of 80 + 80 columns, 68 landmarks) with image
    size uniform in {128, 192, 256, 384, 512}^2 and spp in {4, 8, 16, 32};
    each request runs `init` landmark iterations, then Stage I and Stage II.
    The arrival rate is 0.9 x the served closed-loop capacity measured first
    on a short prefix.  Served (continuous batching, BF16 tensor-core morphs,
    max_slots slots) and plain (one face at a time, FP32) see the same stream;
    final losses are evaluated at 32 spp with a fixed evaluation stream."""
    import torch

    from paper_2101_05356_gb300 import facert, optim, serve, synth
    sc, rng, sizes, spps, targets, marks = _c4_requests(n_requests, seed)
    sched = optim.Schedule(stage1=stage1, stage2=stage2, init=init)

    def stream(arrivals):
        return [serve.Request(rid=k, target=targets[k], spp=int(spps[k]), schedule=sched, arrival=float(arrivals[k]),
                              init=synth.init_params(sc), landmarks=marks[k]) for k in range(n_requests)]

    # closed-loop capacity of the served form on a prefix (all arrive at once)
    n_cap = min(n_requests, 2 * max_slots)
    srv = _c4_server(sc, max_slots, facert.FLAG_MORPH_BF16, "native" in forms)
    srv.run(stream(np.zeros(n_requests))[:n_cap])
    capacity = n_cap / srv.elapsed
    _close_server(srv)
    rate = 0.9 * capacity
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_requests))
    out = {"workload": "%d Poisson requests, sizes {128..512}^2, spp {4,8,16,32}, %d landmark + %d + %d "
                       "iterations, 35,709-vertex face, 40 lights, statistical albedo 80+80, 68 landmarks"
                       % (n_requests, init, stage1, stage2),
           "closed_loop_capacity_faces_per_s": capacity, "arrival_rate_per_s": rate}
    for name, slots, flags, native in (("served", max_slots, facert.FLAG_MORPH_BF16, False),
                                       ("native", max_slots, facert.FLAG_MORPH_BF16, True),
                                       ("plain", 1, 0, False)):
        if name not in forms:
            continue
        srv = _c4_server(sc, slots, flags, native)
        reqs = srv.run(stream(arrivals))
        out[name] = _serving_summary(serve, srv, reqs)
        _close_server(srv)
        torch.cuda.synchronize()
    for name in ("served", "native"):
        if name in out and "plain" in out:
            out[name + "_faces_per_s_speedup"] = out[name]["faces_per_s"] / out["plain"]["faces_per_s"]
            out[name + "_final_loss_ratio"] = out[name]["mean_final_loss"] / out["plain"]["mean_final_loss"]
    return out


def large_bench(batch=8, steps=3, warmup=2):
    """The large workload: a batch of `batch` faces of the 100,000-triangle
    mesh (K = 20), 1024 x 1024, 64 spp, 80 lights, 2048^2 textures, BF16
    tensor-core morph, one fused forward + loss + adjoint call per step
    (fr_render_batch); the hit records exceed their budget, so the adjoint
    recomputes them tile by tile (a visibility-only pass of the forward kernel
    per tile, then the recorded adjoint).  Device-resident inputs (far larger
    than L2), CUDA events around each step, stage times from the library's
    events, and the roofline of the forward kernel (one launch per step; the
    adjoint stage is several launches: its tiles' record passes of the same
    kernel and the recorded adjoint)."""
    import torch

    from paper_2101_05356_gb300 import facert, synth
    sc = synth.make_scene("c5")
    r = facert.Renderer(sc, edge_spp=1, flags=facert.FLAG_MORPH_BF16, max_batch=batch)
    items = []
    rng = np.random.default_rng(3)
    for k in range(batch):
        dp = r.device_params(synth.random_params(sc, 800 + k))
        tgt = r.forward(r.device_params(synth.random_params(sc, 900 + k)), iteration=10 ** 7, face_id=k)
        tgt = (tgt + torch.as_tensor(rng.normal(0.0, 0.01, tuple(tgt.shape)), dtype=torch.float32).cuda()).contiguous()
        items.append(dict(width=sc.width, height=sc.height, spp=sc.spp, edge_spp=1, flags=0, iteration=0, face_id=k,
                          params=dp, target=tgt, image=torch.zeros_like(tgt),
                          loss=torch.zeros(1, dtype=torch.float64, device="cuda"), grads=r.zero_grads(dp)))
    stream = torch.cuda.current_stream()
    ms, stages = [], []
    for k in range(warmup + steps):
        for it in items:
            it["iteration"] = k
            it["grads"].zero_()
        if k == warmup:
            torch.cuda.synchronize()
            facert.fr_counters(r.ctx, reset=True)
            facert.fr_set_timing(r.ctx, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        facert.fr_render_batch(r.ctx, items)
        e1.record(stream)
        e1.synchronize()
        if k >= warmup:
            ms.append(e0.elapsed_time(e1))
            stages.append(facert.fr_get_timing(r.ctx))
    facert.fr_set_timing(r.ctx, False)
    cnt = facert.fr_counters(r.ctx, reset=True)
    rays = sum(v["rays"] for v in cnt.values()) / steps
    status = r.status()
    roof = traversal_roofline(cnt, stages, steps, kernel="forward")
    r.close()
    torch.cuda.empty_cache()
    s_step = float(np.mean(ms)) / 1000.0
    return {"workload": "batch of %d faces: 50,002 verts / 100,000 tris, K = 20, 1024 x 1024, 64 spp, 80 lights, "
                        "2048^2 textures, BF16 morph, hit records recomputed tile by tile" % batch,
            "s_per_step": s_step, "rays_per_step": rays, "rays_per_s": rays / s_step,
            "face_steps_per_s": batch / s_step, "steps": steps, "warmup": warmup, "status": int(status),
            "l2": "inputs far larger than L2 (2048^2 textures per face, records recomputed per tile)",
            "stage_ms": {k: float(np.mean([st[k] for st in stages])) for k in stages[0]},
            "roofline": roof}


def albedo_bench(batch=8, reps=10):
    """Statistical albedo morph (Sec. 3.2) at the paper-scale texture size
    (512^2 texels, K = 80 per albedo, diffuse + specular in one call) as the
    BF16 tensor-core GEMM and in FP32, and its FP64-summed transpose, for a
    batch of faces; HBM roofline on the algorithmic bytes (basis read once,
    means, textures or texture gradients)."""
    import torch

    from paper_2101_05356_gb300 import facert, synth
    sc = synth.make_scene("c2", albedo_k=80)
    M, K = sc.tex_size, 80
    rows = 3 * M * M
    pk, src = peaks()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(0)
    coefs = [torch.as_tensor(rng.normal(size=K).astype(np.float32)).cuda() for _ in range(2 * batch)]
    tex = [torch.empty((M, M, 3), device="cuda") for _ in range(2 * batch)]
    gco = [torch.zeros(K, device="cuda") for _ in range(2 * batch)]
    out = {"workload": "512^2 x 3 texels, K = 80 diffuse + 80 specular, batch %d" % batch,
           "l2": "ms: mean of 20 back-to-back calls (each reads a basis larger than L2); ms_single: one "
                 "call after an L2 flush, its launch latency included"}

    def timed(fn, back_to_back=20):
        """(per-launch ms of `back_to_back` calls issued together: the bases,
        252 MB BF16 / 503 MB FP32, are larger than L2, so no flush between
        them; ms of one call after an L2 flush, launch latency included)"""
        ms = []
        for k in range(reps + 2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            e1.synchronize()
            if k >= 2:
                ms.append(e0.elapsed_time(e1))
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(back_to_back):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / back_to_back, float(np.median(ms))

    for name, flags, basis_bytes in (("morph_bf16_tc", facert.FLAG_MORPH_BF16, 2), ("morph_fp32", 0, 4)):
        r = facert.Renderer(sc, flags=flags, max_batch=batch)
        for n in (1, batch):
            ms, ms1 = timed(lambda: facert.fr_albedo_morph(r.ctx, coefs[:n], coefs[batch:batch + n], tex[:n],
                                                           tex[batch:batch + n]))
            nbytes = 2 * (rows * K * basis_bytes + rows * 4 + n * rows * 4)
            out["%s_b%d" % (name, n)] = {"ms": ms, "GB/s": nbytes / ms / 1e6,
                                         "frac_hbm": nbytes / ms / 1e6 / pk["hbm_gbs"], "ms_single": ms1}
        if flags == 0:
            for n in (1, batch):
                ms, ms1 = timed(lambda: facert.fr_albedo_adjoint(r.ctx, tex[:n], tex[batch:batch + n], gco[:n],
                                                                 gco[batch:batch + n]))
                nbytes = 2 * (rows * K * 4 + n * rows * 4)
                out["adjoint_b%d" % n] = {"ms": ms, "GB/s": nbytes / ms / 1e6,
                                          "frac_hbm": nbytes / ms / 1e6 / pk["hbm_gbs"], "ms_single": ms1}
        r.close()
    out["peak_hbm_gbs"] = pk["hbm_gbs"]
    out["peak_source"] = src
    return out


def cpu_baseline(sample_pixels, threads=0, c1_full=True):
    """The FP64 oracle as it stands, timed on the host cores.

    * Headline sample: forward + adjoint (all terms) of the benchmark's face
      restricted to `sample_pixels` random pixels; rays/s over that sample.
    * One full forward + adjoint iteration of that face and a two-stage
      reconstruction (20 landmark + 100 + 100 iterations, the paper's
      schedule) EXTRAPOLATED from the sample's time per pixel (Stage II has no
      edge terms, so the reconstruction figure overstates it somewhat).
    * With c1_full: the small face (2,562 vertices, 64 x 64, 4 spp, 8 lights)
      forward + adjoint in full, measured."""
    import oracle
    from paper_2101_05356_gb300 import synth
    sc, params, tparams = make_workload(0)
    rng = np.random.default_rng(1)
    npx = sc.width * sc.height
    pix = np.sort(rng.choice(npx, size=sample_pixels, replace=False)).astype(np.int32)
    adj = np.zeros((sc.height, sc.width, 3))
    adj.reshape(-1, 3)[pix] = rng.uniform(0.2, 1.0, (sample_pixels, 3))
    cores = threads or (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    oracle.build()
    oracle.ray_count(reset=True)
    t0 = time.perf_counter()
    oracle.render(sc, params, pixels=pix, n_threads=cores)
    oracle.grad(sc, params, adj, n_threads=cores, edge_spp=1)
    dt = time.perf_counter() - t0
    rays = oracle.ray_count(reset=True)
    it_s = dt / sample_pixels * npx
    out = {"value": rays / dt, "unit": "rays/s", "cores": cores, "kind": "oracle",
           "sample": "%d of %d pixels of the workload (16 spp, 40 lights), forward + adjoint with all "
                     "edge terms; %d rays in %.1f s" % (sample_pixels, npx, rays, dt),
           "seconds": dt,
           "iteration_s_extrapolated": it_s,
           "reconstruction_s_extrapolated": 220 * it_s,
           "extrapolation": "time per sampled pixel x %d pixels; reconstruction = 220 such iterations "
                            "(20 landmark-only iterations cost far less, and Stage II has no edge terms)" % npx}
    if c1_full:
        s1 = synth.make_scene("c1")
        p1 = synth.init_params(s1)
        t1 = oracle.render(s1, synth.random_params(s1, 3), n_threads=cores).astype(np.float32)
        oracle.ray_count(reset=True)
        t0 = time.perf_counter()
        img = oracle.render(s1, p1, n_threads=cores)
        _, _, a1 = oracle.loss(img, t1)
        oracle.grad(s1, p1, a1, n_threads=cores, edge_spp=1)
        d1 = time.perf_counter() - t0
        r1 = oracle.ray_count(reset=True)
        out["c1_full"] = {"workload": "2,562 verts / 5,120 tris, K = 20, 64 x 64, 4 spp, 8 lights, forward + loss + "
                                      "adjoint with all terms, every pixel", "seconds": d1, "rays": r1,
                          "rays_per_s": r1 / d1}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--retrace-steps", type=int, default=5)
    ap.add_argument("--cpu-pixels", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-albedo", action="store_true")
    ap.add_argument("--serve-c4", type=int, default=0, help="run the serving workload with this many requests")
    ap.add_argument("--serve-c4-stage1", type=int, default=100)
    ap.add_argument("--serve-c4-stage2", type=int, default=100)
    ap.add_argument("--serve-c4-init", type=int, default=20)
    ap.add_argument("--serve-c4-forms", default="served,native,plain",
                    help="which forms of the serving workload to run (comma-separated: served = the Python "
                         "server, native = the library's server, plain = one face at a time)")
    ap.add_argument("--large", action="store_true",
                    help="run the large workload (batch of 8 faces, 1024^2, 64 spp, 100,000 triangles) on its own line")
    ap.add_argument("--large-steps", type=int, default=3,
                    help="timed steps of the large-workload leg (0: skip it)")
    ap.add_argument("--large-warmup", type=int, default=2)
    ap.add_argument("--capacity-requests", type=int, default=24,
                    help="requests of the closed-loop served vs plain capacity leg (0: skip it)")
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="requests of the reduced Poisson stream leg (0: skip it)")
    ap.add_argument("--serve-iters", type=int, default=6)
    ap.add_argument("--serve-rate", type=float, default=40.0)
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))

    if args.large:
        res = large_bench(steps=max(args.large_steps, 1), warmup=args.large_warmup)
        print(json.dumps({"metric": "rays/s fwd+adjoint (large workload)", "value": res["rays_per_s"],
                          "unit": "rays/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
                          "large": res}))
        return

    if args.serve_c4 > 0:
        # the full serving workload, reported on its own line (not the step benchmark)
        forms = tuple(f.strip() for f in args.serve_c4_forms.split(",") if f.strip())
        res = serving_c4(args.serve_c4, args.serve_c4_stage1, args.serve_c4_stage2, args.serve_c4_init, forms=forms)
        head = "native" if "native" in res else "served"
        print(json.dumps({"metric": "faces/s (served reconstruction stream)", "value": res[head]["faces_per_s"],
                          "unit": "faces/s", "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
                          "serving": res}))
        return

    if args.impl == "reference":
        if rank != 0:
            return
        per = []
        for k in range(args.warmup + args.steps):
            b = cpu_baseline(max(4, args.cpu_pixels // 8), c1_full=False)
            if k >= args.warmup:
                per.append(b)
        v = float(np.mean([b["value"] for b in per]))
        out = {"metric": METRIC, "value": v, "unit": "rays/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean([b["seconds"] for b in per])),
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "impl": "reference",
               "config": {"workload": WORKLOAD},
               "cpu_baseline": {"value": v, "unit": "rays/s", "cores": per[0]["cores"], "kind": "oracle",
                                "sample": per[0]["sample"]},
               "e2e": {"value": v, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = gpu_arm(args, rank, world)
    if rank == 0 and world == 1 and args.large_steps > 0:
        out["large"] = large_bench(steps=args.large_steps, warmup=args.large_warmup)
    if rank == 0 and world == 1 and args.capacity_requests > 0:
        out["serving_capacity"] = serving_capacity(args.capacity_requests)
    if rank == 0 and world == 1 and args.serve_requests > 0:
        out["serving"] = serving_bench(args.serve_requests, args.serve_iters, args.serve_rate)
    if rank == 0 and world == 1 and not args.no_albedo:
        out["albedo"] = albedo_bench()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = {k: v for k, v in cpu_baseline(args.cpu_pixels).items() if k != "seconds"}
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
