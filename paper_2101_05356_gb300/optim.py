"""Two-stage reconstruction (Sec. 4) with device-resident state.

Stage I optimises shape and expression coefficients, pose and light-stage
intensities against E_ph + E_p + E_b (Eq. loss1); Stage II optimises the
personalised diffuse, specular and roughness textures with geometry and lights
fixed against E_ph + symmetry + chromaticity + smoothness + box terms
(Eq. loss3).  Every step is one fused render/loss/adjoint call (fr_render)
followed by one fused Adam + regulariser launch pair (fr_adam).  Learning
rates and weights are the paper's (Sec. 5, "Implementation Details").
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import facert

LR = dict(light=1e-3, identity=1e-2, expression=1e-3, rot=1e-3, trans=1e-3, texture=5e-3)
W = dict(w_i=0.0025, w1=0.01, w2=0.3, w3=0.3, w4=0.0002, box=1.0)


@dataclasses.dataclass
class Schedule:
    stage1: int = 100
    stage2: int = 100


class Reconstruction:
    """One face: parameters, gradients and Adam moments live on the device."""

    def __init__(self, renderer, target, init_params, face_id=0, schedule=Schedule(), flags=0):
        import torch
        self.torch = torch
        self.r = renderer
        self.target = target
        self.face_id = face_id
        self.schedule = schedule
        self.flags = flags
        self.p = renderer.device_params(init_params)
        self.g = renderer.zero_grads(self.p)
        self.m = {n: torch.zeros_like(v) for n, v in self.p.items()}
        self.v = {n: torch.zeros_like(v) for n, v in self.p.items()}
        sc = renderer.scene
        self.ks = sc.n_shape
        self.light_scale = torch.as_tensor(sc.light_d ** 2 / sc.light_a, dtype=torch.float32).cuda()
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.reg = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.image = renderer.image_buffer()
        self.it = 0
        self.ref_diffuse = None
        self.ref_specular = None
        self.history = []

    @property
    def stage(self):
        return 1 if self.it < self.schedule.stage1 else 2

    @property
    def done(self):
        return self.it >= self.schedule.stage1 + self.schedule.stage2

    def _groups_stage1(self):
        p, g, m, v, ks = self.p, self.g, self.m, self.v, self.ks
        out = []
        if ks > 0:
            out.append(facert.opt_group(p["coef"][:ks], m["coef"][:ks], v["coef"][:ks], g["coef"][:ks],
                                        kind=facert.GROUP_COEF, lr=LR["identity"], n_prior=ks, w_prior=W["w_i"]))
        if p["coef"].numel() > ks:
            out.append(facert.opt_group(p["coef"][ks:], m["coef"][ks:], v["coef"][ks:], g["coef"][ks:],
                                        kind=facert.GROUP_COEF, lr=LR["expression"], n_prior=0, w_box=W["box"]))
        out.append(facert.opt_group(p["rot"], m["rot"], v["rot"], g["rot"], lr=LR["rot"]))
        out.append(facert.opt_group(p["trans"], m["trans"], v["trans"], g["trans"], lr=LR["trans"]))
        out.append(facert.opt_group(p["light_i"], m["light_i"], v["light_i"], g["light_i"], aux=self.light_scale,
                                    kind=facert.GROUP_LIGHT, lr=LR["light"], w_prior=W["w1"], w_box=W["box"]))
        return out

    def _groups_stage2(self):
        p, g, m, v = self.p, self.g, self.m, self.v
        M = self.r.scene.tex_size
        return [
            facert.opt_group(p["diffuse"], m["diffuse"], v["diffuse"], g["diffuse"], aux=self.ref_diffuse,
                             kind=facert.GROUP_TEX_RGB, width=M, lr=LR["texture"], w_sym=W["w2"],
                             w_chroma=W["w3"], w_smooth=W["w4"]),
            facert.opt_group(p["specular"], m["specular"], v["specular"], g["specular"], aux=self.ref_specular,
                             kind=facert.GROUP_TEX_RGB, width=M, lr=LR["texture"], w_sym=W["w2"],
                             w_chroma=W["w3"], w_smooth=W["w4"], w_box=W["box"]),
            facert.opt_group(p["roughness"], m["roughness"], v["roughness"], g["roughness"],
                             kind=facert.GROUP_TEX_MONO, width=M, lr=LR["texture"], w_smooth=W["w4"],
                             w_box=W["box"], clamp=(0.02, 1.5)),
        ]

    def step(self):
        """One optimisation iteration (render + loss + adjoint + Adam)."""
        if self.done:
            return
        stage = self.stage
        if stage == 2 and self.ref_diffuse is None:
            # Stage II starts from the Stage I albedos and keeps them as the
            # chromaticity reference (Eq. loss3)
            self.ref_diffuse = self.p["diffuse"].clone()
            self.ref_specular = self.p["specular"].clone()
            facert.fr_set_flags(self.r.ctx, self.flags | facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE)
        elif stage == 1:
            facert.fr_set_flags(self.r.ctx, self.flags)
        for t in self.g.values():
            t.zero_()
        facert.fr_render(self.r.ctx, self.p, self.target, self.image, self.loss, self.g, self.it, self.face_id)
        groups = self._groups_stage1() if stage == 1 else self._groups_stage2()
        step = self.it + 1 if stage == 1 else self.it - self.schedule.stage1 + 1
        facert.fr_adam(groups, step, reg_energy=self.reg)
        self.it += 1

    def run(self, record_every=0):
        while not self.done:
            self.step()
            if record_every and self.it % record_every == 0:
                self.history.append((self.it, float(self.loss.item())))
        return self


def photometric_loss(renderer, params, target, iteration=10 ** 6, face_id=0):
    """E_ph of `params` against `target` with an evaluation Philox iteration."""
    import torch
    img = renderer.forward(params, iteration, face_id)
    loss, _, _ = renderer.loss(img, target)
    return float(loss.item())
