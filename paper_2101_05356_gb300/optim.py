"""Two-stage reconstruction (Sec. 4) with device-resident state.

Stage I optimises shape and expression coefficients, pose, light-stage
intensities (and, when the parameters carry it, the light-stage geometry
d, a, p of Sec. 3.3; under an environment map of Sec. 7 its texels, each a
light with the same prior and box) and (when the scene has a statistical albedo model, Sec. 3.2) the
albedo coefficients beta and gamma against E_ph + E_p + E_b (Eq. loss1): each
Stage I step morphs the textures from beta, gamma (fr_albedo_morph) before the
render and maps the texture gradients back (fr_albedo_adjoint) after it.
Stage II starts the personalised textures from the last statistical albedos
and optimises the
personalised diffuse, specular and roughness textures with geometry and lights
fixed against E_ph + symmetry + chromaticity + smoothness + box terms
(Eq. loss3).  Every step is one fused render/loss/adjoint call (fr_render, or
one item of fr_render_batch when served) followed by one fused Adam +
regulariser launch pair (fr_adam).  Learning rates and weights are the paper's
(Sec. 5, "Implementation Details").
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import facert

ALPHA1 = 1.0             # weight of E_land in E_d (Sec. 5)
LR = dict(light=1e-3, identity=1e-2, expression=1e-3, rot=1e-3, trans=1e-3, texture=5e-3, albedo=2e-2)
W = dict(w_i=0.0025, w_c=0.0025, w_s=0.0025, w1=0.01, w2=0.3, w3=0.3, w4=0.0002, box=1.0)
STAGE2_FLAGS = facert.FLAG_NO_PRIMARY_EDGE | facert.FLAG_NO_SHADOW_EDGE | facert.FLAG_NO_SPECULAR_EDGE
# hard floor on d, a and p after each update (keeps d^2/a finite; the soft boxes do the rest)
STAGE_CLAMP = (1e-3, 1e3)


@dataclasses.dataclass
class Schedule:
    stage1: int = 100
    stage2: int = 100
    init: int = 0           # landmark-only pose and expression iterations before Stage I


class FaceState:
    """Parameters, gradients, Adam moments and buffers of one face (device)."""

    def __init__(self, renderer, target, init_params, face_id=0, schedule=Schedule(), flags=0,
                 width=None, height=None, spp=None, landmarks=None):
        import torch
        self.torch = torch
        sc = renderer.scene
        self.width = width or sc.width
        self.height = height or sc.height
        self.spp = spp or sc.spp
        self.target = target
        self.face_id = face_id
        self.schedule = schedule
        self.flags = flags
        self.p = renderer.device_params(init_params)
        self.g = renderer.zero_grads(self.p)
        self.m = {n: torch.zeros_like(v) for n, v in self.p.items()}
        self.v = {n: torch.zeros_like(v) for n, v in self.p.items()}
        self.ks = sc.n_shape
        self.tex = sc.tex_size
        # the lights' fixed d and a: the optimiser kernel forms the scales d^2 / a
        self.light_da = torch.as_tensor(np.concatenate([sc.light_d, sc.light_a]), dtype=torch.float32).cuda()
        # environment-map texels are lights of scale 1 (Sec. 7); light_i is used by the area lights only
        self.area_lights = bool((sc.lights[:, 0] != facert.LIGHT_ENV).any())
        self.env_scale = (torch.ones(self.p["env"].numel() // 3, dtype=torch.float32, device="cuda")
                          if "env" in self.p else None)
        # light-stage geometry (d, a, p) when the parameters carry it: one
        # contiguous [d | a | p] block per state so that one STAGE group covers it
        self.stage_block = None
        if all(n in self.p for n in facert.STAGE_NAMES):
            self.stage_block = {}
            nl = self.p["light_d"].numel()
            for q, dct in (("x", self.p), ("g", self.g), ("m", self.m), ("v", self.v)):
                blk = torch.cat([dct["light_d"].reshape(-1), dct["light_a"].reshape(-1),
                                 dct["light_p"].reshape(-1)]).contiguous()
                dct["light_d"], dct["light_a"] = blk[:nl], blk[nl:2 * nl]
                dct["light_p"] = blk[2 * nl:].view(nl, 2)
                self.stage_block[q] = blk
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.reg = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.image = torch.zeros((self.height, self.width, 3), dtype=torch.float32, device="cuda")
        self.it = 0
        # landmark targets z [L][2] (pixels of this face's image), E_land weight alpha_1
        self.landmarks = None if landmarks is None else torch.as_tensor(landmarks, dtype=torch.float32).cuda()
        self.n_init = schedule.init if landmarks is not None else 0   # no targets: no initialisation stage
        self.land_loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.ref_diffuse = None
        self.ref_specular = None
        # statistical albedo coefficients (Stage I), zero = the mean albedo
        am = getattr(renderer, "albedo", None)
        self.albedo = am is not None
        self.ab = {}
        if self.albedo:
            for name, k in (("beta", am.k_diffuse), ("gamma", am.k_specular)):
                self.ab[name] = {q: torch.zeros(max(k, 1), dtype=torch.float32, device="cuda")
                                 for q in ("x", "g", "m", "v")}
                self.ab[name]["k"] = k

    def nbytes(self):
        """Device memory owned by this face's state."""
        ts = [t for dct in (self.p, self.g, self.m, self.v) for n, t in dct.items() if n not in facert.STAGE_NAMES]
        ts += [self.image, self.target]
        ts += list(self.stage_block.values()) if self.stage_block else []
        ts += [t for a in self.ab.values() for q, t in a.items() if q != "k"]
        b = sum(t.numel() * t.element_size() for t in ts)
        return b + 2 * self.p["diffuse"].numel() * 4          # Stage II albedo references

    @property
    def stage(self):
        """0: landmark-only initialisation, 1: Stage I, 2: Stage II."""
        if self.it < self.n_init:
            return 0
        return 1 if self.it < self.n_init + self.schedule.stage1 else 2

    @property
    def done(self):
        return self.it >= self.n_init + self.schedule.stage1 + self.schedule.stage2

    def landmark_term(self, renderer):
        """alpha_1 E_land and its gradient (added into g) for stages 0 and 1."""
        if self.landmarks is not None and self.stage <= 1:
            facert.fr_landmark_loss(renderer.ctx, self.p, self.width, self.height, self.landmarks, ALPHA1,
                                    self.land_loss, self.g)

    def begin_step(self):
        """Zero gradients (and take the Stage I albedos as Stage II references)."""
        if self.stage == 1 and self.it == self.n_init > 0:
            for n in ("rot", "trans", "coef"):     # Stage I restarts Adam after the landmark initialisation
                self.m[n].zero_()
                self.v[n].zero_()
        if self.stage == 2 and self.ref_diffuse is None:
            self.ref_diffuse = self.p["diffuse"].clone()
            self.ref_specular = self.p["specular"].clone()
        self.g.zero_()                  # the gradient views share one buffer: one fill
        for a in self.ab.values():
            a["g"].zero_()

    @property
    def stat_albedo(self):
        """True while the textures are the statistical albedos (Stage I with a model)."""
        return self.albedo and self.stage == 1

    def item_flags(self):
        return self.flags | (STAGE2_FLAGS if self.stage == 2 else 0)

    def item(self, edge_spp=1):
        """This face's entry of an fr_render_batch call."""
        return dict(width=self.width, height=self.height, spp=self.spp, edge_spp=edge_spp,
                    flags=self.item_flags(), iteration=self.it, face_id=self.face_id, params=self.p,
                    target=self.target, image=self.image, loss=self.loss, grads=self.g)

    def groups(self):
        """Adam + regulariser groups of the current stage, with this face's step."""
        p, g, m, v, ks = self.p, self.g, self.m, self.v, self.ks
        if self.stage == 0:
            step = self.it + 1
            out = [facert.opt_group(p["rot"], m["rot"], v["rot"], g["rot"], lr=LR["rot"], step=step),
                   facert.opt_group(p["trans"], m["trans"], v["trans"], g["trans"], lr=LR["trans"], step=step)]
            if p["coef"].numel() > ks:
                out.append(facert.opt_group(p["coef"][ks:], m["coef"][ks:], v["coef"][ks:], g["coef"][ks:],
                                            kind=facert.GROUP_COEF, lr=LR["expression"], n_prior=0,
                                            w_box=W["box"], step=step))
            return out
        if self.stage == 1:
            step = self.it - self.n_init + 1
            out = []
            if ks > 0:
                out.append(facert.opt_group(p["coef"][:ks], m["coef"][:ks], v["coef"][:ks], g["coef"][:ks],
                                            kind=facert.GROUP_COEF, lr=LR["identity"], n_prior=ks,
                                            w_prior=W["w_i"], step=step))
            if p["coef"].numel() > ks:
                out.append(facert.opt_group(p["coef"][ks:], m["coef"][ks:], v["coef"][ks:], g["coef"][ks:],
                                            kind=facert.GROUP_COEF, lr=LR["expression"], n_prior=0,
                                            w_box=W["box"], step=step))
            out.append(facert.opt_group(p["rot"], m["rot"], v["rot"], g["rot"], lr=LR["rot"], step=step))
            out.append(facert.opt_group(p["trans"], m["trans"], v["trans"], g["trans"], lr=LR["trans"], step=step))
            sb = self.stage_block
            if self.area_lights:
                out.append(facert.opt_group(p["light_i"], m["light_i"], v["light_i"], g["light_i"],
                                            aux=None, aux2=sb["x"] if sb else self.light_da,
                                            kind=facert.GROUP_LIGHT, lr=LR["light"], w_prior=W["w1"],
                                            w_box=W["box"], step=step))
            if "env" in p:          # environment map (Sec. 7): each texel a light with the light prior
                out.append(facert.opt_group(p["env"], m["env"], v["env"], g["env"], aux=self.env_scale,
                                            kind=facert.GROUP_LIGHT, lr=LR["light"], w_prior=W["w1"],
                                            w_box=W["box"], step=step))
            if sb:                  # light geometry: prior through d^2/a, soft boxes (Sec. 4, E_b)
                out.append(facert.opt_group(sb["x"], sb["m"], sb["v"], sb["g"], aux=p["light_i"],
                                            kind=facert.GROUP_STAGE, lr=LR["light"], w_prior=W["w1"],
                                            w_box=W["box"], clamp=STAGE_CLAMP, step=step))
            for name, w in (("beta", W["w_c"]), ("gamma", W["w_s"])):
                a = self.ab.get(name)
                if a and a["k"] > 0:
                    out.append(facert.opt_group(a["x"], a["m"], a["v"], a["g"], kind=facert.GROUP_COEF,
                                                lr=LR["albedo"], n_prior=a["k"], w_prior=w, step=step))
            return out
        step = self.it - self.n_init - self.schedule.stage1 + 1
        M = self.tex
        return [
            facert.opt_group(p["diffuse"], m["diffuse"], v["diffuse"], g["diffuse"], aux=self.ref_diffuse,
                             kind=facert.GROUP_TEX_RGB, width=M, lr=LR["texture"], w_sym=W["w2"],
                             w_chroma=W["w3"], w_smooth=W["w4"], step=step),
            facert.opt_group(p["specular"], m["specular"], v["specular"], g["specular"], aux=self.ref_specular,
                             kind=facert.GROUP_TEX_RGB, width=M, lr=LR["texture"], w_sym=W["w2"],
                             w_chroma=W["w3"], w_smooth=W["w4"], w_box=W["box"], step=step),
            facert.opt_group(p["roughness"], m["roughness"], v["roughness"], g["roughness"],
                             kind=facert.GROUP_TEX_MONO, width=M, lr=LR["texture"], w_smooth=W["w4"],
                             w_box=W["box"], clamp=(0.02, 1.5), step=step),
        ]


class Reconstruction(FaceState):
    """One face reconstructed alone through the single-face calls."""

    def __init__(self, renderer, target, init_params, face_id=0, schedule=Schedule(), flags=0, landmarks=None):
        super().__init__(renderer, target, init_params, face_id, schedule, flags, landmarks=landmarks)
        self.r = renderer
        self.history = []

    def step(self):
        """One optimisation iteration (render + loss + adjoint + Adam)."""
        if self.done:
            return
        self.begin_step()
        if self.stage > 0:
            facert.fr_set_flags(self.r.ctx, self.item_flags())
            albedo_morph(self.r, [self])
            facert.fr_render(self.r.ctx, self.p, self.target, self.image, self.loss, self.g, self.it, self.face_id)
            albedo_adjoint(self.r, [self])
        self.landmark_term(self.r)
        facert.fr_adam(self.groups(), reg_energy=self.reg)
        self.it += 1

    def run(self, record_every=0):
        while not self.done:
            self.step()
            if record_every and self.it % record_every == 0:
                self.history.append((self.it, float(self.loss.item())))
        facert.fr_set_flags(self.r.ctx, self.flags)
        return self


def albedo_morph(renderer, states):
    """Textures of the faces in `states` that are in Stage I with a statistical
    albedo model, from their beta and gamma (one batched call)."""
    s1 = [st for st in states if st.stat_albedo]
    if s1:
        facert.fr_albedo_morph(renderer.ctx, [st.ab["beta"]["x"] for st in s1], [st.ab["gamma"]["x"] for st in s1],
                               [st.p["diffuse"] for st in s1], [st.p["specular"] for st in s1])


def albedo_adjoint(renderer, states):
    """dE/dbeta, dE/dgamma of those faces from their texture gradients."""
    s1 = [st for st in states if st.stat_albedo]
    if s1:
        facert.fr_albedo_adjoint(renderer.ctx, [st.g["diffuse"] for st in s1], [st.g["specular"] for st in s1],
                                 [st.ab["beta"]["g"] for st in s1], [st.ab["gamma"]["g"] for st in s1])


def photometric_loss(renderer, params, target, iteration=10 ** 6, face_id=0):
    """E_ph of `params` against `target` with an evaluation Philox iteration."""
    img = renderer.forward(params, iteration, face_id)
    loss, _, _ = renderer.loss(img, target)
    return float(loss.item())
