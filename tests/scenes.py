"""Hand-built scenes for closed-form pins (inputs only; no method arithmetic)."""
import numpy as np

from paper_2101_05356_gb300 import synth


def make(verts, faces, basis, lights, width=16, height=16, spp=4, tex=4,
         light_i=None, diffuse=(0.7, 0.5, 0.3)):
    """Scene whose model space is camera space (rot = 0, T = 0)."""
    verts = np.asarray(verts, np.float32)
    n = verts.shape[0]
    basis = np.asarray(basis, np.float32).reshape(-1, n, 3)
    lights = np.asarray(lights, np.float32).reshape(-1, 11)
    nl = lights.shape[0]
    uv = np.stack([np.linspace(0.1, 0.9, n), np.linspace(0.9, 0.1, n)], 1).astype(np.float32)
    sc = synth.Scene(mean=verts, basis=basis, n_shape=basis.shape[0], n_expr=0,
                     faces=np.asarray(faces, np.int32), uv=uv, lights=lights,
                     light_d=np.ones(nl, np.float32), light_a=np.ones(nl, np.float32),
                     width=width, height=height, spp=spp, tex_size=tex, fov_deg=60.0)
    li = np.ones((nl, 3), np.float32) if light_i is None else np.asarray(light_i, np.float32)
    pr = synth.Params(coef=np.zeros(basis.shape[0], np.float32), rot=np.zeros(3, np.float32),
                      trans=np.zeros(3, np.float32), focal=np.array([16.0], np.float32),
                      light_i=li,
                      diffuse=np.tile(np.asarray(diffuse, np.float32), (tex, tex, 1)),
                      specular=np.zeros((tex, tex, 3), np.float32),
                      roughness=np.full((tex, tex), 0.5, np.float32))
    return sc, pr


def quad_light(c, e1, e2, kind=synth.LIGHT_QUAD):
    r = np.zeros(11, np.float32)
    r[0] = kind
    r[1:4], r[4:7], r[7:10] = c, e1, e2
    return r


FAR_TRIANGLE = [[100.0, 100.0, 100.0], [101.0, 100.0, 100.0], [100.0, 101.0, 100.0]]


def shadow_box(width=32, height=32, spp=4, tex=8, seed=0):
    """Floor at z = -4 facing the camera, an occluding triangle above it and two
    emitters (a quad and a disk) between the occluder and the camera, so that
    soft shadows and their boundaries cover much of the image.  Model space is
    camera space (rot = 0, T = 0); the basis moves occluder and floor vertices."""
    verts = [[-1.6, -1.6, -4.0], [1.6, -1.6, -4.0], [1.6, 1.6, -4.0], [-1.6, 1.6, -4.0],
             [-0.35, -0.25, -3.1], [0.55, 0.05, -3.2], [0.0, 0.6, -3.05]]
    faces = [[0, 1, 2], [0, 2, 3], [4, 5, 6]]
    basis = np.zeros((4, 7, 3))
    basis[0, 4, 0] = 1.0
    basis[1, 5, 1] = 1.0
    basis[2, 6, 2] = 1.0
    basis[3, 2, 0] = 0.5
    basis[3, 2, 1] = 0.5
    lights = [quad_light([0.3, 0.2, -1.6], [0.9, 0.0, 0.0], [0.0, -0.9, 0.0]),
              quad_light([-0.4, -0.3, -1.9], [0.0, 0.35, 0.0], [0.35, 0.0, 0.0], synth.LIGHT_DISK)]
    rng = np.random.default_rng(seed)
    sc, pr = make(verts, faces, basis, lights, width=width, height=height, spp=spp, tex=tex,
                  light_i=[(2.0, 1.6, 1.2), (1.0, 1.4, 1.8)])
    sc.uv = rng.uniform(0.05, 0.95, size=(7, 2)).astype(np.float32)
    pr.focal = np.array([float(width)], np.float32)
    pr.diffuse = rng.uniform(0.2, 0.8, size=(tex, tex, 3)).astype(np.float32)
    pr.specular = np.full((tex, tex, 3), 0.05, np.float32)
    pr.roughness = rng.uniform(0.3, 0.6, size=(tex, tex)).astype(np.float32)
    pr.coef = np.array([0.02, -0.03, 0.01, 0.05], np.float32)
    return sc, pr


def stage_box(width=32, height=32, spp=4, tex=8, seed=0):
    """The shadow box lit by a two-light virtual light stage (Sec. 3.3) instead:
    two triangular lights between the occluder and the camera, each in its
    frame's face scaled by d about a centre below the floor, so that moving
    them (d, a, p) moves the occluder's shadow boundaries across the floor."""
    sc, pr = shadow_box(width, height, spp, tex, seed)
    stage = np.array([[0, 0, -4.5, -0.4, -0.3, 1.0, 0.5, -0.3, 1.0, 0.0, 0.5, 1.0],
                      [0, 0, -4.5, -0.6, 0.2, 1.0, 0.0, 0.0, 1.0, -0.3, 0.6, 1.0]], np.float32)
    d, a = np.array([2.7, 2.5], np.float32), np.array([0.6, 0.5], np.float32)
    p = np.array([[0.3, 0.35], [0.4, 0.3]], np.float32)
    rec, dd, aa = synth.stage_records(stage, d, a, p)
    import dataclasses
    sc = dataclasses.replace(sc, lights=rec, light_d=dd, light_a=aa, stage=stage)
    pr.light_d, pr.light_a, pr.light_p = d.copy(), a.copy(), p.copy()
    return sc, pr



def env_box(width=32, height=32, spp=4, tex=8, seed=0, env_size=8, block=2):
    """The shadow box lit by an environment map of lights at infinity (Sec. 7)
    instead of area emitters: env_size^2 texels in blocks of block x block, a
    dim coloured sky and one bright texel towards the camera side, so that the
    occluder casts a sharp shadow on the floor."""
    import dataclasses
    sc, pr = shadow_box(width, height, spp, tex, seed)
    rec, d, a = synth.env_blocks(env_size, block)
    sc = dataclasses.replace(sc, lights=rec, light_d=d, light_a=a, env_size=env_size)
    rng = np.random.default_rng(seed + 3)
    env = rng.uniform(0.1, 0.4, size=(env_size, env_size, 3))
    env[(3 * env_size) // 8, 0] = (6.0, 5.0, 4.0)   # polar 67.5-90 degrees, azimuth 0-45 degrees: +z side
    pr.env = env.astype(np.float32)
    pr.light_i = np.ones((rec.shape[0], 3), np.float32)
    return sc, pr


def mixed_box(width=32, height=32, spp=4, tex=8, seed=0):
    """The shadow box lit by its two area emitters and, together with them, a
    dim 8 x 8 environment map in four blocks with one bright texel."""
    import dataclasses
    sc, pr = shadow_box(width, height, spp, tex, seed)
    rec, d, a = synth.env_blocks(8, 4)
    lights = np.concatenate([sc.lights, rec])
    sc = dataclasses.replace(sc, lights=lights, light_d=np.concatenate([sc.light_d, d]),
                             light_a=np.concatenate([sc.light_a, a]), env_size=8)
    env = np.random.default_rng(seed + 3).uniform(0.05, 0.2, size=(8, 8, 3))
    env[3, 0] = (3.0, 2.5, 2.0)
    pr.env = env.astype(np.float32)
    pr.light_i = np.concatenate([pr.light_i, np.ones((rec.shape[0], 3), np.float32)])
    return sc, pr


def many_box(width=32, height=32, spp=4, tex=8, seed=0, n_lights=80):
    """The shadow box lit by n_lights small quads (a 10 x 8 grid between the
    occluder and the camera, each facing the floor), so that every light casts
    its own shadow of the occluder on the floor, those past the 64th too."""
    import dataclasses
    sc, pr = shadow_box(width, height, spp, tex, seed)
    rng = np.random.default_rng(seed + 5)
    lights = []
    for k in range(n_lights):
        i, j = k % 10, k // 10
        c = [-1.1 + 0.245 * i + rng.uniform(-0.03, 0.03), -0.9 + 0.26 * j + rng.uniform(-0.03, 0.03),
             -2.2 + rng.uniform(-0.2, 0.2)]
        lights.append(quad_light(c, [0.0, 0.14, 0.0], [0.14, 0.0, 0.0]))   # e1 x e2 towards -z
    lights = np.asarray(lights, np.float32)
    sc = dataclasses.replace(sc, lights=lights, light_d=np.ones(n_lights, np.float32),
                             light_a=np.ones(n_lights, np.float32))
    pr.light_i = rng.uniform(0.3, 1.2, size=(n_lights, 3)).astype(np.float32)
    return sc, pr


def ico_box(width=32, height=32, spp=4, tex=8, seed=0):
    """The shadow box under the paper's icosahedral light stage (20 triangular
    lights around a centre below the floor, d = 2.7, a = 0.25): the lights
    above the occluder cast its shadow on the floor."""
    import dataclasses
    sc, pr = shadow_box(width, height, spp, tex, seed)
    rec, d, a = synth.polyhedral_stage("ico", d=2.7, a=0.25, centre=(0.0, 0.0, -4.5))
    sc = dataclasses.replace(sc, lights=rec, light_d=d, light_a=a)
    pr.light_i = np.random.default_rng(seed + 6).uniform(0.5, 1.5, size=(rec.shape[0], 3)).astype(np.float32)
    return sc, pr


def tube(width=32, height=32, spp=16, tex=4, sides=8):
    """An open prism of `sides` faces around the y axis through (0, 0, -4),
    taller than the view, vertex angles 42.5 + 360 k / sides degrees from +z.
    With eight sides the front-facing faces next to the silhouettes (centred
    at +-65 degrees) have one vertex normal turned towards the camera and one
    turned away, so the curve n_s . o = 0 runs through them; two quad lights
    at the sides light them at grazing angles, with a strong specular lobe.
    The basis moves every vertex radially (the prism's radius)."""
    ang = np.deg2rad(42.5 + 360.0 / sides * np.arange(sides))
    ring = np.stack([np.sin(ang), np.zeros(sides), np.cos(ang)], 1)
    verts = np.concatenate([ring + [0.0, -3.0, -4.0], ring + [0.0, 3.0, -4.0]])
    faces = []
    for k in range(sides):
        a, b = k, (k + 1) % sides
        faces += [[a, b, sides + b], [a, sides + b, sides + a]]
    basis = np.zeros((1, 2 * sides, 3))
    basis[0] = np.concatenate([ring, ring]) * 0.5
    lights = [quad_light([3.0, 0.0, -3.0], [0.6, 0.0, 1.2], [0.0, 1.5, 0.0]),
              quad_light([-3.0, 0.0, -3.0], [0.0, 1.5, 0.0], [-0.6, 0.0, 1.2])]
    sc, pr = make(verts, faces, basis, lights, width=width, height=height, spp=spp, tex=tex,
                  light_i=[(3.0, 2.6, 2.2), (2.2, 2.6, 3.0)], diffuse=(0.1, 0.1, 0.1))
    pr.focal = np.array([float(width)], np.float32)
    pr.specular = np.full((tex, tex, 3), 0.6, np.float32)
    pr.roughness = np.full((tex, tex), 0.4, np.float32)
    pr.coef = np.array([0.04], np.float32)
    return sc, pr
