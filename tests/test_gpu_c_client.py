"""The C ABI from plain C: tests/c_client/render_once.c, compiled with gcc
against include/facert.h, libfacert.so and the CUDA runtime, runs one fused
render of the tiny face and prints the loss and gradients; they equal the
Python binding's for the same inputs bit for bit (the same library calls on
the same data)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2101_05356_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def test_c_client_matches_the_binding(tmp_path):
    from paper_2101_05356_gb300 import build, facert
    lib = build.build()
    cuda = _cuda_home()
    exe = tmp_path / "render_once"
    libdir = os.path.dirname(lib)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), "-I",
                        os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_client", "render_once.c"),
                        "-o", str(exe), "-L", libdir, "-lfacert", "-L", os.path.join(cuda, "lib64"), "-lcudart",
                        "-Wl,-rpath," + libdir], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

    sc = synth.make_scene("tiny")
    pr = synth.random_params(sc, 4)
    tgt = np.random.default_rng(9).uniform(0.0, 0.3, (sc.height, sc.width, 3)).astype(np.float32)
    it, face = 3, 2
    d = tmp_path / "scene"
    d.mkdir()
    (d / "sizes.txt").write_text("%d %d %d %d %d %d %d %d %d %d\n" % (
        sc.width, sc.height, sc.spp, sc.tex_size, sc.n_basis, sc.n_vertices, sc.n_triangles, sc.n_lights,
        it, face))
    arrays = dict(mean=sc.mean, basis=sc.basis, faces=sc.faces, uv=sc.uv, lights=sc.lights, light_d=sc.light_d,
                  light_a=sc.light_a, target=tgt)
    arrays.update({n: getattr(pr, n) for n in facert.PARAM_NAMES})
    for n, a in arrays.items():
        dt = np.int32 if n == "faces" else np.float32
        np.ascontiguousarray(a, dt).tofile(str(d / (n + ".bin")))
    out = subprocess.run([str(exe), str(d)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    vals = {}
    for line in out.stdout.split("\n"):
        f = line.split()
        if not f:
            continue
        if f[0] == "loss":
            vals["loss"] = float(f[1])
        else:
            vals[(f[0], int(f[1]))] = float(f[2])

    r_ = facert.Renderer(sc)
    dp = r_.device_params(pr)
    img, loss, g = r_.render(dp, torch.as_tensor(tgt).cuda(), iteration=it, face_id=face)
    assert r_.status() == 0
    assert vals["loss"] == loss.item()
    coef = g["coef"].cpu().numpy()
    rot = g["rot"].cpu().numpy()
    assert np.abs(coef).max() > 0.0
    for k in range(sc.n_basis):
        assert np.float32(vals[("coef", k)]) == coef[k], k
    for k in range(3):
        assert np.float32(vals[("rot", k)]) == rot[k], k
