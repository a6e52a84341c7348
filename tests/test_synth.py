"""Input generators: the refined 100,000-triangle head of the large workload
is a closed, consistently oriented sphere-topology mesh; the polyhedral light
stages place each light in its homothetic face."""
import numpy as np
import pytest

from paper_2101_05356_gb300 import synth


def test_large_head_is_closed_and_oriented():
    p, faces = synth.icosphere(2)
    rng = np.random.default_rng(0)
    q, f = synth.bisect_edges(p, faces, 30, rng)
    assert q.shape[0] == p.shape[0] + 30 and f.shape[0] == faces.shape[0] + 60
    for verts, tris in ((q, f),):
        e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
        directed = set(map(tuple, e))
        assert len(directed) == len(e)                       # each directed edge once
        assert all((b, a) in directed for a, b in directed)  # closed, consistent orientation
        a, b, c = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
        n = np.cross(b - a, c - a)
        assert np.all(np.sum(n * (a + b + c), axis=1) > 0.0)  # outward on the sphere
        assert np.allclose(np.linalg.norm(verts, axis=1), 1.0)


def test_large_workload_sizes():
    mean, basis, faces, uv = synth.face_subdivided(np.random.default_rng(1), 100_000, 6, 20)
    V, T = mean.shape[0], faces.shape[0]
    E = T * 3 // 2
    assert (V, T) == (50_002, 100_000) and V - E + T == 2
    assert basis.shape == (20, V, 3) and uv.shape == (V, 2)
    assert np.all((uv >= 0.0) & (uv <= 1.0))


def test_polyhedral_light_stage():
    """Sec. 3.3: each light is its face's homothetic copy (scale d) shrunk by
    sqrt(a) around its barycentric centre, parallel to the face, emitting
    towards the stage centre."""
    centre = np.array(synth.STAGE_CENTRE)
    for name, n in (("tetra", 4), ("octa", 8), ("ico", 20), ("sphere80", 80)):
        v, f = synth._polyhedron(name)
        p = np.random.default_rng(1).dirichlet([4, 4, 4], size=n)
        d = np.linspace(2.5, 3.5, n)
        a = np.linspace(0.1, 0.9, n)
        rec, dd, aa = synth.polyhedral_stage(name, d, a, p)
        assert rec.shape == (n, 11) and np.all(rec[:, 0] == synth.LIGHT_TRI)
        assert np.allclose(dd, d) and np.allclose(aa, a)
        for j in range(n):
            A, B, C = (v[f[j, k]] * d[j] + centre for k in range(3))
            t0 = rec[j, 1:4].astype(np.float64)
            t1, t2 = t0 + rec[j, 4:7], t0 + rec[j, 7:10]
            fn = np.cross(B - A, C - A)
            area_face = 0.5 * np.linalg.norm(fn)
            ln = np.cross(t1 - t0, t2 - t0)
            assert 0.5 * np.linalg.norm(ln) == pytest.approx(a[j] * area_face, rel=1e-5)
            assert np.dot(ln, fn) < 0 and np.linalg.norm(np.cross(ln, fn)) < 1e-5 * np.linalg.norm(ln) * np.linalg.norm(fn)
            # centroid at the barycentric point p of the homothetic face
            assert np.allclose((t0 + t1 + t2) / 3, p[j, 0] * A + p[j, 1] * B + p[j, 2] * C, atol=1e-5)
