"""Input generators: the refined 100,000-triangle head of the large workload
is a closed, consistently oriented sphere-topology mesh."""
import numpy as np

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
