"""Pins of the oracle's boundary term for the specular lobe's cutoff inside
triangles (App. A, Eq. brdf_spec: the lobe needs n_s . o > 0 and does not
vanish there, so the image jumps on the curve n_s . o = 0; edge sampling,
Sec. 4, applied to that curve along image scanlines).

* The crossings of a scanline with the curve against brute force: the
  scanline placed from the Philox stream (pinned by its known-answer test),
  camera rays along it intersected with every triangle by a plain
  Moller-Trumbore test, n_s . o sampled densely on each front-facing hit and
  its sign changes bisected.  A wrong chord, a wrong quadratic or a wrong
  scanline offset moves or drops crossings.
* The full gradient (interior + primary + shadow + this term) against central
  finite differences of the rendered image with common random numbers, on a
  coarse prism whose silhouette-adjacent faces carry the curve under a strong
  specular lobe: without the term the camera and shape gradients miss by many
  standard errors; with it they agree.  The same under the reading that cuts
  every contribution (diffuse included) where n_s . o <= 0."""
import dataclasses

import numpy as np
import pytest

import oracle
import scenes
from paper_2101_05356_gb300 import synth

STREAM_EDGE_SPECULAR = 3


def _scan_coordinate(sc, scan, iteration, face_id=0, seed=0, k=1):
    """(is a row, its coordinate in pixels) from the line's Philox draw."""
    w = oracle.philox(seed, STREAM_EDGE_SPECULAR, 0xFFFFFFFF, (scan << 16) | 0, iteration, face_id)
    u = float(w[0] >> 8) * 2.0 ** -24
    row = scan < sc.height * k
    idx = scan if row else scan - sc.height * k
    return row, (idx + u) / k


def _brute_crossings(sc, pr, scan, iteration, n_fine=4000):
    """Crossings of the scanline with n_s . o = 0 by dense sampling: {triangle:
    sorted coordinates}.  Per front-facing triangle: the interval of the line
    inside its projection (clipped in the image plane), n_s . o of the camera
    ray's hit sampled on a fine grid over it and its sign changes bisected."""
    v, n = oracle.geometry(sc, pr)
    row, c = _scan_coordinate(sc, scan, iteration)
    f = float(pr.focal[0])
    W, H = sc.width, sc.height

    def dirs(ts):
        ts = np.atleast_1d(np.asarray(ts, float))
        if row:
            return np.stack([(ts - 0.5 * W) / f, np.full_like(ts, -(c - 0.5 * H) / f), -np.ones_like(ts)], 1)
        return np.stack([np.full_like(ts, (c - 0.5 * W) / f), -(ts - 0.5 * H) / f, -np.ones_like(ts)], 1)

    out = {}
    for t, (a, b, cc) in enumerate(sc.faces):
        v0, v1, v2 = v[a], v[b], v[cc]
        if not (v0[2] < 0 and v1[2] < 0 and v2[2] < 0):
            continue
        if not np.dot(np.cross(v1 - v0, v2 - v0), -v0) > 0:
            continue

        def q_at(x):
            dd = dirs(x)
            e1, e2 = v1 - v0, v2 - v0
            pv = np.cross(dd, e2)
            det = pv @ e1
            sv = -v0
            b1 = (pv @ sv) / det
            b2 = (dd @ np.cross(sv, e1)) / det
            b0 = 1.0 - b1 - b2
            inside = (b0 >= 0) & (b1 >= 0) & (b2 >= 0)
            m = b0[:, None] * n[a] + b1[:, None] * n[b] + b2[:, None] * n[cc]
            p = b0[:, None] * v0 + b1[:, None] * v1 + b2[:, None] * v2
            return np.einsum("ij,ij->i", m, -p), inside

        # the rays that hit the triangle: its projection clipped by the scanline (2D)
        pj = [(0.5 * W + f * q[0] / -q[2], 0.5 * H - f * q[1] / -q[2]) for q in (v0, v1, v2)]
        ax, bx = (1, 0) if row else (0, 1)           # (scanline axis, along-line axis)
        ends = []
        for i in range(3):
            p0, p1 = pj[i], pj[(i + 1) % 3]
            if (p0[ax] > c) != (p1[ax] > c):
                s_ = (c - p0[ax]) / (p1[ax] - p0[ax])
                ends.append(p0[bx] + s_ * (p1[bx] - p0[bx]))
        if len(ends) != 2:
            continue
        lo, hi = min(ends), max(ends)
        xs = np.linspace(lo, hi, n_fine)
        q, _ = q_at(xs)
        found = []
        for i in np.nonzero(np.sign(q[:-1]) != np.sign(q[1:]))[0]:
            a_, b_ = xs[i], xs[i + 1]
            for _ in range(60):
                mid = 0.5 * (a_ + b_)
                if np.sign(q_at(mid)[0][0]) == np.sign(q[i]):
                    a_ = mid
                else:
                    b_ = mid
            found.append(0.5 * (a_ + b_))
        if found:
            out[t] = sorted(found)
    return row, c, out


@pytest.mark.parametrize("case", ["tube", "tiny"])
def test_crossings_match_brute_force(case):
    if case == "tube":
        sc, pr = scenes.tube()
        scans = [0, 5, 16, 31, 32, 40, 50, 63]
    else:
        sc = synth.make_scene("tiny")
        pr = synth.random_params(sc, 5, coef_scale=0.5)
        scans = list(range(sc.width + sc.height))
    total = 0
    for scan in scans:
        row, c, brute = _brute_crossings(sc, pr, scan, iteration=3)
        tr, xy = oracle.spec_crossings(sc, pr, scan, iteration=3)
        got = {}
        for (t, r), (x, y) in zip(tr, xy):
            assert (y if row else x) == pytest.approx(c, abs=1e-12)        # on the scanline
            got.setdefault(int(t), []).append((int(r), x if row else y))
        assert set(got) == set(brute), (scan, sorted(got), sorted(brute))
        for t, pts in got.items():
            assert [r for r, _ in pts] == list(range(len(pts)))           # roots in order along the line
            assert np.allclose([p for _, p in pts], brute[t], atol=1e-6), (scan, t, pts, brute[t])
            total += len(pts)
    assert total >= 8                                                      # the cases do cross the curve


N_ITER = 24


def _z(make, fields, h, flags=0, spp=16, edge_spp=4, n_iter=N_ITER):
    """z of (all terms, all but the specular boundary) against central finite differences."""
    sc, pr = make()
    sc = dataclasses.replace(sc, spp=spp)
    yy, xx = np.mgrid[0:sc.height, 0:sc.width]
    w = 1.0 + 0.5 * np.sin(xx / 3.0)[..., None] * np.cos(yy / 4.0)[..., None] * np.array([1.0, 0.7, -0.4])
    fd, full, part = ({f: [] for f in fields} for _ in range(3))
    for it in range(n_iter):
        g_all = oracle.grad(sc, pr, w, iteration=1000 + it, edge_spp=edge_spp, flags=flags)
        g_part = oracle.grad(sc, pr, w, iteration=1000 + it, edge_spp=edge_spp, flags=flags,
                             terms=oracle.TERM_ALL & ~oracle.TERM_SPECULAR)
        for name, idx in fields:
            full[(name, idx)].append(np.asarray(g_all[name]).flat[idx])
            part[(name, idx)].append(np.asarray(g_part[name]).flat[idx])
            pp, pm = pr.copy(), pr.copy()
            getattr(pp, name).flat[idx] += h[name]
            getattr(pm, name).flat[idx] -= h[name]
            dimg = oracle.render(sc, pp, iteration=it, flags=flags) - oracle.render(sc, pm, iteration=it, flags=flags)
            fd[(name, idx)].append(float(np.sum(w * dimg)) / (2.0 * h[name]))

    def se(a):
        return np.std(a, ddof=1) / np.sqrt(len(a))

    out = {}
    for k in fields:
        f, g, p = np.array(fd[k]), np.array(full[k]), np.array(part[k])
        out[k] = ((g.mean() - f.mean()) / np.hypot(se(g), se(f)), (p.mean() - f.mean()) / np.hypot(se(p), se(f)),
                  f.mean(), g.mean())
    print({"%s[%d]" % k: tuple(round(x, 3) for x in v) for k, v in out.items()})
    return out


TUBE = [("focal", 0), ("trans", 0), ("trans", 2), ("rot", 1), ("coef", 0)]
TUBE_H = {"focal": 0.2, "trans": 2e-3, "rot": 1e-3, "coef": 5e-3}


def test_tube_gradient_matches_finite_differences():
    z = _z(scenes.tube, TUBE, TUBE_H)
    for k, (z_full, _, fd, g) in z.items():
        assert abs(z_full) <= 3.5, (k, z_full)
        assert abs(g - fd) <= 0.03 * abs(fd) + 1e-9 or abs(z_full) <= 2.0, (k, fd, g)
    assert max(abs(z_part) for _, z_part, _, _ in z.values()) > 6.0     # the term matters here


def test_view_cutoff_reading_is_sampled_too():
    """Cutting every contribution where n_s . o <= 0 puts a larger jump on the
    same curve (the diffuse term too): the boundary term carries it."""
    z = _z(scenes.tube, [("focal", 0), ("trans", 0)], TUBE_H, flags=oracle.VIEW_CUTOFF)
    for k, (z_full, _, _, _) in z.items():
        assert abs(z_full) <= 3.5, (k, z_full)
    assert max(abs(z_part) for _, z_part, _, _ in z.values()) > 6.0


def _c1_face():
    sc = dataclasses.replace(synth.make_scene("c1"), width=48, height=48)
    pr = synth.random_params(sc, 5, coef_scale=0.5)
    pr.focal = pr.focal * (48.0 / 64.0)
    return sc, pr


def test_smooth_face_focal_gradient():
    """On a smooth closed face the vertex normals along the silhouette are
    nearly perpendicular to the view, so the curve n_s . o = 0 runs right next
    to the silhouette: the jump must be the cutoff's own (the one-sided limits
    on the crossing's triangle), not a radiance difference across the curve
    that also straddles the silhouette."""
    z = _z(_c1_face, [("focal", 0)], {"focal": 0.2}, spp=8, edge_spp=1, n_iter=12)
    z_full, z_part, fd, g = z[("focal", 0)]
    assert abs(z_full) <= 3.5, z
    assert abs(g - fd) <= 0.04 * abs(fd), z         # a difference straddling the silhouette: +12%
