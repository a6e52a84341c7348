"""FP64 oracle of the sparse landmark loss (Sec. 4, Eq. landmark).

TEST INFRASTRUCTURE ONLY (imported by tests, never by the product path).
E_land = sum_l || Pi(Gamma(v_l)) - z_l ||^2 with v = mean + sum_k coef_k
basis_k (Sec. 3.1), Gamma(v) = R^T (v - T), R = Rz(t2) Ry(t1) Rx(t0), and the
pinhole Pi of the renderer's camera: screen x = W/2 - f v'_x / v'_z,
y = H/2 + f v'_y / v'_z (camera at the origin looking down -z, image y down).
The gradient is derived by hand here; tests/test_landmark_oracle.py pins the
energy by closed forms and by casting the oracle renderer's camera ray through
each projection, and the gradient by central finite differences.
"""
import numpy as np


def rotation(rot):
    """R = Rz Ry Rx and dR/dt0, dR/dt1, dR/dt2 (float64)."""
    a, b, c = (float(x) for x in rot)
    sx, cx, sy, cy, sz, cz = np.sin(a), np.cos(a), np.sin(b), np.cos(b), np.sin(c), np.cos(c)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    dRx = np.array([[0, 0, 0], [0, -sx, -cx], [0, cx, -sx]])
    dRy = np.array([[-sy, 0, cy], [0, 0, 0], [-cy, 0, -sy]])
    dRz = np.array([[-sz, -cz, 0], [cz, -sz, 0], [0, 0, 0]])
    return Rz @ Ry @ Rx, (Rz @ Ry @ dRx, Rz @ dRy @ Rx, dRz @ Ry @ Rx)


def _posed(scene, params, idx):
    mean = np.asarray(scene.mean, np.float64)[idx]
    basis = np.asarray(scene.basis, np.float64)[:, idx]
    coef = np.asarray(params.coef, np.float64)
    v = mean + np.tensordot(coef, basis, axes=(0, 0)) if coef.size else mean
    w = v - np.asarray(params.trans, np.float64)
    R, dR = rotation(params.rot)
    vp = w @ R                                   # row l: R^T w_l
    return w, vp, R, dR


def project(scene, params, idx, width, height):
    _, vp, _, _ = _posed(scene, params, idx)
    f = float(params.focal[0])
    return np.stack([0.5 * width - f * vp[:, 0] / vp[:, 2], 0.5 * height + f * vp[:, 1] / vp[:, 2]], axis=1)


def energy(scene, params, idx, z, width, height):
    r = project(scene, params, idx, width, height) - np.asarray(z, np.float64)
    return float(np.sum(r * r))


def grad(scene, params, idx, z, width, height):
    """dE/d(coef, rot, trans, focal) as a dict of float64 arrays."""
    w, vp, R, dR = _posed(scene, params, idx)
    f = float(params.focal[0])
    iz = 1.0 / vp[:, 2]
    x = 0.5 * width - f * vp[:, 0] * iz
    y = 0.5 * height + f * vp[:, 1] * iz
    z = np.asarray(z, np.float64)
    ex, ey = 2.0 * (x - z[:, 0]), 2.0 * (y - z[:, 1])
    # dE/dv' per landmark
    gp = np.stack([-ex * f * iz, ey * f * iz, f * iz * iz * (ex * vp[:, 0] - ey * vp[:, 1])], axis=1)
    gw = gp @ R.T                                # dE/dw = R g'
    basis = np.asarray(scene.basis, np.float64)[:, idx]
    out = {
        "coef": np.tensordot(basis, gw, axes=([1, 2], [0, 1])) if basis.shape[0] else np.zeros(0),
        "trans": -gw.sum(axis=0),
        "rot": np.array([np.sum(gp * (w @ D)) for D in dR]),
        "focal": np.array([np.sum(-ex * vp[:, 0] * iz + ey * vp[:, 1] * iz)]),
    }
    return out
