"""FP64 oracle of the optimiser step (Sec. 4, Eq. loss1 and loss3; Adam).

TEST INFRASTRUCTURE ONLY (imported by tests and the benchmark's CPU leg, never
by the product path).  Energies are the definitions written out; gradients are
derived by hand here, independently of the CUDA kernel, and pinned by finite
differences of the energies in tests/test_optim_oracle.py.

Readings: the shape prior is squared (w_i sum (alpha_k / sigma_k)^2, sigma_k = 1
for normalised coefficients); soft boxes are quadratic outside the interval;
the light prior holds m_j = mean(I_j) fixed; the virtual light stage's
geometry (Sec. 3.3) is kept in range by soft boxes d_j >= 0, a_j in [0, 1]
and, for the light to stay inside its homothetic face, every barycentric
coordinate of its three corners >= 0, i.e. p_jm >= sqrt(a_j) / 3 for
m = 0, 1, 2 with p_j2 = 1 - p_j0 - p_j1 (the light is the face shrunk by
sqrt(a_j) around p_j); flip(x) maps texel column c to
M - 1 - c; kappa(c) = c / (c_r + c_g + c_b + 1e-6); the smoothness sums every
texel's 4-neighbourhood (so each neighbouring pair appears twice).
"""
import numpy as np


def box_energy(x, w):
    lo = np.minimum(x, 0.0)
    hi = np.maximum(x - 1.0, 0.0)
    return w * float(np.sum(lo * lo + hi * hi))


def box_grad(x, w):
    return 2.0 * w * (np.minimum(x, 0.0) + np.maximum(x - 1.0, 0.0))


def coef_energy(x, n_prior, w_prior, w_box):
    return w_prior * float(np.sum(x[:n_prior] ** 2)) + box_energy(x[n_prior:], w_box)


def coef_grad(x, n_prior, w_prior, w_box):
    g = np.zeros_like(x)
    g[:n_prior] = 2.0 * w_prior * x[:n_prior]
    g[n_prior:] = box_grad(x[n_prior:], w_box)
    return g


def light_energy(i, scale, w_prior, w_box, mean_fixed=None):
    I = i * scale[:, None]
    m = I.mean(axis=1, keepdims=True) if mean_fixed is None else mean_fixed
    return w_prior * float(np.sum((I - m) ** 2)) + w_box * float(np.sum(np.minimum(i, 0.0) ** 2))


def light_grad(i, scale, w_prior, w_box):
    I = i * scale[:, None]
    m = I.mean(axis=1, keepdims=True)
    return 2.0 * w_prior * (I - m) * scale[:, None] + 2.0 * w_box * np.minimum(i, 0.0)


def stage_split(x):
    """[d (N_L) | a (N_L) | p (N_L x 2)] -> d, a, p [N_L][3] (third coordinate implied)."""
    n = x.size // 4
    d, a, p = x[:n], x[n:2 * n], x[2 * n:].reshape(n, 2)
    return d, a, np.concatenate([p, 1.0 - p.sum(axis=1, keepdims=True)], axis=1)


def stage_box_energy(x, w_box):
    """Soft boxes of the light-stage geometry (Sec. 4, E_b): d >= 0, a in
    [0, 1], every corner of light j inside its homothetic face."""
    d, a, p = stage_split(x)
    r = np.sqrt(np.maximum(a, 0.0)) / 3.0
    inside = np.minimum(p - r[:, None], 0.0)
    return w_box * float(np.sum(np.minimum(d, 0.0) ** 2) + box_energy(a, 1.0) + np.sum(inside ** 2))


def stage_light_energy(x, i, w_prior, mean_fixed=None):
    """The light prior w1 sum_j |I_j - m_j|^2 as a function of the geometry:
    I_j = (d_j^2 / a_j) i_j (Eq. light intensity)."""
    d, a, _ = stage_split(x)
    return light_energy(i, d * d / a, w_prior, 0.0, mean_fixed)


def stage_grad(x, i, w_prior, w_box):
    """Gradient of stage_light_energy + stage_box_energy with respect to
    [d | a | p0 p1], derived by hand."""
    n = x.size // 4
    d, a, p = stage_split(x)
    s = d * d / a
    I = i * s[:, None]
    dE_ds = 2.0 * w_prior * np.sum((I - I.mean(axis=1, keepdims=True)) * i, axis=1)
    gd = dE_ds * 2.0 * d / a + 2.0 * w_box * np.minimum(d, 0.0)
    ga = dE_ds * (-s / a) + box_grad(a, w_box)
    ra = np.sqrt(np.maximum(a, 0.0))
    inside = np.minimum(p - ra[:, None] / 3.0, 0.0)              # [N_L][3]
    dr_da = np.where(a > 0.0, 1.0 / (6.0 * np.where(a > 0.0, ra, 1.0)), 0.0)
    ga += 2.0 * w_box * np.sum(inside, axis=1) * (-dr_da)
    gp = 2.0 * w_box * (inside[:, :2] - inside[:, 2:3])           # p2 = 1 - p0 - p1
    return np.concatenate([gd, ga, gp.ravel()])


def smooth_energy(X):
    X = X.reshape(X.shape[0], X.shape[1], -1)
    dh = X[:, 1:] - X[:, :-1]
    dv = X[1:, :] - X[:-1, :]
    return 2.0 * float(np.sum(dh * dh) + np.sum(dv * dv))


def smooth_grad(X):
    shp = X.shape
    X = X.reshape(shp[0], shp[1], -1)
    G = np.zeros_like(X)
    dh = X[:, 1:] - X[:, :-1]
    dv = X[1:, :] - X[:-1, :]
    G[:, :-1] -= 4.0 * dh
    G[:, 1:] += 4.0 * dh
    G[:-1, :] -= 4.0 * dv
    G[1:, :] += 4.0 * dv
    return G.reshape(shp)


def sym_energy(X):
    return float(np.sum(np.abs(X - X[:, ::-1])))


def sym_grad(X):
    return 2.0 * np.sign(X - X[:, ::-1])


def kappa(X):
    return X / (X.sum(axis=-1, keepdims=True) + 1e-6)


def chroma_energy(X, X0):
    return float(np.sum(np.abs(kappa(X) - kappa(X0))))


def chroma_grad(X, X0):
    S = X.sum(axis=-1, keepdims=True) + 1e-6
    sg = np.sign(kappa(X) - kappa(X0))
    return (sg - np.sum(sg * kappa(X), axis=-1, keepdims=True)) / S


def tex_energy(X, w_smooth, w_sym, w_chroma, w_box, X0=None):
    e = w_smooth * smooth_energy(X) + w_sym * sym_energy(X) + box_energy(X, w_box)
    if w_chroma and X0 is not None:
        e += w_chroma * chroma_energy(X, X0)
    return e


def tex_grad(X, w_smooth, w_sym, w_chroma, w_box, X0=None):
    g = w_smooth * smooth_grad(X) + w_sym * sym_grad(X) + box_grad(X, w_box)
    if w_chroma and X0 is not None:
        g = g + w_chroma * chroma_grad(X, X0)
    return g


def adam(x, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8, clamp=None):
    """Kingma & Ba: bias-corrected moments and update; returns (x, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    x = x - lr * mh / (np.sqrt(vh) + eps)
    if clamp is not None:
        x = np.clip(x, clamp[0], clamp[1])
    return x, m, v
