"""FP64 oracle of the optimiser step (Sec. 4, Eq. loss1 and loss3; Adam).

TEST INFRASTRUCTURE ONLY (imported by tests and the benchmark's CPU leg, never
by the product path).  Energies are the definitions written out; gradients are
derived by hand here, independently of the CUDA kernel, and pinned by finite
differences of the energies in tests/test_optim_oracle.py.

Readings: the shape prior is squared (w_i sum (alpha_k / sigma_k)^2, sigma_k = 1
for normalised coefficients); soft boxes are quadratic outside the interval;
the light prior holds m_j = mean(I_j) fixed; flip(x) maps texel column c to
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
