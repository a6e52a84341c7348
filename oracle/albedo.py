"""FP64 oracle of the statistical albedo model (Sec. 3.2).

TEST INFRASTRUCTURE ONLY (imported by tests, never by the product path).  The
model is linear, so the oracle is its definition written out in double
precision: the diffuse albedo texture C = a_r + Sigma_r beta and the specular
S = a_b + Sigma_b gamma, each [M, M, 3], with basis [K, M, M, 3] (column k is
the texture-space field of coefficient k); the gradient of an energy E with
respect to the coefficients is the transpose applied to dE/dC:
dE/dbeta_k = sum over texels and channels of Sigma_r[k] * dE/dC.  Pinned in
tests/test_albedo_oracle.py by the adjoint identity, the column structure and
finite differences of the renderer's energy through the oracle's own texture
gradient.
"""
import numpy as np


def morph(mean, basis, coef):
    """mean [M, M, 3] + sum_k coef[k] basis[k] (float64)."""
    mean = np.asarray(mean, np.float64)
    basis = np.asarray(basis, np.float64)
    coef = np.asarray(coef, np.float64)
    return mean + np.tensordot(coef, basis, axes=(0, 0))


def adjoint(basis, g):
    """sum over texels of basis[k] * g for every k (float64 [K])."""
    basis = np.asarray(basis, np.float64)
    g = np.asarray(g, np.float64)
    return np.tensordot(basis, g, axes=([1, 2, 3], [0, 1, 2]))
