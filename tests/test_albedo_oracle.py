"""Pins of the statistical-albedo oracle (Sec. 3.2): the adjoint is the
transpose of the morph (so a transposed or shifted index fails), each column is
the response to a unit coefficient, and the chain through the renderer matches
central finite differences of the oracle's own render."""
import numpy as np
import pytest

import oracle
from oracle import albedo
from paper_2101_05356_gb300 import synth


@pytest.fixture(scope="module")
def model():
    return synth.albedo_model(np.random.default_rng(3), 8, 5, 4)


def test_adjoint_identity(model):
    rng = np.random.default_rng(0)
    for mean, basis in ((model.mean_diffuse, model.basis_diffuse), (model.mean_specular, model.basis_specular)):
        c = rng.normal(size=basis.shape[0])
        g = rng.normal(size=mean.shape)
        lhs = float(np.sum((albedo.morph(mean, basis, c) - mean) * g))
        rhs = float(np.dot(c, albedo.adjoint(basis, g)))
        assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-15)


def test_columns_are_unit_responses(model):
    mean, basis = model.mean_diffuse, model.basis_diffuse
    for k in range(basis.shape[0]):
        e = np.zeros(basis.shape[0])
        e[k] = 1.0
        assert np.allclose(albedo.morph(mean, basis, e) - mean, basis[k], rtol=0, atol=1e-7)
    # zero coefficients give the mean albedo; a non-uniform basis makes
    # transposed texel indices detectable
    assert np.array_equal(albedo.morph(mean, basis, np.zeros(basis.shape[0])), mean.astype(np.float64))
    assert not np.allclose(basis[0], np.transpose(basis[0], (1, 0, 2)))


def test_chain_through_the_render_matches_finite_differences():
    """J(beta, gamma) = sum adj * render(textures(beta, gamma)) (interior term,
    samples fixed) is affine in the coefficients, so central differences are
    exact up to rounding."""
    sc = synth.make_scene("tiny", width=12, height=12, spp=2, albedo_k=3)
    pr = synth.random_params(sc, 2)
    am = sc.albedo
    rng = np.random.default_rng(5)
    beta, gamma = rng.normal(size=3) * 0.5, rng.normal(size=3) * 0.5
    adj = rng.uniform(0.2, 1.0, (12, 12, 3))

    def with_coef(b, c):
        q = pr.copy()
        q.diffuse = albedo.morph(am.mean_diffuse, am.basis_diffuse, b).astype(np.float32)
        q.specular = albedo.morph(am.mean_specular, am.basis_specular, c).astype(np.float32)
        return q

    g = oracle.grad(sc, with_coef(beta, gamma), adj, terms=oracle.TERM_INTERIOR)
    gb = albedo.adjoint(am.basis_diffuse, g["diffuse"])
    gc = albedo.adjoint(am.basis_specular, g["specular"])
    h = 1e-2
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        # the float32 textures the render reads: difference them exactly
        jp = np.sum(adj * oracle.render(sc, with_coef(beta + e, gamma)))
        jm = np.sum(adj * oracle.render(sc, with_coef(beta - e, gamma)))
        assert (jp - jm) / (2 * h) == pytest.approx(gb[k], rel=2e-4)
        jp = np.sum(adj * oracle.render(sc, with_coef(beta, gamma + e)))
        jm = np.sum(adj * oracle.render(sc, with_coef(beta, gamma - e)))
        assert (jp - jm) / (2 * h) == pytest.approx(gc[k], rel=2e-4)
