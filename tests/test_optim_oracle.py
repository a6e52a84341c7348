"""Pins of the optimiser oracle: finite differences of the regulariser energies
and Adam's closed-form behaviour."""
import numpy as np
import pytest

from oracle import optim


def _fd(f, x, h=1e-6, n=40, seed=0):
    rng = np.random.default_rng(seed)
    idx = rng.choice(x.size, size=min(n, x.size), replace=False)
    out = []
    for i in idx:
        xp, xm = x.copy(), x.copy()
        xp.flat[i] += h
        xm.flat[i] -= h
        out.append((i, (f(xp) - f(xm)) / (2 * h)))
    return out


def test_coef_and_light_gradients_match_fd():
    rng = np.random.default_rng(1)
    x = rng.normal(size=30)
    x[20:] = rng.uniform(-0.5, 1.5, 10)
    g = optim.coef_grad(x, 20, 0.0025, 1.0)
    for i, fd in _fd(lambda z: optim.coef_energy(z, 20, 0.0025, 1.0), x):
        assert g.flat[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    li = rng.uniform(-0.3, 1.5, (8, 3))
    sc = rng.uniform(1.0, 9.0, 8)
    gl = optim.light_grad(li, sc, 0.01, 1.0)
    m_fixed = (li * sc[:, None]).mean(axis=1, keepdims=True)   # the prior's mean is held fixed
    for i, fd in _fd(lambda z: optim.light_energy(z, sc, 0.01, 1.0, mean_fixed=m_fixed), li):
        assert gl.flat[i] == pytest.approx(fd, rel=1e-6, abs=1e-9)


@pytest.mark.parametrize("rgb", [True, False])
def test_texture_regulariser_gradients_match_fd(rgb):
    rng = np.random.default_rng(2)
    M = 9
    X = rng.uniform(-0.2, 1.2, (M, M, 3) if rgb else (M, M))
    X0 = rng.uniform(0.1, 0.9, (M, M, 3)) if rgb else None
    args = (0.0002, 0.3, 0.3 if rgb else 0.0, 1.0, X0)
    G = optim.tex_grad(X, *args)
    for i, fd in _fd(lambda Z: optim.tex_energy(Z, *args), X, n=80):
        assert G.flat[i] == pytest.approx(fd, rel=1e-5, abs=1e-8)


def test_smoothness_of_constant_and_ramp():
    assert optim.smooth_energy(np.full((5, 5), 0.3)) == 0.0
    ramp = np.tile(np.arange(4.0), (4, 1))          # horizontal unit steps, 4 rows x 3 pairs
    assert optim.smooth_energy(ramp) == pytest.approx(2.0 * 12.0)
    assert optim.sym_energy(np.tile(np.array([0.1, 0.5, 0.1]), (2, 1))) == 0.0


def test_adam_first_step_moves_by_lr_sign():
    """From zero moments, bias correction makes the first update lr * g/(|g| + eps)."""
    rng = np.random.default_rng(3)
    x = rng.normal(size=50)
    g = rng.normal(size=50)
    x1, m, v = optim.adam(x, g, np.zeros(50), np.zeros(50), 1, 0.01)
    assert np.allclose(x - x1, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    # a constant gradient keeps the bias-corrected step at lr * g/(|g| + eps)
    for s in range(2, 6):
        x2, m, v = optim.adam(x1, g, m, v, s, 0.01)
        assert np.allclose(x1 - x2, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-9)
        x1 = x2
