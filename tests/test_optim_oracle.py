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


def _stage_point(rng, n=7):
    d = rng.uniform(-0.4, 4.0, n)
    a = rng.uniform(-0.2, 1.3, n)
    a[a > 0.0] = np.maximum(a[a > 0.0], 0.05)           # away from the kink of sqrt at 0
    p = rng.uniform(-0.2, 0.9, (n, 2))
    return np.concatenate([d, a, p.ravel()]), rng.uniform(-0.3, 1.5, (n, 3))


def test_stage_geometry_gradients_match_fd():
    rng = np.random.default_rng(4)
    x, i = _stage_point(rng)
    x[7:14] = np.abs(x[7:14]) + 0.05                    # the prior needs a > 0
    g = optim.stage_grad(x, i, 0.01, 1.0)
    d, a, _ = optim.stage_split(x)
    m_fixed = (i * (d * d / a)[:, None]).mean(axis=1, keepdims=True)
    f = lambda z: optim.stage_light_energy(z, i, 0.01) + optim.stage_box_energy(z, 1.0)
    for k, fd in _fd(f, x, h=1e-7, n=x.size):
        assert g.flat[k] == pytest.approx(fd, rel=1e-5, abs=1e-7), k
    # the prior's gradient in d and a is the same whether or not m_j is held fixed
    fm = lambda z: optim.stage_light_energy(z, i, 0.01, mean_fixed=m_fixed) + optim.stage_box_energy(z, 1.0)
    for k, fd in _fd(fm, x, h=1e-7, n=x.size):
        assert g.flat[k] == pytest.approx(fd, rel=1e-5, abs=1e-7), k


def test_stage_box_closed_forms():
    # a light at its face's centroid with a = 1 fills the face: in range, zero energy
    n = 3
    x = np.concatenate([np.full(n, 2.0), np.ones(n), np.full(2 * n, 1.0 / 3.0)])
    assert optim.stage_box_energy(x, 1.0) == pytest.approx(0.0, abs=1e-30)
    # a point light (a = 0) may sit anywhere in the face, corners included
    x = np.concatenate([[1.0], [0.0], [1.0, 0.0]])
    assert optim.stage_box_energy(x, 1.0) == 0.0
    # corner p = (1, 0, 0) with a = 0.36: two coordinates are 0.2 below sqrt(a)/3 = 0.2
    x = np.concatenate([[1.0], [0.36], [1.0, 0.0]])
    assert optim.stage_box_energy(x, 2.0) == pytest.approx(2.0 * 2 * 0.2 ** 2)
    # d below zero and a above one: plain quadratic boxes
    x = np.concatenate([[-0.5], [1.5], [1.0 / 3.0, 1.0 / 3.0]])
    r = np.sqrt(1.5) / 3.0 - 1.0 / 3.0
    assert optim.stage_box_energy(x, 1.0) == pytest.approx(0.25 + 0.25 + 3 * r * r)
    # a grey light has no prior energy whatever its geometry
    x = np.concatenate([[2.5], [0.3], [0.2, 0.5]])
    assert optim.stage_light_energy(x, np.full((1, 3), 0.7), 0.01) == pytest.approx(0.0, abs=1e-30)
    assert np.allclose(optim.stage_grad(x, np.full((1, 3), 0.7), 0.01, 0.0), 0.0)


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
