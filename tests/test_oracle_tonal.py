"""Pins for the oracle's tonal optimisation (Sec. 4, eqs. 4-5).

Fixed by the paper and the mathematics of least squares: the minimiser of
||B g - f||^2 satisfies the normal equations B^T (B g - f) = 0; on tiny
meshes B can be formed column by column and the minimiser found by a dense
least-squares solve; B^T is the adjoint of B; the gradient of
1/2 ||B g - f||^2 is B^T (B g - f) (checked by central differences).
"""
import numpy as np
import pytest

import pins
import seeded_inputs as S


def _tiny_case(oracle_mod, N=17, seed=0, density=0.25):
    f = S.make_image(N, seed)
    m, _ = oracle_mod.spatial(f, density, 0.0)
    return f, m


def _dense_B(oracle_mod, m):
    nK = int(m.mask.sum())
    cols = []
    for k in range(nK):
        e = np.zeros(nK); e[k] = 1.0
        cols.append(oracle_mod.apply_B(m, e).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("seed", range(3))
def test_adjoint_identity(oracle_mod, seed):
    f = S.make_image(65, seed)
    m, _ = oracle_mod.spatial(f, 0.05, 0.01)
    rng = np.random.default_rng(seed)
    g = rng.normal(size=int(m.mask.sum()))
    r = rng.normal(size=(65, 65))
    lhs = np.vdot(oracle_mod.apply_B(m, g), r)
    rhs = np.vdot(g, oracle_mod.apply_BT(m, r))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("seed", range(3))
def test_tonal_matches_dense_lstsq(oracle_mod, seed):
    f, m = _tiny_case(oracle_mod, seed=seed)
    B = _dense_B(oracle_mod, m)
    # each mask pixel's row of B is a unit vector, so B^T B >= I (full column rank)
    kidx = np.flatnonzero(m.mask)
    rows = B[m.vy[kidx].astype(int) * m.N + m.vx[kidx]]
    np.testing.assert_allclose(rows, np.eye(len(kidx)), atol=1e-14)
    g_star = np.linalg.lstsq(B, f.ravel().astype(np.float64), rcond=None)[0]
    g, st = oracle_mod.tonal(m, f, tol=1e-13, maxit=1000)
    np.testing.assert_allclose(g, g_star, rtol=0, atol=1e-9)
    # optimality: B^T (B g - f) = 0, and the error cannot be above the start
    res = B @ g - f.ravel()
    assert np.abs(B.T @ res).max() < 1e-9
    g0 = oracle_mod.g_from_f(m, f)
    assert np.sum(res ** 2) <= np.sum((B @ g0 - f.ravel()) ** 2)
    np.testing.assert_allclose(st["sse"], np.sum(res ** 2), rtol=1e-10)


def test_gradient_by_central_differences(oracle_mod):
    """L(g) = 1/2 ||B g - f||^2 is quadratic, so central differences are exact
    up to rounding; compare with B^T (B g - f) on random vertices."""
    f = S.make_image(33, 5)
    m, _ = oracle_mod.spatial(f, 0.1, 0.01)
    fd = f.astype(np.float64)
    rng = np.random.default_rng(3)
    g = oracle_mod.g_from_f(m, f) + rng.normal(scale=0.05, size=int(m.mask.sum()))
    grad = oracle_mod.apply_BT(m, oracle_mod.apply_B(m, g) - fd)
    L = lambda gg: 0.5 * np.sum((oracle_mod.apply_B(m, gg) - fd) ** 2)
    h = 1e-4
    for k in rng.choice(len(g), size=8, replace=False):
        e = np.zeros_like(g); e[k] = h
        fdk = (L(g + e) - L(g - e)) / (2 * h)
        assert abs(fdk - grad[k]) <= 1e-7 * max(1.0, abs(grad[k])), (k, fdk, grad[k])


def test_tonal_reduces_error_on_medium_image(oracle_mod):
    f = S.make_image(129, 2)
    m, _ = oracle_mod.spatial(f, 0.04, 0.01)
    g0 = oracle_mod.g_from_f(m, f)
    e0 = np.sum((oracle_mod.apply_B(m, g0) - f) ** 2)
    g, st = oracle_mod.tonal(m, f, tol=1e-8)
    assert st["relres"] <= 1e-8
    assert st["sse"] < e0
