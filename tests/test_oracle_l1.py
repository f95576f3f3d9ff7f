"""Pins for the oracle's L1 data term (reading R11 of Sec. 5: iteratively
reweighted least squares with weights 1 / max(|B g - f|, eps)): each step
against a dense weighted least-squares solve, the monotone Huber objective
of the majorise-minimise scheme, and L1 against the L2 minimiser."""
import numpy as np
import pytest

import seeded_inputs as S


def _case(oracle_mod, N=17, seed=3, density=0.3):
    f = S.make_image(N, seed)
    # a few outliers, which the L1 term should largely ignore
    rng = np.random.default_rng(seed)
    idx = rng.choice(N * N, size=N, replace=False)
    f.ravel()[idx] = np.clip(f.ravel()[idx] + rng.choice([-0.6, 0.6], size=N), 0, 1)
    m, _ = oracle_mod.spatial(f, density, 0.1)
    return f, m


def _dense_B(oracle_mod, m):
    nK = int(m.mask.sum())
    return np.stack([oracle_mod.apply_B(m, np.eye(nK)[j]).ravel() for j in range(nK)], axis=1)


def test_irls_steps_equal_dense_weighted_least_squares(oracle_mod):
    f, m = _case(oracle_mod)
    B = _dense_B(oracle_mod, m)
    fd = f.astype(np.float64).ravel()
    eps = 1e-3
    g = oracle_mod.g_from_f(m, f)
    for k in range(1, 5):
        w = 1.0 / np.maximum(np.abs(B @ g - fd), eps)
        sw = np.sqrt(w)
        g = np.linalg.lstsq(B * sw[:, None], fd * sw, rcond=None)[0]  # B has full column rank here
        g_or, st = oracle_mod.tonal_l1(m, f, irls=k, eps=eps, tol=1e-13)
        np.testing.assert_allclose(g_or, g, rtol=1e-7, atol=1e-9)


def test_huber_objective_does_not_increase_and_l1_beats_l2(oracle_mod):
    f, m = _case(oracle_mod, N=33, seed=4, density=0.2)
    eps = 1e-3
    hub = []
    for k in range(0, 7):
        g, st = oracle_mod.tonal_l1(m, f, irls=k, eps=eps, tol=1e-12)
        hub.append(st["huber"])
    assert all(b <= a * (1 + 1e-9) for a, b in zip(hub, hub[1:])), hub
    g2, _ = oracle_mod.tonal(m, f, tol=1e-12)
    l1_of_l2 = np.abs(oracle_mod.apply_B(m, g2) - f.astype(np.float64)).sum()
    assert st["l1"] < l1_of_l2


def test_zero_steps_leave_g_unchanged(oracle_mod):
    f, m = _case(oracle_mod)
    g0 = oracle_mod.g_from_f(m, f)
    g, st = oracle_mod.tonal_l1(m, f, irls=0)
    np.testing.assert_array_equal(g, g0)
    assert st["l1"] == pytest.approx(np.abs(oracle_mod.apply_B(m, g0) - f.astype(np.float64)).sum(), rel=1e-12)


def test_irls_reaches_the_linear_programming_l1_minimum(oracle_mod):
    """min_g sum_p |(B g)_p - f_p| is a linear program (g free, t >= |B g - f|);
    the Huber minimiser's L1 objective is within P eps / 2 of its optimum, since
    |r| - eps/2 <= huber(r) <= |r|."""
    linprog = pytest.importorskip("scipy.optimize").linprog
    f, m = _case(oracle_mod, N=17, seed=5, density=0.3)
    B = _dense_B(oracle_mod, m)
    fd = f.astype(np.float64).ravel()
    P, nK = B.shape
    c = np.concatenate([np.zeros(nK), np.ones(P)])
    I = np.eye(P)
    A = np.block([[B, -I], [-B, -I]])
    b = np.concatenate([fd, -fd])
    lp = linprog(c, A_ub=A, b_ub=b, bounds=[(None, None)] * nK + [(0, None)] * P, method="highs")
    assert lp.status == 0
    eps = 1e-4
    _, st = oracle_mod.tonal_l1(m, f, irls=80, eps=eps, tol=1e-12)
    assert st["l1"] >= lp.fun - 1e-9
    assert st["l1"] <= lp.fun + P * eps / 2, (st["l1"], lp.fun)
