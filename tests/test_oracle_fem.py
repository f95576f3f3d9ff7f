"""Pins for the oracle's P1 FEM matrix and Laplace solve (Sec. 2.2).

Fixed by the paper: the FEM system is SPD once one mask pixel exists, and
with every pixel a vertex the 5-point finite-difference scheme is recovered.
Fixed by mathematics: the P1 energy identity, constants and (under the
Neumann condition) linear functions are reproduced, the discrete maximum
principle (non-obtuse triangles give an M-matrix), dense direct solves.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import pins
import seeded_inputs as S


@pytest.mark.parametrize("seed", range(3))
def test_stiffness_energy_identity(oracle_mod, seed):
    m = pins.random_refined_mesh(oracle_mod, 33, rounds=8, seed=seed)
    A = oracle_mod.stiffness(m)
    x = np.random.default_rng(seed).normal(size=m.V)
    np.testing.assert_allclose(x @ (A @ x), pins.p1_energy(m, x), rtol=1e-12)
    # symmetric, zero row sums (constants in the kernel), entries multiples of 1/2
    assert abs(A - A.T).max() == 0
    np.testing.assert_array_equal(np.asarray(A.sum(axis=1)).ravel(), 0.0)
    d = A.data * 2
    np.testing.assert_array_equal(d, np.round(d))


def test_fdm_equivalence_on_fully_refined_mesh(oracle_mod):
    """Every non-mask pixel an unknown vertex: FEM = 5-point FDM (Sec. 2.2)."""
    N = 17
    m = pins.fully_refined_mesh(oracle_mod, N)
    rng = np.random.default_rng(0)
    pix = m.vy.astype(np.int64) * N + m.vx
    mask_pix = rng.uniform(size=N * N) < 0.3
    mask_pix[0] = True
    m = m.with_mask(mask_pix[pix])
    g = rng.uniform(size=int(m.mask.sum()))
    v, it, rr = oracle_mod.solve(m, g, tol=1e-14)
    # independent FDM solve on the pixel grid
    L = pins.fdm_matrix(N).tocsr()
    u_fdm = np.zeros(N * N)
    u_fdm[pix[m.mask.astype(bool)]] = g
    unk = ~mask_pix
    rhs = -(L[unk][:, mask_pix] @ u_fdm[mask_pix])
    u_fdm[unk] = spla.spsolve(L[unk][:, unk].tocsc(), rhs)
    u_fem = np.zeros(N * N)
    u_fem[pix] = v
    np.testing.assert_allclose(u_fem, u_fdm, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(3))
def test_auu_spd(oracle_mod, seed):
    m = pins.random_refined_mesh(oracle_mod, 33, rounds=8, seed=seed)
    rng = np.random.default_rng(seed)
    mk = rng.uniform(size=m.V) < 0.3
    mk[rng.integers(m.V)] = True
    m = m.with_mask(mk)
    A = oracle_mod.stiffness(m).toarray()
    U = ~mk
    assert np.linalg.eigvalsh(A[np.ix_(U, U)]).min() > 1e-10


@pytest.mark.parametrize("seed", range(3))
def test_solve_matches_dense_direct(oracle_mod, seed):
    m = pins.random_refined_mesh(oracle_mod, 33, rounds=9, seed=seed)
    rng = np.random.default_rng(seed)
    mk = rng.uniform(size=m.V) < 0.4
    mk[:4] = True
    m = m.with_mask(mk)
    g = rng.uniform(size=int(mk.sum()))
    v, it, rr = oracle_mod.solve(m, g, tol=1e-14)
    A = oracle_mod.stiffness(m).toarray()
    U, K = ~mk, mk
    xd = np.linalg.solve(A[np.ix_(U, U)], -A[np.ix_(U, K)] @ g)
    np.testing.assert_allclose(v[U], xd, rtol=0, atol=1e-12 * max(1, abs(g).max()))
    np.testing.assert_array_equal(v[K], g)


def test_constants_reproduced(oracle_mod):
    f = S.make_image(65, 1)
    m, _ = oracle_mod.spatial(f, 0.05, 0.01)
    g = np.full(int(m.mask.sum()), 0.37)
    v, _, _ = oracle_mod.solve(m, g)
    u, _, _ = oracle_mod.raster(m, v)
    np.testing.assert_allclose(u, 0.37, rtol=0, atol=1e-13)


def test_linear_reproduced_under_neumann_condition(oracle_mod):
    """u = a + b x is harmonic with zero normal derivative on the top and
    bottom sides; with every vertex on x = 0 and x = N-1 in the mask the FEM
    solution is exactly that linear function."""
    f = S.make_image(65, 2)
    m, _ = oracle_mod.spatial(f, 0.05, 0.01)
    mk = m.mask.astype(bool) | (m.vx == 0) | (m.vx == 64)
    m = m.with_mask(mk)
    a, b = 0.2, 0.01
    g = a + b * m.vx[mk]
    v, _, _ = oracle_mod.solve(m, g, tol=1e-14)
    u, _, _ = oracle_mod.raster(m, v)
    xs = np.arange(65)[None, :].repeat(65, 0)
    np.testing.assert_allclose(u, a + b * xs, rtol=0, atol=1e-12)
    assert (~mk).sum() > 0


@pytest.mark.parametrize("seed", range(3))
def test_discrete_maximum_principle(oracle_mod, seed):
    f = S.make_image(129, seed)
    m, _ = oracle_mod.spatial(f, 0.03, 0.01)
    g = np.random.default_rng(seed).uniform(-1, 2, size=int(m.mask.sum()))
    v, _, _ = oracle_mod.solve(m, g)
    u, _, _ = oracle_mod.raster(m, v)
    assert u.min() >= g.min() - 1e-13 and u.max() <= g.max() + 1e-13


def test_solve_reports_residual_and_warm_start(oracle_mod):
    f = S.make_image(129, 4)
    m, _ = oracle_mod.spatial(f, 0.04, 0.01)
    g = oracle_mod.g_from_f(m, f)
    v, it, rr = oracle_mod.solve(m, g, tol=1e-13)
    assert rr <= 1e-13
    v2, it2, rr2 = oracle_mod.solve(m, g, start=v, tol=1e-13)
    assert it2 == 0 and np.array_equal(v, v2)
