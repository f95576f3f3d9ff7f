"""Pins for the oracle's images of any size (reading R9): a W x H image in
the smallest (2^L + 1)^2 domain, only image pixels as data.

The restriction to the image is checked against the square-domain oracle,
which is pinned on its own (ownership, closed forms, FDM equivalence): the
same mesh with the image padded by its edge values to the whole domain
gives, cropped to the image, the same interpolant, owners, per-triangle
sums and adjoint.  Least squares on a tiny image is checked against a dense
solve, and the loop's invariants (stopping count, mask inside the image)
directly."""
import math

import numpy as np
import pytest

import seeded_inputs as S

SIZES = [(50, 37), (37, 50), (64, 64), (65, 40), (33, 65), (100, 61), (61, 100)]


def _image(W, H, seed):
    return np.ascontiguousarray(S.make_image(max(W, H), seed)[:H, :W])


def _square_twin(oracle_mod, m):
    """The same mesh with the image filling the domain."""
    return oracle_mod.Mesh(m.N, m.vx, m.vy, m.mask, m.ta, m.tb, m.tc)


@pytest.mark.parametrize("W,H", SIZES)
def test_domain_is_the_smallest_square_that_holds_the_image(oracle_mod, W, H):
    m = oracle_mod.mesh_init(W, H)
    assert (m.W, m.H) == (W, H)
    assert (m.N - 1) & (m.N - 2) == 0 and m.N >= max(W, H) and (m.N - 1) // 2 + 1 < max(W, H)
    assert m.V == 4 and m.T == 2


@pytest.mark.parametrize("W,H", SIZES)
def test_restriction_equals_cropped_square_domain(oracle_mod, W, H):
    f = _image(W, H, 3)
    m, _ = oracle_mod.spatial(f, 0.08, 0.05, max_rounds=25)
    sq = _square_twin(oracle_mod, m)
    N = m.N
    f_sq = np.pad(f, ((0, N - H), (0, N - W)), mode="edge")
    g = oracle_mod.g_from_f(m, f)
    np.testing.assert_array_equal(g, oracle_mod.g_from_f(sq, f_sq))  # clamped = edge padding
    v, _, _ = oracle_mod.solve(m, g)
    u, keys, own = oracle_mod.raster(m, v, f, owner=True)
    u_sq, _, own_sq = oracle_mod.raster(sq, v, f_sq, owner=True)
    np.testing.assert_array_equal(u, u_sq[:H, :W])
    np.testing.assert_array_equal(own, own_sq[:H, :W])
    # the keys are the sums over each triangle's image pixels
    d2 = (u_sq[:H, :W] - f.astype(np.float64)) ** 2
    ref = np.bincount(own_sq[:H, :W].ravel(), weights=d2.ravel(), minlength=m.T)
    np.testing.assert_allclose(keys, ref, rtol=1e-12, atol=1e-300)
    assert abs(keys.sum() - d2.sum()) <= 1e-12 * d2.sum()
    # the adjoint of the restricted interpolation: zero outside the image
    r = np.random.default_rng(1).standard_normal((H, W))
    r_sq = np.zeros((N, N))
    r_sq[:H, :W] = r
    np.testing.assert_allclose(oracle_mod.scatter(m, r), oracle_mod.scatter(sq, r_sq), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("W,H", SIZES)
def test_loop_invariants(oracle_mod, W, H):
    f = _image(W, H, 5)
    density = 0.06
    m, log = oracle_mod.spatial(f, density, 0.02)
    vstar = math.ceil(density * W * H)
    assert vstar == oracle_mod.vstar(W, density, H)
    assert m.V >= vstar and log[-1, 0] < vstar
    # the padding holds no unknowns: every vertex outside the image is a mask vertex
    assert np.all(m.mask[(m.vx >= W) | (m.vy >= H)] == 1)
    # triangles whose bounding box misses the image are never eligible
    xmin = np.minimum(np.minimum(m.vx[m.ta], m.vx[m.tb]), m.vx[m.tc])
    ymin = np.minimum(np.minimum(m.vy[m.ta], m.vy[m.tb]), m.vy[m.tc])
    assert not np.any(oracle_mod.eligible(m) & ((xmin >= W) | (ymin >= H)))
    # every image pixel has exactly one owner
    g = oracle_mod.g_from_f(m, f)
    v, _, _ = oracle_mod.solve(m, g)
    _, _, own = oracle_mod.raster(m, v, None, owner=True)
    assert own.shape == (H, W) and own.min() >= 0


def test_constant_image_is_reproduced(oracle_mod):
    f = np.full((37, 50), 0.375, np.float32)
    m, _ = oracle_mod.spatial(f, 0.1, 0.05, max_rounds=8)
    v, _, _ = oracle_mod.solve(m, oracle_mod.g_from_f(m, f))
    u, keys, _ = oracle_mod.raster(m, v, f)
    np.testing.assert_allclose(u, 0.375, rtol=0, atol=1e-13)
    assert keys.max() <= 1e-24


def test_tonal_least_squares_on_a_tiny_image(oracle_mod):
    """g* = argmin ||B g - f||^2 over the image pixels: CGLS against a dense
    least-squares solve with B formed column by column.  A mask vertex
    outside the image whose triangles hold no image pixel has a zero column,
    so the minimiser is not unique; CGLS from g0 stays in g0 + range(B^T)
    and converges to the minimiser there, g0 + the minimum-norm solution of
    B d = f - B g0."""
    W, H = 7, 5
    f = _image(W, H, 11)
    m, _ = oracle_mod.spatial(f, 0.4, 0.3)
    nK = int(m.mask.sum())
    B = np.stack([oracle_mod.apply_B(m, np.eye(nK)[j]).ravel() for j in range(nK)], axis=1)
    assert B.shape == (W * H, nK)
    g0 = oracle_mod.g_from_f(m, f)
    fd = f.astype(np.float64).ravel()
    g_ls = g0 + np.linalg.lstsq(B, fd - B @ g0, rcond=None)[0]
    g, st = oracle_mod.tonal(m, f, tol=1e-13)
    np.testing.assert_allclose(g, g_ls, rtol=1e-8, atol=1e-10)
    # the columns of vertices that reach no image pixel are zero, and there
    # g keeps its start
    dead = np.flatnonzero(np.abs(B).sum(axis=0) == 0)
    np.testing.assert_array_equal(g[dead], g0[dead])
    # adjoint identity on the restricted operator
    rng = np.random.default_rng(2)
    gg, rr = rng.standard_normal(nK), rng.standard_normal((H, W))
    lhs = float(np.sum(oracle_mod.apply_B(m, gg) * rr))
    rhs = float(gg @ oracle_mod.apply_BT(m, rr))
    assert abs(lhs - rhs) <= 1e-11 * max(1.0, abs(lhs))


def test_square_image_path_unchanged(oracle_mod):
    """A (2^L + 1)^2 image through the image-size constructor gives the
    square-image results."""
    f = S.make_image(65, 8)
    m1, log1 = oracle_mod.spatial(f, 0.1, 0.02)
    m0, log0 = oracle_mod.spatial(f, 0.1, 0.02, mesh=oracle_mod.mesh_init(65))
    np.testing.assert_array_equal(m1.tri, m0.tri)
    np.testing.assert_array_equal(m1.xy, m0.xy)
    np.testing.assert_array_equal(log1, log0)


@pytest.mark.parametrize("W,H", [(50, 37), (33, 65)])
def test_loop_equals_steps_on_an_image_of_any_size(oracle_mod, W, H):
    """The C loop (mask values at clamped positions, warm start, stop count)
    against the same rounds taken one step at a time from the harness."""
    f = _image(W, H, 6)
    m_loop, log = oracle_mod.spatial(f, 0.2, 0.05, max_rounds=6)
    m = oracle_mod.mesh_init(W, H)
    vstar = oracle_mod.vstar(W, 0.2, H)
    for r in range(6):
        v, _, _ = oracle_mod.solve(m, oracle_mod.g_from_f(m, f))
        _, keys, _ = oracle_mod.raster(m, v, f)
        ne = int(oracle_mod.eligible(m).sum())
        k = oracle_mod.topk_count(m.T, 0.05, ne, vstar - m.V)
        assert k == int(log[r, 2])
        sel, margin = oracle_mod.select_topk(m, keys, k)
        assert margin == pytest.approx(log[r, 3], rel=1e-6)
        m, _ = oracle_mod.refine(m, sel)
    np.testing.assert_array_equal(m.tri, m_loop.tri)
    np.testing.assert_array_equal(m.xy, m_loop.xy)
    np.testing.assert_array_equal(m.mask, m_loop.mask)



def test_images_less_than_half_the_domain_high_refine(oracle_mod):
    """100 x 61 in the 129 x 129 domain: both initial triangles bisect at
    (64, 64), below the image.  The selected midpoint becomes a mask vertex
    with the nearest image pixel's value, and the loop goes on to the vertex
    target."""
    W, H = 100, 61
    f = _image(W, H, 3)
    m, log = oracle_mod.spatial(f, 0.1, 0.02)
    assert m.V >= oracle_mod.vstar(W, 0.1, H) and len(log) > 10
    first = oracle_mod.refine(oracle_mod.mesh_init(W, H), [0])[0]
    assert first.V == 5 and first.mask[4] == 1 and (first.vx[4], first.vy[4]) == (64, 64)
    np.testing.assert_array_equal(oracle_mod.g_from_f(first, f)[-1], f[60, 64])
