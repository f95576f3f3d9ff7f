"""Pins for the oracle's colour spatial optimisation (reading R10: C
channels share the mesh, the mask set and A_UU; each channel has its own
mask values and Laplace solve; a triangle's error is the sum over channels
of its squared errors).  Checked against the grey loop (pinned on its own)
and against the loop's steps taken one at a time."""
import numpy as np
import pytest

import seeded_inputs as S


def _colour(W, H, seeds):
    n = max(W, H)
    return np.stack([S.make_image(n, s)[:H, :W] for s in seeds]).astype(np.float32)


def test_one_channel_is_the_grey_loop(oracle_mod):
    f = S.make_image(65, 3)
    m1, log1 = oracle_mod.spatial(f, 0.1, 0.02)
    m2, log2 = oracle_mod.spatial(f[None], 0.1, 0.02)
    np.testing.assert_array_equal(m1.tri, m2.tri)
    np.testing.assert_array_equal(m1.xy, m2.xy)
    np.testing.assert_array_equal(m1.mask, m2.mask)
    np.testing.assert_array_equal(log1, log2)


def test_identical_channels_select_as_grey(oracle_mod):
    """Two equal channels double every key exactly, so the selection and
    the margins are the grey loop's."""
    f = S.make_image(129, 4)
    m1, log1 = oracle_mod.spatial(f, 0.05, 0.01)
    m2, log2 = oracle_mod.spatial(np.stack([f, f]), 0.05, 0.01)
    np.testing.assert_array_equal(m1.tri, m2.tri)
    np.testing.assert_array_equal(m1.mask, m2.mask)
    np.testing.assert_array_equal(log1[:, 3], log2[:, 3])


@pytest.mark.parametrize("W,H", [(65, 65), (60, 41)])
def test_loop_equals_steps(oracle_mod, W, H):
    f = _colour(W, H, (5, 6, 7))
    m_loop, log = oracle_mod.spatial(f, 0.15, 0.05, max_rounds=6)
    assert log[:, 3].min() > 1e-9
    m = oracle_mod.mesh_init(W, H)
    vstar = oracle_mod.vstar(W, 0.15, H)
    for r in range(6):
        keys = np.zeros(m.T)
        for c in range(3):
            v, _, _ = oracle_mod.solve(m, oracle_mod.g_from_f(m, f[c]))
            _, kc, _ = oracle_mod.raster(m, v, f[c])
            keys = keys + kc
        k = oracle_mod.topk_count(m.T, 0.05, int(oracle_mod.eligible(m).sum()), vstar - m.V)
        assert k == int(log[r, 2])
        sel, margin = oracle_mod.select_topk(m, keys, k)
        assert margin == pytest.approx(log[r, 3], rel=1e-6)
        m, _ = oracle_mod.refine(m, sel)
    np.testing.assert_array_equal(m.tri, m_loop.tri)
    np.testing.assert_array_equal(m.xy, m_loop.xy)
    np.testing.assert_array_equal(m.mask, m_loop.mask)


def test_colour_refines_where_any_channel_has_detail(oracle_mod):
    """A channel that is constant adds nothing; the mesh follows the other."""
    f = S.make_image(65, 8)
    flat = np.full_like(f, 0.25)
    m1, log1 = oracle_mod.spatial(f, 0.1, 0.02)
    m2, log2 = oracle_mod.spatial(np.stack([flat, f, flat]), 0.1, 0.02)
    np.testing.assert_array_equal(m1.tri, m2.tri)
    np.testing.assert_array_equal(m1.mask, m2.mask)
