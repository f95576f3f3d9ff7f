"""Pins for the oracle's spatial optimisation loop (Sec. 3, adapted to top-k
newest-vertex bisection).  The loop is a composition of pinned pieces; these
tests check the composition against the same steps taken one at a time, the
stopping rule and the mask rule."""
import math

import numpy as np
import pytest

import seeded_inputs as S


def test_loop_equals_steps(oracle_mod):
    f = S.make_image(65, 6)
    m_loop, log = oracle_mod.spatial(f, 0.2, 0.05, max_rounds=6)
    m = oracle_mod.mesh_init(65)
    Vstar = oracle_mod.vstar(65, 0.2)
    for r in range(6):
        g = oracle_mod.g_from_f(m, f)
        v, it, rr = oracle_mod.solve(m, g)
        _, keys, _ = oracle_mod.raster(m, v, f)
        ne = int(oracle_mod.eligible(m).sum())
        k = oracle_mod.topk_count(m.T, 0.05, ne, Vstar - m.V)
        assert k == int(log[r, 2])
        assert k == min(max(1, math.ceil(0.05 * m.T)), ne, Vstar - m.V)
        sel, margin = oracle_mod.select_topk(m, keys, k)
        # selected triangles that share their refinement edge give one mask vertex
        distinct = {(min(int(m.ta[t]), int(m.tb[t])), max(int(m.ta[t]), int(m.tb[t]))) for t in sel}
        m, info = oracle_mod.refine(m, sel)
        assert info["new_mask"] == len(distinct)
    for a, b in ((m.vx, m_loop.vx), (m.vy, m_loop.vy), (m.mask, m_loop.mask), (m.ta, m_loop.ta),
                 (m.tb, m_loop.tb), (m.tc, m_loop.tc)):
        np.testing.assert_array_equal(a, b)


def test_mask_is_selected_midpoints(oracle_mod):
    f = S.make_image(65, 7)
    m, _ = oracle_mod.spatial(f, 0.1, 0.02, max_rounds=10)
    g = oracle_mod.g_from_f(m, f)
    v, _, _ = oracle_mod.solve(m, g)
    _, keys, _ = oracle_mod.raster(m, v, f)
    sel, _ = oracle_mod.select_topk(m, keys, 9)
    mids = {((int(m.vx[m.ta[t]]) + int(m.vx[m.tb[t]])) // 2, (int(m.vy[m.ta[t]]) + int(m.vy[m.tb[t]])) // 2) for t in sel}
    m2, info = oracle_mod.refine(m, sel)
    new_mask = {(int(m2.vx[i]), int(m2.vy[i])) for i in range(m.V, m2.V) if m2.mask[i]}
    new_unknown = {(int(m2.vx[i]), int(m2.vy[i])) for i in range(m.V, m2.V) if not m2.mask[i]}
    assert new_mask == mids
    assert not (new_unknown & mids)


@pytest.mark.parametrize("N,density,frac", [(65, 0.05, 0.0), (129, 0.03, 0.01)])
def test_stop_rule(oracle_mod, N, density, frac):
    f = S.make_image(N, 8)
    m, log = oracle_mod.spatial(f, density, frac)
    Vstar = math.ceil(density * N * N)
    assert m.V >= Vstar
    assert log[-1, 0] < Vstar  # the last round started below the target
    assert (np.diff(log[:, 0]) > 0).all()
    assert (log[:, 5] <= 1e-13).all()


def test_config_targets():
    assert math.ceil(0.05 * 257 * 257) == 3303
    assert math.ceil(0.03 * 1025 * 1025) == 31519
    assert math.ceil(0.02 * 8193 * 8193) == 1342505
