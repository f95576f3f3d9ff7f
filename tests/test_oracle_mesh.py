"""Pins for the oracle's mesh, newest-vertex bisection and rasterisation.

The initial mesh and the NVB rules replace the Delaunay mesh of Sec. 2.2; the
rasterisation is the linear interpolation at the end of Sec. 2.2 and the
per-triangle error of Sec. 3.  Nothing here compares the oracle with itself:
the checks are geometry (conformity, Euler, areas, right-isosceles shapes),
a recursive textbook NVB, exact coverage of the pixel grid and exact
reproduction of linear data.
"""
import numpy as np
import pytest

import pins


def _check_mesh_invariants(m):
    N = m.N
    vx, vy = m.vx.astype(np.int64), m.vy.astype(np.int64)
    # vertices on the pixel grid and distinct
    assert vx.min() >= 0 and vy.min() >= 0 and vx.max() <= N - 1 and vy.max() <= N - 1
    assert len(set(zip(vx.tolist(), vy.tolist()))) == m.V
    a, b, c = m.ta, m.tb, m.tc
    abx, aby = vx[b] - vx[a], vy[b] - vy[a]
    cax, cay = vx[a] - vx[c], vy[a] - vy[c]
    cbx, cby = vx[b] - vx[c], vy[b] - vy[c]
    cross = abx * (vy[c] - vy[a]) - aby * (vx[c] - vx[a])
    assert (cross > 0).all(), "orientation must be positive for every triangle"
    # right angle at the newest vertex, equal legs: refinement edge = hypotenuse
    assert (cax * cbx + cay * cby == 0).all()
    assert (cax * cax + cay * cay == cbx * cbx + cby * cby).all()
    # areas tile the image
    assert cross.sum() == 2 * (N - 1) ** 2
    # conformity: interior edges in exactly two triangles, boundary edges in one
    E = pins.edges_of(m)
    for (i, j), n in E.items():
        on_border = ((vx[i] == vx[j]) and vx[i] in (0, N - 1)) or ((vy[i] == vy[j]) and vy[i] in (0, N - 1))
        assert n == (1 if on_border else 2), ((i, j), n)
    # Euler characteristic of a disk
    assert m.V - len(E) + m.T == 1


def test_initial_mesh(oracle_mod):
    m = oracle_mod.mesh_init(17)
    assert m.V == 4 and m.T == 2
    assert m.xy.tolist() == [[0, 0], [16, 0], [0, 16], [16, 16]]
    assert m.mask.tolist() == [1, 1, 1, 1]
    _check_mesh_invariants(m)


@pytest.mark.parametrize("N", [2, 4, 6, 10])
def test_bad_sizes_rejected(oracle_mod, N):
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.mesh_init(N)


@pytest.mark.parametrize("seed", range(6))
def test_refine_invariants_random(oracle_mod, seed):
    m = pins.random_refined_mesh(oracle_mod, 33, rounds=12, seed=seed)
    _check_mesh_invariants(m)


@pytest.mark.parametrize("seed", range(8))
def test_refine_matches_recursive_textbook_nvb(oracle_mod, seed):
    """Closure-based refinement equals the recursive NVB (unique smallest
    conforming refinement), including the newest-vertex labels."""
    rng = np.random.default_rng(100 + seed)
    m = pins.random_refined_mesh(oracle_mod, 17, rounds=4, seed=seed, frac=0.3)
    for _ in range(3):
        el = np.flatnonzero(oracle_mod.eligible(m))
        sel = np.sort(rng.choice(el, size=max(1, len(el) // 5), replace=False))
        before = pins.triangle_set(m)
        sel_tris = [list(pins.triangle_set(oracle_mod.Mesh(m.N, m.vx, m.vy, m.mask, m.ta[[t]], m.tb[[t]], m.tc[[t]])))[0]
                    for t in sel]
        ref_tris, ref_masks = pins.nvb_recursive(list(before), sel_tris)
        m2, info = oracle_mod.refine(m, sel)
        assert pins.triangle_set(m2) == ref_tris
        new = range(m.V, m2.V)
        new_mask = {(int(m2.vx[i]), int(m2.vy[i])) for i in new if m2.mask[i]}
        assert new_mask == ref_masks
        assert info["generations"] <= 2
        m = m2


def test_refine_numbering_rule(oracle_mod):
    """New vertices in ascending pixel index; old ids and old triangles'
    parent slots preserved; new triangle ids appended."""
    m = pins.random_refined_mesh(oracle_mod, 33, rounds=6, seed=3)
    el = np.flatnonzero(oracle_mod.eligible(m))
    m2, info = oracle_mod.refine(m, el[::3])
    assert (m2.vx[: m.V] == m.vx).all() and (m2.vy[: m.V] == m.vy).all()
    pix = m2.vy[m.V:].astype(np.int64) * m.N + m2.vx[m.V:]
    assert (np.diff(pix) > 0).all()
    assert info["new_vertices"] == m2.V - m.V and info["new_triangles"] == m2.T - m.T
    # a triangle keeps its id only as its first child: (c, a, m) of the parent
    for t in range(m.T):
        if (m2.ta[t], m2.tb[t], m2.tc[t]) != (m.ta[t], m.tb[t], m.tc[t]):
            assert m2.ta[t] in (m.tc[t], ) or m2.tb[t] == m.tc[t]


def test_closure_never_reaches_unit_triangles(oracle_mod):
    """Eligibility: unit right triangles (midpoint off the grid) are never
    selected, and closure never asks to bisect one."""
    m = oracle_mod.mesh_init(9)
    rng = np.random.default_rng(7)
    for _ in range(40):
        el = np.flatnonzero(oracle_mod.eligible(m))
        if len(el) == 0:
            break
        m, _ = oracle_mod.refine(m, rng.choice(el, size=1))
    _check_mesh_invariants(m)
    inel = np.flatnonzero(~oracle_mod.eligible(m))
    if len(inel):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.refine(m, inel[:1])


@pytest.mark.parametrize("N", [3, 5, 9, 17])
def test_full_refinement_reaches_every_pixel(oracle_mod, N):
    m = pins.fully_refined_mesh(oracle_mod, N)
    assert m.V == N * N and m.T == 2 * (N - 1) ** 2
    _check_mesh_invariants(m)


@pytest.mark.parametrize("seed", range(5))
def test_every_pixel_owned_once_by_a_containing_triangle(oracle_mod, seed):
    m = pins.random_refined_mesh(oracle_mod, 33, rounds=10, seed=seed)
    _, _, own = oracle_mod.raster(m, np.zeros(m.V), owner=True)  # raises unless owned exactly once
    ys, xs = np.mgrid[0:33, 0:33]
    assert pins.in_closed_triangle(m, own.ravel(), xs.ravel(), ys.ravel()).all()
    # pixel counts per triangle add up to the image
    assert np.bincount(own.ravel(), minlength=m.T).sum() == 33 * 33


@pytest.mark.parametrize("seed", range(4))
def test_raster_reproduces_linear_data_exactly(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    m = pins.random_refined_mesh(oracle_mod, 65, rounds=10, seed=seed)
    c0, cx, cy = rng.normal(size=3)
    v = c0 + cx * m.vx + cy * m.vy
    u, _, _ = oracle_mod.raster(m, v)
    ys, xs = np.mgrid[0:65, 0:65]
    np.testing.assert_allclose(u, c0 + cx * xs + cy * ys, rtol=0, atol=1e-12)
    # at vertex pixels the interpolant is the vertex value itself
    w = rng.normal(size=m.V)
    u2, _, _ = oracle_mod.raster(m, w)
    np.testing.assert_array_equal(u2[m.vy, m.vx], w)


def test_raster_matches_barycentric_solve(oracle_mod):
    """u at each pixel equals the interpolant from barycentric coordinates
    found by a 3x3 linear solve on the owner triangle."""
    m = pins.random_refined_mesh(oracle_mod, 17, rounds=6, seed=11)
    rng = np.random.default_rng(1)
    v = rng.normal(size=m.V)
    u, _, own = oracle_mod.raster(m, v, owner=True)
    for y in range(17):
        for x in range(17):
            t = own[y, x]
            ids = [m.ta[t], m.tb[t], m.tc[t]]
            M = np.array([[m.vx[i] for i in ids], [m.vy[i] for i in ids], [1.0, 1.0, 1.0]])
            lam = np.linalg.solve(M, [x, y, 1.0])
            assert abs(lam @ v[ids] - u[y, x]) < 1e-12


def test_keys_sum_to_sse(oracle_mod):
    import seeded_inputs as S
    f = S.make_image(65, 3)
    m = pins.random_refined_mesh(oracle_mod, 65, rounds=8, seed=2)
    v = np.random.default_rng(0).uniform(size=m.V)
    u, keys, own = oracle_mod.raster(m, v, f, owner=True)
    sse = ((u - f.astype(np.float64)) ** 2)
    np.testing.assert_allclose(keys.sum(), sse.sum(), rtol=1e-12)
    np.testing.assert_allclose(keys, np.bincount(own.ravel(), weights=sse.ravel(), minlength=m.T), rtol=1e-12, atol=1e-300)


def test_topk_against_lexsort(oracle_mod):
    m = pins.random_refined_mesh(oracle_mod, 65, rounds=8, seed=4)
    rng = np.random.default_rng(5)
    keys = np.round(rng.uniform(size=m.T), 2)  # many exact ties
    el = oracle_mod.eligible(m)
    for k in (1, 3, 17, int(el.sum())):
        sel, margin = oracle_mod.select_topk(m, keys, k)
        ids = np.flatnonzero(el)
        order = ids[np.lexsort((ids, -keys[ids]))]
        assert sel.tolist() == order[:k].tolist()
    assert oracle_mod.topk_count(100, 0.01, 50, 1000) == 1
    assert oracle_mod.topk_count(101, 0.01, 50, 1000) == 2
    assert oracle_mod.topk_count(1000, 0.0, 50, 1000) == 1
    assert oracle_mod.topk_count(1000, 0.5, 50, 1000) == 50
    assert oracle_mod.topk_count(1000, 0.5, 500, 7) == 7


def test_refinement_records_the_bisected_edge_of_each_new_vertex(oracle_mod):
    """info["parents"] gives, for every new vertex, the two vertices of the
    edge it bisects: the new vertex is their midpoint, and both existed
    before the round."""
    import seeded_inputs as S
    f = S.make_image(65, 4)
    m = oracle_mod.mesh_init(65)
    for _ in range(8):
        v, _, _ = oracle_mod.solve(m, oracle_mod.g_from_f(m, f))
        _, keys, _ = oracle_mod.raster(m, v, f)
        k = oracle_mod.topk_count(m.T, 0.05, int(oracle_mod.eligible(m).sum()), 10 ** 6)
        sel, _ = oracle_mod.select_topk(m, keys, k)
        V0 = m.V
        m, info = oracle_mod.refine(m, sel)
        par = info["parents"]
        assert par.shape == (m.V - V0, 2)
        assert par.max() < V0 and par.min() >= 0
        new = np.arange(V0, m.V)
        assert np.array_equal(2 * m.vx[new], m.vx[par[:, 0]] + m.vx[par[:, 1]])
        assert np.array_equal(2 * m.vy[new], m.vy[par[:, 0]] + m.vy[par[:, 1]])
