"""The premise of the incremental error pass, on the oracle: a triangle's
key (Sec. 3, the squared error over its owned pixels) depends only on its
corners, its vertex values and the image.  Between two rounds of the
spatial loop, every triangle that keeps its id, its corners and the bits of
its three vertex values keeps the bits of its key; the others are the ones
an incremental pass must recompute."""
import numpy as np

import seeded_inputs as S


def test_unchanged_triangles_keep_their_keys(oracle_mod):
    N, density, frac = 257, 0.06, 0.01
    f = S.make_image(N, 4)
    m = oracle_mod.mesh_init(N)
    vs = oracle_mod.vstar(N, density)
    prev = None
    checked = kept = 0
    for _ in range(40):
        if m.V >= vs:
            break
        g = oracle_mod.g_from_f(m, f)
        start = None
        if prev is not None:
            # warm start: the previous values, new vertices at the mean of the
            # edge they bisect
            start = np.zeros(m.V)
            start[: len(prev["uv"])] = prev["uv"]
            par = info["parents"]
            start[m.V - len(par):] = 0.5 * (start[par[:, 0]] + start[par[:, 1]])
        uv, _, _ = oracle_mod.solve(m, g, start=start)
        _, keys, _ = oracle_mod.raster(m, uv, f)
        tri = m.tri[:, :3].copy()
        if prev is not None:
            T0, V0 = len(prev["tri"]), len(prev["uv"])
            same_geom = np.all(tri[:T0] == prev["tri"], axis=1)
            vb, pb = uv[:V0].view(np.int64), prev["uv"].view(np.int64)
            vchg = np.zeros(m.V, bool)
            vchg[:V0] = vb != pb
            vchg[V0:] = True
            same_vals = ~vchg[tri[:T0]].any(axis=1)
            clean = same_geom & same_vals
            checked += T0
            kept += int(clean.sum())
            np.testing.assert_array_equal(keys[:T0][clean].view(np.int64), prev["keys"][clean].view(np.int64))
        k = oracle_mod.topk_count(m.T, frac, int(oracle_mod.eligible(m).sum()), vs - m.V)
        sel, _ = oracle_mod.select_topk(m, keys, k)
        prev = {"uv": uv, "keys": keys, "tri": tri}
        m, info = oracle_mod.refine(m, sel)
    # the check saw many triangles that an incremental pass would keep
    assert kept > 0.3 * checked, (kept, checked)
