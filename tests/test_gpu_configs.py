"""Parity at the benchmark configurations' full sizes.

2049 x 2049, 4 % (tonal configuration): the oracle still runs the whole
spatial optimisation (about 16 s), so the mesh is compared bit-exactly; the
tonal result is checked through the oracle's own B and B^T (optimality of
the normal equations, eq. 5); the autograd gradient of 1/2 ||B g - f||^2 is
checked against central differences (h = 1e-4) on 32 random mask vertices.

8193 x 8193, 2 %, textured (very large configuration): the oracle cannot run
the spatial loop (hours), so the checks are sampled outputs it can compute
and properties that hold at any size: bisection-mesh invariants, the
per-triangle errors against the oracle's rasteriser on the GPU's mesh and
vertex values, the FEM residual of the GPU solve with the oracle's
stiffness matrix, and after the workload's 50 tonal iterations the normal
residual of the returned g through the oracle's B and B^T (it must match the
residual the GPU reports) and a smaller error ||B g - f|| than at the start.

Tolerances:
  * optimality: the GPU stops at ||B^T r|| <= 1e-9 ||B^T f|| and returns g in
    float32; rounding g (|dg| <= 2^-24 |g|) moves B^T B g by at most
    ||B^T B|| 2^-24 ||g||, a few 1e-8 relative here -> bound 1e-7;
  * gradient: L is quadratic, so central differences are exact up to the
    error of L (float-float keys, ~1e-13 L, from an FP64 solve at 1e-14),
    i.e. ~1e-6 absolute for L ~ 1e3 and h = 1e-4; the autograd gradient
    comes from the FP32 path (u and r in float32) -> bound 1e-5 max(1, |g'|);
  * keys: as in test_gpu_parity (float-float on the GPU, FP64 in the oracle);
  * FEM residual: the GPU solve stops at relative residual 1e-12 measured in
    float-float; recomputed in FP64 with the oracle's matrix -> bound 1e-11.
"""
import numpy as np
import pytest

import seeded_inputs as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fem():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_01586_gb300 as fem
    return fem


def _oracle_mesh(oracle_mod, N, xy, tri, mk):
    return oracle_mod.Mesh(N, xy[:, 0].copy(), xy[:, 1].copy(), mk.copy(), tri[:, 0].copy(), tri[:, 1].copy(),
                           tri[:, 2].copy())


def test_config_2049_mesh_tonal_and_gradient(oracle_mod, fem):
    from paper_2105_01586_gb300.autograd import TonalLoss
    N = 2049
    f_np = S.make_image(N, 2)
    f = torch.from_numpy(f_np).cuda()
    m = fem.Mesh(N)
    m.spatial_refine(f, 0.04, fem.params(topk_frac=0.01))
    xy, tri, mk = m.export()
    om, log = oracle_mod.spatial(f_np, 0.04, 0.01)
    assert log[:, 3].min() > 1e-9
    assert np.array_equal(om.xy, xy) and np.array_equal(om.tri, tri) and np.array_equal(om.mask, mk)

    g = m.tonal_opt(f, p=fem.params(tonal_tol=1e-9)).double().cpu().numpy()
    c = oracle_mod.apply_BT(om, f_np.astype(np.float64))
    res = oracle_mod.apply_BT(om, oracle_mod.apply_B(om, g) - f_np)
    assert np.linalg.norm(res) <= 1e-7 * np.linalg.norm(c)
    # g itself against the oracle's converged minimiser (the 1e-6 target)
    g_ref, st = oracle_mod.tonal(om, f_np, tol=1e-12)
    assert st["relres"] <= 1e-12
    assert np.linalg.norm(g - g_ref) <= 1e-6 * np.linalg.norm(g_ref)

    g0 = m.g_from_f(f)
    gg = g0.clone().requires_grad_(True)
    TonalLoss.apply(gg, f, m).backward()
    ad = gg.grad.double().cpu().numpy()
    p64 = fem.params(precision=fem.FEM_PREC_FP64, tol=1e-14)

    def L(gv):
        uv = torch.empty(m.V, dtype=torch.float64, device="cuda")
        fem.fem_inpaint(m.h, gv, None, uv, p64)
        return 0.5 * float(m.triangle_errors(uv, f).sum())

    rng = np.random.default_rng(3)
    for k in rng.choice(m.nmask, 32, replace=False):
        gp, gm = g0.clone(), g0.clone()
        gp[k] += 1e-4
        gm[k] -= 1e-4
        h = (float(gp[k]) - float(gm[k])) / 2.0  # the step actually taken in float32
        fd = (L(gp) - L(gm)) / (2.0 * h)
        assert abs(fd - ad[k]) <= 1e-5 * max(1.0, abs(ad[k])), (k, fd, ad[k])


def test_config_8193_sampled(oracle_mod, fem):
    from test_gpu_parity import key_err_tol
    N = 8193
    f_np = S.make_image(N, 3, texture=True)
    f = torch.from_numpy(f_np).cuda()
    m = fem.Mesh(N)
    m.spatial_refine(f, 0.02, fem.params(topk_frac=0.01))
    V, T, K = m.info
    assert V >= int(np.ceil(0.02 * N * N))
    xy, tri, mk = m.export()
    # bisection-mesh invariants (vectorised)
    x, y = xy[:, 0].astype(np.int64), xy[:, 1].astype(np.int64)
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
    cross = (x[b] - x[a]) * (y[c] - y[a]) - (y[b] - y[a]) * (x[c] - x[a])
    assert (cross > 0).all() and cross.sum() == 2 * (N - 1) ** 2
    cax, cay, cbx, cby = x[a] - x[c], y[a] - y[c], x[b] - x[c], y[b] - y[c]
    assert (cax * cbx + cay * cby == 0).all() and (cax ** 2 + cay ** 2 == cbx ** 2 + cby ** 2).all()
    e = np.sort(np.stack([np.concatenate([a, b, c]), np.concatenate([b, c, a])], 1), axis=1)
    key = e[:, 0].astype(np.int64) * V + e[:, 1]
    uk, cnt = np.unique(key, return_counts=True)
    i0, i1 = uk // V, uk % V
    border = ((x[i0] == x[i1]) & np.isin(x[i0], [0, N - 1])) | ((y[i0] == y[i1]) & np.isin(y[i0], [0, N - 1]))
    assert (cnt == np.where(border, 1, 2)).all()
    assert V - len(uk) + T == 1
    # the solve: FEM residual with the oracle's stiffness matrix
    g = m.g_from_f(f)
    _, uv = m.inpaint(g, want_uv=True)
    uvn = uv.cpu().numpy()
    om = _oracle_mesh(oracle_mod, N, xy, tri, mk)
    A = oracle_mod.stiffness(om)
    U, Km = ~mk.astype(bool), mk.astype(bool)
    rhs = -(A[U][:, Km] @ uvn[Km])
    r = A[U][:, U] @ uvn[U] - rhs
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(rhs)
    # per-triangle errors against the oracle's rasteriser (same mesh and values)
    _, keys_ref, own = oracle_mod.raster(om, uvn, f_np, owner=True)
    err = m.triangle_errors(uv, f).cpu().numpy()
    assert (np.abs(err - keys_ref) <= key_err_tol(keys_ref, own, np.abs(uvn).max())).all()
    # 50 tonal iterations (the workload's count): the oracle's B and B^T on
    # the GPU's mesh give the normal residual of the returned g, which must
    # match the residual the GPU reports, and the error ||B g - f|| must fall
    p = fem.params(tonal_tol=0.0, inner_tol=1e-13)
    p.tonal_maxit = 50
    g50 = g.clone()
    fem.fem_tonal_opt(m.h, f, g50, p, allow_not_converged=True)
    st = m.stats()
    assert st["tonal_iters"] == 50
    g50n = g50.double().cpu().numpy()
    c = oracle_mod.apply_BT(om, f_np.astype(np.float64))
    r50 = oracle_mod.apply_B(om, g50n) - f_np
    res = np.linalg.norm(oracle_mod.apply_BT(om, r50)) / np.linalg.norm(c)
    assert abs(res - st["tonal_relres"]) <= 1e-3 * st["tonal_relres"] + 1e-7, (res, st["tonal_relres"])
    r0 = oracle_mod.apply_B(om, g.double().cpu().numpy()) - f_np
    assert np.linalg.norm(r50) < np.linalg.norm(r0)
