"""GPU parity against the CPU oracle, through the C ABI.

Tolerances (derived from the arithmetic):
  * mesh topology, pixel ownership: bit-exact (integer work);
  * per-triangle errors: the GPU evaluates u and (u - f)^2 in float-float
    (about 48 bits) and the oracle in FP64, so per pixel |du| <= 2^-47 max|v|
    and, by Cauchy-Schwarz over the n_t pixels of triangle t,
    |d key_t| <= 2 |du| sqrt(n_t key_t) + 1e-12 key_t (key_err_tol below);
  * inpainting solve: vertex values relative L2 1e-9 (FP32-IR and FP64 both
    stop at FP64 relative residual 1e-12; the oracle at 1e-14);
  * u image (float32 output): absolute 2e-7 (one float32 rounding of values
    in [0, 1] plus the solve error);
  * tonal optimisation: g relative L2 1e-6 (the stated target);
  * adjoint: relative L2 1e-6 against the oracle's B^T r (float32 input and
    output), and the adjoint identity <B g, r> = <g, B^T r> to 1e-6.
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


def key_err_tol(keys_ref, own, vmax):
    n_t = np.bincount(own.ravel(), minlength=len(keys_ref)).astype(np.float64)
    du = 2.0 ** -47 * max(1.0, vmax)
    return 2.0 * du * np.sqrt(n_t * keys_ref) + 1e-12 * keys_ref + 1e-300


def _gpu_mesh(fem, om):
    m = fem.Mesh(om.N)
    m.import_(om.xy, om.tri, om.mask)
    return m


def _same_mesh(m, om):
    xy, tri, mk = m.export()
    return np.array_equal(xy, om.xy) and np.array_equal(tri, om.tri) and np.array_equal(mk, om.mask)


@pytest.mark.parametrize("N,seed,density,frac", [(33, 0, 0.3, 0.05), (129, 1, 0.05, 0.01), (257, 2, 0.02, 0.01)])
def test_triangle_errors_and_raster(oracle_mod, fem, N, seed, density, frac):
    f_np = S.make_image(N, seed)
    om, _ = oracle_mod.spatial(f_np, density, frac)
    m = _gpu_mesh(fem, om)
    rng = np.random.default_rng(seed)
    v = rng.uniform(-0.5, 1.5, size=om.V)
    u_ref, keys_ref, own_ref = oracle_mod.raster(om, v, f_np, owner=True)
    uv = torch.from_numpy(v).cuda()
    f = torch.from_numpy(f_np).cuda()
    err = m.triangle_errors(uv, f).cpu().numpy()
    assert (np.abs(err - keys_ref) <= key_err_tol(keys_ref, own_ref, np.abs(v).max())).all()
    u, own = m.rasterize(uv, want_owner=True)
    np.testing.assert_array_equal(own.cpu().numpy(), own_ref)
    np.testing.assert_allclose(u.cpu().numpy(), u_ref, rtol=0, atol=2e-7 * max(1.0, np.abs(v).max()))


def test_raster_full_refinement_and_initial_mesh(oracle_mod, fem):
    """Degenerate extremes: the 2-triangle mesh and the fully refined mesh
    (every pixel a vertex, triangles owning zero or one pixel)."""
    import pins
    for om in (oracle_mod.mesh_init(17), pins.fully_refined_mesh(oracle_mod, 17)):
        m = _gpu_mesh(fem, om)
        v = np.random.default_rng(0).normal(size=om.V)
        f_np = S.make_image(17, 3)
        u_ref, keys_ref, own_ref = oracle_mod.raster(om, v, f_np, owner=True)
        err = m.triangle_errors(torch.from_numpy(v).cuda(), torch.from_numpy(f_np).cuda()).cpu().numpy()
        assert (np.abs(err - keys_ref) <= key_err_tol(keys_ref, own_ref, np.abs(v).max())).all()
        _, own = m.rasterize(torch.from_numpy(v).cuda(), want_owner=True)
        np.testing.assert_array_equal(own.cpu().numpy(), own_ref)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,seed", [(65, 3), (513, 4)])
def test_inpaint_matches_oracle(oracle_mod, fem, N, seed, prec):
    f_np = S.make_image(N, seed)
    om, _ = oracle_mod.spatial(f_np, 0.04, 0.01)
    m = _gpu_mesh(fem, om)
    g_np = oracle_mod.g_from_f(om, f_np)  # f is float32, so g is exactly representable
    v_ref, _, _ = oracle_mod.solve(om, g_np, tol=1e-14)
    g = torch.from_numpy(g_np.astype(np.float32)).cuda()
    u, uv = m.inpaint(g, fem.params(precision=prec), want_uv=True)
    uv = uv.cpu().numpy()
    assert np.linalg.norm(uv - v_ref) <= 1e-9 * np.linalg.norm(v_ref)
    u_ref, _, _ = oracle_mod.raster(om, v_ref)
    np.testing.assert_allclose(u.cpu().numpy(), u_ref, rtol=0, atol=2e-7)
    st = m.stats()
    assert st["relres"] <= 1e-12


def test_inpaint_all_mask_and_constants(oracle_mod, fem):
    """No unknown vertices (pure linear spline), and constant data."""
    f_np = S.make_image(65, 5)
    om, _ = oracle_mod.spatial(f_np, 0.05, 0.01)
    m = _gpu_mesh(fem, om.with_mask(np.ones(om.V, np.uint8)))
    g = torch.from_numpy(f_np[om.vy, om.vx].copy()).cuda()
    u = m.inpaint(g)
    u_ref, _, _ = oracle_mod.raster(om, f_np[om.vy, om.vx].astype(np.float64))
    np.testing.assert_allclose(u.cpu().numpy(), u_ref, atol=2e-7)
    m2 = _gpu_mesh(fem, om)
    u2 = m2.inpaint(torch.full((int(om.mask.sum()),), 0.25, device="cuda"))
    np.testing.assert_allclose(u2.cpu().numpy(), 0.25, atol=1e-7)


@pytest.mark.parametrize("N,seed,density,frac", [(65, 0, 0.1, 0.0), (129, 1, 0.05, 0.01), (257, 0, 0.05, 0.0),
                                                  (513, 7, 0.03, 0.01)])
def test_spatial_refine_bit_exact(oracle_mod, fem, N, seed, density, frac):
    f_np = S.make_image(N, seed)
    om, log = oracle_mod.spatial(f_np, density, frac)
    m = fem.Mesh(N)
    f = torch.from_numpy(f_np).cuda()
    m.spatial_refine(f, density, fem.params(topk_frac=frac))
    st = m.stats()
    assert st["rounds"] == len(log)
    assert _same_mesh(m, om), "GPU mesh differs from the oracle mesh"
    assert m.info == (om.V, om.T, int(om.mask.sum()))
    g = m.g_from_f(f).cpu().numpy()
    np.testing.assert_array_equal(g, f_np[om.vy[om.mask.astype(bool)], om.vx[om.mask.astype(bool)]])


@pytest.mark.parametrize("prec", [0, 1])
def test_spatial_refine_config_1025(oracle_mod, fem, prec):
    """1025 x 1025, top-k 1 % per round, 3 % vertex density (the spatial
    optimisation workload), in both precisions: mesh bit-exact."""
    f_np = S.make_image(1025, 1)
    om, log = oracle_mod.spatial(f_np, 0.03, 0.01)
    assert log[:, 3].min() > 1e-9  # every top-k decision has a clear margin
    m = fem.Mesh(1025)
    m.spatial_refine(torch.from_numpy(f_np).cuda(), 0.03, fem.params(topk_frac=0.01, precision=prec))
    assert _same_mesh(m, om)


@pytest.mark.parametrize("N,seed,density,frac", [(65, 0, 0.1, 0.0), (129, 1, 0.05, 0.01), (257, 0, 0.05, 0.0),
                                                  (513, 7, 0.03, 0.01), (1025, 1, 0.03, 0.01)])
def test_spatial_fast_keys_bit_exact(oracle_mod, fem, N, seed, density, frac):
    """Selection on FP32 keys with error bounds plus an exact band (forced on
    at every size): the same meshes as the oracle."""
    f_np = S.make_image(N, seed)
    om, log = oracle_mod.spatial(f_np, density, frac)
    m = fem.Mesh(N)
    m.spatial_refine(torch.from_numpy(f_np).cuda(), density, fem.params(topk_frac=frac, fast_keys=1))
    assert m.stats()["rounds"] == len(log)
    assert _same_mesh(m, om), "fast-key mesh differs from the oracle mesh"


@pytest.mark.parametrize("W,H,seed,texture,density", [(2049, 2049, 3, True, 0.02), (1025, 1025, 1, False, 0.03),
                                                       (1500, 1100, 5, True, 0.03), (700, 1300, 2, False, 0.05)])
def test_incremental_pass_equals_full_pass(fem, W, H, seed, texture, density):
    """After a call's first round the FP32 pass covers only the squares of
    the triangles a round can have changed and keeps the other intervals
    (fast_keys 1); a full pass every round (fast_keys 2) must give the same
    rounds, the same selection margins and the same mesh, bit for bit."""
    f_np = np.ascontiguousarray(S.make_image(max(W, H), seed, texture=texture)[:H, :W])
    f = torch.from_numpy(f_np).cuda()
    out = []
    for fast in (1, 2):
        m = fem.Mesh(W, H)
        m.spatial_refine(f, density, fem.params(topk_frac=0.01, fast_keys=fast))
        st = m.stats()
        out.append((m.export(), st["rounds"], st["min_margin"], st["cg_iters"]))
        m.close()
    (inc, r1, mm1, cg1), (full, r2, mm2, cg2) = out
    assert r1 == r2 and r1 > 100
    assert mm1 == mm2 and cg1 == cg2
    assert all(np.array_equal(a, b) for a, b in zip(inc, full))


@pytest.mark.parametrize("fast", [0, 1])
@pytest.mark.parametrize("N,value", [(65, 0.5), (257, 0.3)])
def test_spatial_constant_image_ties_by_id(oracle_mod, fem, N, value, fast):
    """A constant image: the solves reproduce the constant exactly, every key
    is 0, and the selection is decided by triangle ids alone (both key modes)."""
    f_np = np.full((N, N), value, dtype=np.float32)
    om, log = oracle_mod.spatial(f_np, 0.05, 0.01)
    m = fem.Mesh(N)
    f = torch.from_numpy(f_np).cuda()
    m.spatial_refine(f, 0.05, fem.params(topk_frac=0.01, fast_keys=fast))
    assert m.stats()["rounds"] == len(log)
    assert _same_mesh(m, om)
    g = m.g_from_f(f)
    _, uv = m.inpaint(g, want_uv=True)
    assert float(m.triangle_errors(uv, f).abs().max()) == 0.0


@pytest.mark.parametrize("fast", [0, 1])
@pytest.mark.parametrize("N,density,frac", [(3, 1.0, 0.0), (5, 0.8, 0.01), (9, 0.5, 1.0), (33, 0.3, 1.0)])
def test_spatial_smallest_images_and_all_eligible(oracle_mod, fem, N, density, frac, fast):
    """The smallest images (down to 3 x 3, where a full mesh is every pixel)
    and frac = 1 (every eligible triangle selected each round): bit-exact."""
    f_np = S.make_image(N, 11)
    om, log = oracle_mod.spatial(f_np, density, frac)
    m = fem.Mesh(N)
    m.spatial_refine(torch.from_numpy(f_np).cuda(), density, fem.params(topk_frac=frac, fast_keys=fast))
    assert m.stats()["rounds"] == len(log)
    assert _same_mesh(m, om)


@pytest.mark.parametrize("N,seed,texture", [(257, 5, False), (1025, 1, False), (2049, 3, True)])
def test_error_bounds_contain_exact_keys(oracle_mod, fem, N, seed, texture):
    """The FP32 intervals contain the float-float keys (and the oracle's FP64
    keys) for every triangle, and are narrow where the selection happens:
    below 1e-4 relative over the largest 5 % of the keys.  (Small keys get
    relatively wider intervals: the FP32 error of u, about 1e-7 |u|, enters
    the bound through sqrt(n key).)"""
    f_np = S.make_image(N, seed, texture=texture)
    f = torch.from_numpy(f_np).cuda()
    m = fem.Mesh(N)
    m.spatial_refine(f, 0.03, fem.params(topk_frac=0.01, fast_keys=0))
    g = m.g_from_f(f)
    _, uv = m.inpaint(g, want_uv=True)
    keys = m.triangle_errors(uv, f).cpu().numpy()
    lo, hi = m.triangle_error_bounds(uv, f)
    lo, hi = lo.cpu().numpy(), hi.cpu().numpy()
    assert (lo <= keys).all() and (keys <= hi).all()
    big = keys >= np.quantile(keys, 0.95)
    assert ((hi - lo)[big] <= 1e-4 * keys[big]).all()
    if N <= 257:
        xy, tri, mk = m.export()
        om = oracle_mod.Mesh(N, xy[:, 0].copy(), xy[:, 1].copy(), mk.copy(), tri[:, 0].copy(), tri[:, 1].copy(),
                             tri[:, 2].copy())
        _, kref, _ = oracle_mod.raster(om, uv.cpu().numpy(), f_np, owner=True)
        assert (lo <= kref).all() and (kref <= hi).all()


@pytest.mark.parametrize("N,seed", [(65, 2), (257, 3)])
def test_tonal_matches_oracle(oracle_mod, fem, N, seed):
    f_np = S.make_image(N, seed)
    om, _ = oracle_mod.spatial(f_np, 0.05, 0.01)
    g_ref, _ = oracle_mod.tonal(om, f_np, tol=1e-12)
    m = _gpu_mesh(fem, om)
    g = m.tonal_opt(torch.from_numpy(f_np).cuda(), p=fem.params(tonal_tol=1e-10)).double().cpu().numpy()
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-6, rel
    st = m.stats()
    assert st["tonal_relres"] <= 1e-10


def test_adjoint_matches_oracle_and_identity(oracle_mod, fem):
    f_np = S.make_image(129, 6)
    om, _ = oracle_mod.spatial(f_np, 0.05, 0.01)
    m = _gpu_mesh(fem, om)
    r_np = S.make_residual(129, 9)
    ref = oracle_mod.apply_BT(om, r_np.astype(np.float64))
    gbar = m.adjoint(torch.from_numpy(r_np).cuda()).double().cpu().numpy()
    assert np.linalg.norm(gbar - ref) <= 1e-6 * np.linalg.norm(ref)
    g_np = S.make_vector(int(om.mask.sum()), 10)
    u = m.inpaint(torch.from_numpy(g_np).cuda()).double().cpu().numpy()
    lhs = float(np.vdot(u, r_np.astype(np.float64)))
    rhs = float(np.vdot(g_np.astype(np.float64), gbar))
    assert abs(lhs - rhs) <= 1e-6 * (abs(lhs) + abs(rhs))


def test_autograd_gradient(oracle_mod, fem):
    from paper_2105_01586_gb300.autograd import FemInpaint, TonalLoss
    f_np = S.make_image(65, 4)
    om, _ = oracle_mod.spatial(f_np, 0.1, 0.01)
    m = _gpu_mesh(fem, om)
    f = torch.from_numpy(f_np).cuda()
    g0 = torch.from_numpy(oracle_mod.g_from_f(om, f_np).astype(np.float32)).cuda()
    g = g0.clone().requires_grad_(True)
    loss = TonalLoss.apply(g, f, m)
    loss.backward()
    ref = oracle_mod.apply_BT(om, oracle_mod.apply_B(om, g0.double().cpu().numpy()) - f_np)
    np.testing.assert_allclose(g.grad.double().cpu().numpy(), ref, rtol=0, atol=1e-5 * np.abs(ref).max())
    g2 = g0.clone().requires_grad_(True)
    u = FemInpaint.apply(g2, m)
    (u * torch.from_numpy(S.make_residual(65, 1)).cuda()).sum().backward()
    ref2 = oracle_mod.apply_BT(om, S.make_residual(65, 1).astype(np.float64))
    np.testing.assert_allclose(g2.grad.double().cpu().numpy(), ref2, rtol=0, atol=1e-5 * np.abs(ref2).max())


def test_errors_are_reported(fem):
    m = fem.Mesh(33)
    with pytest.raises(fem.FemError) as e:
        m.import_(np.array([[0, 0], [32, 0], [0, 32]]), np.array([[0, 2, 1]]), np.ones(3))
    assert e.value.status == fem.FEM_E_INVALID
    for w, h in ((1, 5), (5, 1), (40000, 5)):  # image sides must be 2..32769
        with pytest.raises(fem.FemError) as e:
            fem.Mesh(w, h)
        assert e.value.status == fem.FEM_E_SHAPE


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("N,mask_frac", [(129, 0.3), (257, 0.2)])
def test_inpaint_large_systems(oracle_mod, fem, N, mask_frac, prec):
    """Fully refined meshes (every pixel a vertex) with a random mask: about
    11.6k unknowns (one-block solver, vectors in global memory) and 53k
    unknowns (grid solver), both against the oracle."""
    import pins
    om = pins.fully_refined_mesh(oracle_mod, N)
    rng = np.random.default_rng(N)
    mk = (rng.uniform(size=om.V) < mask_frac).astype(np.uint8)
    mk[:4] = 1
    om = om.with_mask(mk)
    g_np = rng.uniform(size=int(mk.sum()))
    v_ref, _, _ = oracle_mod.solve(om, g_np, tol=1e-14)
    m = _gpu_mesh(fem, om)
    _, uv = m.inpaint(torch.from_numpy(g_np.astype(np.float32)).cuda(), fem.params(precision=prec), want_uv=True)
    v_ref32, _, _ = oracle_mod.solve(om, g_np.astype(np.float32).astype(np.float64), tol=1e-14)
    uv = uv.cpu().numpy()
    assert np.linalg.norm(uv - v_ref32) <= 1e-9 * np.linalg.norm(v_ref32)
    assert m.stats()["relres"] <= 1e-12


def test_bounded_wait_reports_timeout(fem):
    """A grid barrier whose second block never arrives gives up after its
    limit and reports FEM_E_TIMEOUT; the context stays usable."""
    assert fem.fem_selftest_wait_timeout() == fem.FEM_E_TIMEOUT
    m = fem.Mesh(33)
    u = m.inpaint(torch.full((4,), 0.5, device="cuda"))
    assert torch.allclose(u, torch.full_like(u, 0.5))


@pytest.mark.parametrize("N,density,frac", [(129, 0.1, 0.01), (513, 0.03, 0.01)])
def test_curve_order_is_continuous(fem, N, density, frac):
    """The triangles' visiting order after refinement is the bisection tree's
    space-filling curve: a permutation in which each triangle is left at the
    vertex where the next one is entered (axis-aligned legs: entered at a,
    left at b; diagonal legs: entered at b, left at a)."""
    f = torch.from_numpy(S.make_image(N, 3)).cuda()
    m = fem.Mesh(N)
    m.spatial_refine(f, density, fem.params(topk_frac=frac))
    order, is_curve = fem.fem_mesh_curve_order(m.h)
    xy, tri, _ = m.export()
    assert is_curve and np.array_equal(np.sort(order), np.arange(m.T))
    a, b, c = tri[order, 0], tri[order, 1], tri[order, 2]
    diag = (xy[c, 0] != xy[a, 0]) & (xy[c, 1] != xy[a, 1])
    entry = np.where(diag, b, a)
    exit_ = np.where(diag, a, b)
    assert (exit_[:-1] == entry[1:]).all()
    assert entry[0] == 0 and exit_[-1] == 0  # the curve starts and ends at the corner (0, 0)
