"""Images of any size (NEXT-4; reading R9 of the oracle): a W x H image in
the smallest (2^L + 1)^2 domain, only image pixels as data.  GPU against
the oracle, through the C ABI: meshes bit for bit (exact and fast keys),
per-triangle errors, interpolant and owners, inpainting, the adjoint and
the tonal optimisation.  Sizes include the paper's 2^k images (Table 2:
1024 x 1024) and shapes much wider than tall."""
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


def _image(W, H, seed, texture=False):
    return np.ascontiguousarray(S.make_image(max(W, H), seed, texture=texture)[:H, :W])


def _gpu_mesh(fem, om):
    m = fem.Mesh(om.W, om.H)
    assert m.n == om.N
    m.import_(om.xy, om.tri, om.mask)
    return m


def _same_mesh(m, om):
    xy, tri, mk = m.export()
    return np.array_equal(xy, om.xy) and np.array_equal(tri, om.tri) and np.array_equal(mk, om.mask)


def key_err_tol(keys_ref, own, vmax):
    n_t = np.bincount(own.ravel(), minlength=len(keys_ref)).astype(np.float64)
    du = 2.0 ** -47 * max(1.0, vmax)
    return 2.0 * du * np.sqrt(n_t * keys_ref) + 1e-12 * keys_ref + 1e-300


@pytest.mark.parametrize("W,H,seed,density,frac,fast", [
    (200, 130, 1, 0.05, 0.01, 0), (130, 200, 2, 0.05, 0.01, 0), (100, 61, 3, 0.1, 0.02, 0), (61, 100, 3, 0.1, 0.02, 1),
    (513, 140, 4, 0.04, 0.01, 0), (200, 130, 1, 0.05, 0.01, 1), (1024, 1024, 5, 0.03, 0.01, 0),
    (1024, 1024, 5, 0.03, 0.01, 1)])
def test_spatial_refine_bit_exact(oracle_mod, fem, W, H, seed, density, frac, fast):
    f_np = _image(W, H, seed)
    om, log = oracle_mod.spatial(f_np, density, frac)
    assert log[:, 3].min() > 1e-9  # every selection decided by a clear margin
    m = fem.Mesh(W, H)
    f = torch.from_numpy(f_np).cuda()
    m.spatial_refine(f, density, fem.params(topk_frac=frac, fast_keys=fast))
    assert m.stats()["rounds"] == len(log)
    assert _same_mesh(m, om), "GPU mesh differs from the oracle mesh"
    g = m.g_from_f(f).cpu().numpy()
    np.testing.assert_array_equal(g, oracle_mod.g_from_f(om, f_np).astype(np.float32))


@pytest.mark.parametrize("W,H,seed", [(200, 130, 1), (33, 65, 2), (513, 140, 4)])
def test_errors_raster_and_bounds(oracle_mod, fem, W, H, seed):
    f_np = _image(W, H, seed)
    om, _ = oracle_mod.spatial(f_np, 0.05, 0.02)
    m = _gpu_mesh(fem, om)
    v = np.random.default_rng(seed).uniform(-0.5, 1.5, size=om.V)
    u_ref, keys_ref, own_ref = oracle_mod.raster(om, v, f_np, owner=True)
    uv = torch.from_numpy(v).cuda()
    f = torch.from_numpy(f_np).cuda()
    err = m.triangle_errors(uv, f).cpu().numpy()
    assert (np.abs(err - keys_ref) <= key_err_tol(keys_ref, own_ref, np.abs(v).max())).all()
    lo, hi = m.triangle_error_bounds(uv, f)
    lo, hi = lo.cpu().numpy(), hi.cpu().numpy()
    assert np.all(lo <= keys_ref) and np.all(keys_ref <= hi)
    u, own = m.rasterize(uv, want_owner=True)
    assert tuple(u.shape) == (H, W)
    np.testing.assert_array_equal(own.cpu().numpy(), own_ref)
    np.testing.assert_allclose(u.cpu().numpy(), u_ref, rtol=0, atol=2e-7 * max(1.0, np.abs(v).max()))


@pytest.mark.parametrize("prec", [0, 1])
def test_inpaint_and_adjoint(oracle_mod, fem, prec):
    W, H = 300, 170
    f_np = _image(W, H, 6)
    om, _ = oracle_mod.spatial(f_np, 0.04, 0.01)
    m = _gpu_mesh(fem, om)
    g_np = oracle_mod.g_from_f(om, f_np)
    v_ref, _, _ = oracle_mod.solve(om, g_np, tol=1e-14)
    u, uv = m.inpaint(torch.from_numpy(g_np.astype(np.float32)).cuda(), fem.params(precision=prec), want_uv=True)
    assert np.linalg.norm(uv.cpu().numpy() - v_ref) <= 1e-9 * np.linalg.norm(v_ref)
    u_ref, _, _ = oracle_mod.raster(om, v_ref)
    np.testing.assert_allclose(u.cpu().numpy(), u_ref, rtol=0, atol=2e-7)
    r_np = np.random.default_rng(1).standard_normal((H, W)).astype(np.float32)
    gbar = m.adjoint(torch.from_numpy(r_np).cuda(), fem.params(precision=prec, inner_tol=1e-13)).cpu().numpy()
    ref = oracle_mod.apply_BT(om, r_np.astype(np.float64))
    np.testing.assert_allclose(gbar, ref, rtol=0, atol=1e-5 * np.abs(ref).max())


def test_tonal_matches_converged_oracle(oracle_mod, fem):
    """The padding's mask vertices reach few image pixels or none: their
    columns of B are small or zero, so g there depends on how far CG is
    driven, while the reconstruction does not.  Both sides run CG from
    g0 = f at the mask; compared are the well-conditioned quantities: the
    objective, the reconstruction B g on the image, and g at the mask
    vertices inside the image."""
    W, H = 200, 130
    f_np = _image(W, H, 7)
    om, _ = oracle_mod.spatial(f_np, 0.05, 0.01)
    m = _gpu_mesh(fem, om)
    f = torch.from_numpy(f_np).cuda()
    p = fem.params(tonal_tol=1e-10, inner_tol=1e-13, precision=fem.FEM_PREC_FP64)
    g = m.g_from_f(f)
    fem.fem_tonal_opt(m.h, f, g, p)
    g_ref, st = oracle_mod.tonal(om, f_np, tol=1e-12)
    g_gpu = g.double().cpu().numpy()
    u_gpu, u_ref = oracle_mod.apply_B(om, g_gpu), oracle_mod.apply_B(om, g_ref)
    assert np.linalg.norm(u_gpu - u_ref) <= 1e-6 * np.linalg.norm(u_ref)
    sse = float(np.sum((u_gpu - f_np) ** 2))
    assert abs(sse - st["sse"]) <= 1e-7 * st["sse"], (sse, st["sse"])
    k = np.flatnonzero(om.mask)
    inside = (om.vx[k] < W) & (om.vy[k] < H)
    rel = np.linalg.norm(g_gpu[inside] - g_ref[inside]) / np.linalg.norm(g_ref[inside])
    assert rel <= 1e-6, rel
