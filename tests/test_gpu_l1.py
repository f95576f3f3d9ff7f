"""The L1 data term of the tonal optimisation (NEXT-2b; reading R11: IRLS
with weights 1 / max(|B g - f|, eps)) on the GPU through the C ABI, against
the oracle's IRLS after the same number of steps, each step's weighted
least-squares problem solved to a tight tolerance on both sides."""
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


def _case(oracle_mod, N, seed, density):
    f = S.make_image(N, seed)
    rng = np.random.default_rng(seed)
    idx = rng.choice(N * N, size=N, replace=False)
    f.ravel()[idx] = np.clip(f.ravel()[idx] + rng.choice([-0.6, 0.6], size=N), 0, 1)  # outliers
    om, _ = oracle_mod.spatial(f, density, 0.02)
    return f, om


@pytest.mark.parametrize("N,seed,density,steps", [(65, 3, 0.1, 3), (257, 4, 0.04, 4)])
def test_l1_matches_oracle_irls(oracle_mod, fem, N, seed, density, steps):
    f_np, om = _case(oracle_mod, N, seed, density)
    m = fem.Mesh(N)
    m.import_(om.xy, om.tri, om.mask)
    f = torch.from_numpy(f_np).cuda()
    g = m.g_from_f(f)
    p = fem.params(tonal_tol=1e-11, inner_tol=1e-13, precision=fem.FEM_PREC_FP64)
    p.tonal_maxit = 20000
    fem.fem_tonal_opt_l1(m.h, f, g, steps, 1e-3, p)
    g_ref, st = oracle_mod.tonal_l1(om, f_np, irls=steps, eps=1e-3, tol=1e-12)
    g_gpu = g.double().cpu().numpy()
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel <= 1e-5, rel
    l1 = float(np.abs(oracle_mod.apply_B(om, g_gpu) - f_np).sum())
    assert abs(l1 - st["l1"]) <= 1e-6 * st["l1"], (l1, st["l1"])


def test_l1_after_l2_keeps_the_l2_path_intact(oracle_mod, fem):
    """The weighted pixel-mass matrix of an IRLS step must not leak into a
    later unweighted tonal optimisation on the same mesh."""
    f_np, om = _case(oracle_mod, 65, 5, 0.1)
    m = fem.Mesh(65)
    m.import_(om.xy, om.tri, om.mask)
    f = torch.from_numpy(f_np).cuda()
    p = fem.params(tonal_tol=1e-10, inner_tol=1e-13, precision=fem.FEM_PREC_FP64)
    g1 = m.g_from_f(f)
    fem.fem_tonal_opt(m.h, f, g1, p)
    g2 = m.g_from_f(f)
    fem.fem_tonal_opt_l1(m.h, f, g2, 2, 1e-3, p)
    g3 = m.g_from_f(f)
    fem.fem_tonal_opt(m.h, f, g3, p)
    np.testing.assert_array_equal(g1.cpu().numpy(), g3.cpu().numpy())
