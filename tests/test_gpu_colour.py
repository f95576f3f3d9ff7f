"""Colour spatial optimisation (NEXT-2; reading R10 of the oracle) on the
GPU through the C ABI against the oracle: meshes bit for bit, with one,
two equal, and three different channels, square and not."""
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


def _colour(W, H, seeds):
    n = max(W, H)
    return np.ascontiguousarray(np.stack([S.make_image(n, s)[:H, :W] for s in seeds]).astype(np.float32))


def _same_mesh(m, om):
    xy, tri, mk = m.export()
    return np.array_equal(xy, om.xy) and np.array_equal(tri, om.tri) and np.array_equal(mk, om.mask)


@pytest.mark.parametrize("W,H,seeds,density,frac,prec", [
    (257, 257, (1, 2, 3), 0.04, 0.01, 0), (257, 257, (1, 2, 3), 0.04, 0.01, 1), (300, 170, (4, 5, 6), 0.04, 0.01, 0),
    (513, 513, (7, 8), 0.03, 0.01, 0), (129, 129, (9,), 0.1, 0.02, 0)])
def test_colour_spatial_matches_oracle(oracle_mod, fem, W, H, seeds, density, frac, prec):
    f_np = _colour(W, H, seeds)
    om, log = oracle_mod.spatial(f_np, density, frac)
    assert log[:, 3].min() > 1e-9
    m = fem.Mesh(W, H)
    f = torch.from_numpy(f_np).cuda()
    m.spatial_refine(f, density, fem.params(topk_frac=frac, precision=prec))
    assert m.stats()["rounds"] == len(log)
    assert _same_mesh(m, om)
    for c in range(len(seeds)):
        g = m.g_from_f(f[c].contiguous()).cpu().numpy()
        np.testing.assert_array_equal(g, oracle_mod.g_from_f(om, f_np[c]).astype(np.float32))


def test_one_channel_and_equal_channels_match_grey(fem):
    f_np = S.make_image(257, 11)
    f = torch.from_numpy(f_np).cuda()
    ref = fem.Mesh(257)
    ref.spatial_refine(f, 0.04, fem.params(topk_frac=0.01, fast_keys=0))
    for stack in (f[None], torch.stack([f, f])):
        m = fem.Mesh(257)
        m.spatial_refine(stack.contiguous(), 0.04, fem.params(topk_frac=0.01))
        for a, b in zip(m.export(), ref.export()):
            assert np.array_equal(a, b)


def test_channel_count_is_checked(fem):
    m = fem.Mesh(33)
    f = torch.zeros((5, 33, 33), device="cuda")
    with pytest.raises(fem.FemError) as e:
        m.spatial_refine(f, 0.1)
    assert e.value.status == fem.FEM_E_INVALID
