"""The allocation-free error entry point (fem_triangle_errors_noalloc).

It serves callers that cannot allocate device memory (programs whose own
caching allocator has reserved all device memory, loops that must not
allocate after start-up).  It must give the same per-triangle errors as
fem_triangle_errors, on two calls in a row (the shared scratch keeps the
previous call's contents), alone in a fresh process or after other tests.
This file is named so that pytest collects it last.
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


def _case(oracle_mod, fem, N, seed, density):
    f_np = S.make_image(N, seed)
    om, _ = oracle_mod.spatial(f_np, density, 0.01)
    m = fem.Mesh(N)
    m.import_(om.xy, om.tri, om.mask)
    xy = torch.from_numpy(om.xy.astype(np.int32)).cuda().contiguous()
    tri4 = torch.zeros((om.T, 4), dtype=torch.int32)
    tri4[:, :3] = torch.from_numpy(om.tri.astype(np.int32))
    tri4 = tri4.cuda().contiguous()
    uv = torch.from_numpy(np.random.default_rng(seed).uniform(-0.2, 1.2, om.V)).cuda()
    f = torch.from_numpy(f_np).cuda()
    return m, xy, tri4, uv, f


def test_noalloc_matches_allocating_entry_point_twice(oracle_mod, fem):
    # two different meshes one after the other: the second call must not see the first one's scratch
    for N, seed, density in ((257, 1, 0.03), (129, 2, 0.08)):
        m, xy, tri4, uv, f = _case(oracle_mod, fem, N, seed, density)
        ref = m.triangle_errors(uv, f)
        for _ in range(2):
            err = torch.full((tri4.shape[0],), -1.0, dtype=torch.float64, device="cuda")
            fem.fem_triangle_errors_noalloc(N, xy, tri4, uv, f, err)
            torch.cuda.synchronize()
            np.testing.assert_allclose(err.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-300)


def test_noalloc_rejects_sizes_beyond_its_scratch(fem):
    xy = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    big = torch.zeros((65537, 4), dtype=torch.int32, device="cuda")
    uv = torch.zeros(4, dtype=torch.float64, device="cuda")
    err = torch.zeros(65537, dtype=torch.float64, device="cuda")
    f = torch.zeros((129, 129), dtype=torch.float32, device="cuda")
    with pytest.raises(fem.FemError) as e:
        fem.fem_triangle_errors_noalloc(129, xy, big, uv, f, err)
    assert e.value.status == fem.FEM_E_INVALID and "65536" in str(e.value)
    f2 = torch.zeros((4097, 4097), dtype=torch.float32, device="cuda")
    with pytest.raises(fem.FemError) as e:
        fem.fem_triangle_errors_noalloc(4097, xy, big[:2], uv, f2, err[:2])
    assert e.value.status == fem.FEM_E_SHAPE


def test_noalloc_allocates_no_device_memory(oracle_mod, fem):
    # the defining property: after the first calls (which load the library's
    # kernels and look up the fixed array's address), a call leaves the
    # device's free memory exactly where it was
    m, xy, tri4, uv, f = _case(oracle_mod, fem, 257, 1, 0.03)
    err = torch.empty((tri4.shape[0],), dtype=torch.float64, device="cuda")
    for _ in range(2):
        fem.fem_triangle_errors_noalloc(257, xy, tri4, uv, f, err)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        fem.fem_triangle_errors_noalloc(257, xy, tri4, uv, f, err)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_overflow_is_reported_and_the_next_call_is_correct(oracle_mod, fem):
    # 200 copies of the two image-sized triangles of a 2049 x 2049 image: every
    # index is in range, but the triangles need about 410k rasterisation items,
    # more than the fixed scratch holds (3 * 65536 + 2049^2 / 128 + 1024)
    n = 2049
    xy = torch.tensor([[0, 0], [n - 1, 0], [0, n - 1], [n - 1, n - 1]], dtype=torch.int32, device="cuda")
    tri4 = torch.tensor([[0, 3, 2, 0], [3, 0, 1, 0]] * 100, dtype=torch.int32, device="cuda")
    uv = torch.zeros(4, dtype=torch.float64, device="cuda")
    f = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    err = torch.zeros(tri4.shape[0], dtype=torch.float64, device="cuda")
    with pytest.raises(fem.FemError) as e:
        fem.fem_triangle_errors_noalloc(n, xy, tri4, uv, f, err)
    assert e.value.status == fem.FEM_E_INVALID and "items" in str(e.value)
    # the context is still usable and a valid call after it is exact
    m, xy2, tri2, uv2, f2 = _case(oracle_mod, fem, 257, 1, 0.03)
    ref = m.triangle_errors(uv2, f2)
    out = torch.full((tri2.shape[0],), -1.0, dtype=torch.float64, device="cuda")
    fem.fem_triangle_errors_noalloc(257, xy2, tri2, uv2, f2, out)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), ref.cpu().numpy(), rtol=1e-12, atol=1e-300)
