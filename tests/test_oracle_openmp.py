"""The OpenMP build of the oracle (the multi-core CPU baseline) computes the
same bits as the single-thread build: the per-triangle raster loop and the
rows of A_UU x are shared among threads, and every output element is still
computed by one thread in the same order."""
import numpy as np
import pytest

import seeded_inputs as S


@pytest.fixture()
def oracle_omp(oracle_mod):
    try:
        oracle_mod.build(openmp=True)
    except Exception as e:  # noqa: BLE001
        pytest.skip(f"no OpenMP toolchain: {e}")
    yield oracle_mod
    oracle_mod.use_openmp(False)


def test_openmp_build_is_bit_identical(oracle_omp):
    o = oracle_omp
    f = S.make_image(129, 7)
    assert o.use_openmp(False) == 1
    m1, log1 = o.spatial(f, 0.06, 0.01)
    v1, _, _ = o.solve(m1, o.g_from_f(m1, f))
    u1, k1, _ = o.raster(m1, v1, f)
    g1, st1 = o.tonal(m1, f, tol=0.0, maxit=5, allow_not_converged=True)
    threads = o.use_openmp(True)
    assert threads >= 1
    m2, log2 = o.spatial(f, 0.06, 0.01)
    assert np.array_equal(m1.xy, m2.xy) and np.array_equal(m1.tri, m2.tri) and np.array_equal(m1.mask, m2.mask)
    assert np.array_equal(log1, log2)
    v2, _, _ = o.solve(m2, o.g_from_f(m2, f))
    u2, k2, _ = o.raster(m2, v2, f)
    assert np.array_equal(v1, v2) and np.array_equal(u1, u2) and np.array_equal(k1, k2)
    g2, st2 = o.tonal(m2, f, tol=0.0, maxit=5, allow_not_converged=True)
    assert np.array_equal(g1, g2) and st1["sse"] == st2["sse"]


def test_openmp_raster_keeps_ownership_check(oracle_omp):
    """With an owner map the raster runs on one thread and still proves every
    pixel is owned exactly once."""
    o = oracle_omp
    o.use_openmp(True)
    f = S.make_image(65, 2)
    m, _ = o.spatial(f, 0.1, 0.02)
    v, _, _ = o.solve(m, o.g_from_f(m, f))
    _, _, owner = o.raster(m, v, f, owner=True)
    assert owner.min() >= 0 and np.bincount(owner.ravel(), minlength=m.T).sum() == 65 * 65
