"""Serving (continuous batching): every request's result is the same alone
and in the mix, and admission by device memory works."""
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


def _jobs():
    rng = np.random.default_rng(5)
    out = []
    for i in range(10):
        n = int(rng.choice([65, 129, 257]))
        out.append((S.make_image(n, 100 + i), float(rng.uniform(0.05, 0.12))))
    return out


def test_results_same_alone_and_in_the_mix(fem):
    from paper_2105_01586_gb300.serving import Server
    jobs = _jobs()
    p = fem.params(tonal_tol=1e-9)
    alone = []
    with Server(slots=1) as sv:
        for f, d in jobs:
            rid = sv.submit(f, d, p)
            assert sv.wait(rid)
            alone.append(sv.result(rid))
    with Server(slots=4) as sv:
        ids = [sv.submit(f, d, p) for f, d in jobs]
        mixed = []
        for rid in ids:
            assert sv.wait(rid, 600.0)
            mixed.append(sv.result(rid))
    for a, b in zip(alone, mixed):
        assert a["status"] == 0 and b["status"] == 0
        for k in ("xy", "tri", "mask"):
            np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_allclose(b["g"], a["g"], rtol=0, atol=1e-6 * max(1.0, np.abs(a["g"]).max()))
    # the mix ran concurrently: some request started before an earlier one ended
    starts = np.array([r["t_start"] for r in mixed])
    ends = np.array([r["t_end"] for r in mixed])
    assert any(starts[j] < ends[i] for i in range(len(mixed)) for j in range(len(mixed)) if i != j)


def test_admission_by_memory_serialises_when_the_budget_is_small(fem):
    from paper_2105_01586_gb300.serving import Server
    jobs = _jobs()[:5]
    with Server(slots=4, mem_budget_bytes=1) as sv:   # every request exceeds the budget: one at a time
        ids = [sv.submit(f, d) for f, d in jobs]
        res = [sv.result(rid) if sv.wait(rid, 600.0) else None for rid in ids]
    iv = sorted((r["t_start"], r["t_end"]) for r in res)
    for (s0, e0), (s1, e1) in zip(iv, iv[1:]):
        assert s1 >= e0 - 1e-6


def test_measured_peak_is_within_the_static_estimate(fem):
    """Each request's device allocations are counted on its slot's stream:
    the measured peak holds at least the request's image copy and stays
    below the static upper estimate that admission is scaled from."""
    from paper_2105_01586_gb300.serving import Server
    jobs = _jobs()[:6]
    with Server(slots=2) as sv:
        ids = [sv.submit(f, d) for f, d in jobs]
        res = [sv.result(rid) if sv.wait(rid, 600.0) else None for rid in ids]
    for (f, _), r in zip(jobs, res):
        assert r is not None and r["status"] == 0
        assert 4 * f.size <= r["mem_measured"] <= r["mem_estimate"]


def test_serving_matches_the_direct_api(fem):
    """A served request returns the same mesh and g as calling the library
    directly on one stream."""
    from paper_2105_01586_gb300.serving import Server
    f_np, d = _jobs()[0]
    with Server(slots=2) as sv:
        rid = sv.submit(f_np, d)
        assert sv.wait(rid, 600.0)
        r = sv.result(rid)
    m = fem.Mesh(f_np.shape[0])
    f = torch.from_numpy(f_np).cuda()
    m.spatial_refine(f, d)
    g = m.tonal_opt(f)
    xy, tri, mk = m.export()
    np.testing.assert_array_equal(xy, r["xy"])
    np.testing.assert_array_equal(tri, r["tri"])
    np.testing.assert_array_equal(mk, r["mask"])
    np.testing.assert_allclose(r["g"], g.cpu().numpy(), rtol=0, atol=1e-6)
