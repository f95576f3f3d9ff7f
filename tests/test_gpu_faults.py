"""Host-side failure handling on the GPU path, with no device fault: device
allocations that fail (injected by fem_debug_alloc_fault, which makes the
n-th allocation fail before any CUDA call), a caller-provided memory pool,
and the cancellation of served requests.  Every failure here is made on the
host; the kernels only ever see valid memory."""
import ctypes
import ctypes.util
import time

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


def _job(fem, f, density=0.05):
    """A small whole job (spatial + tonal) through the public API; returns
    the mesh arrays and g, or raises FemError."""
    m = fem.Mesh(f.shape[0])
    try:
        p = fem.params(topk_frac=0.01)
        m.spatial_refine(f, density, p)
        g = m.g_from_f(f)
        fem.fem_tonal_opt(m.h, f, g, p)
        xy, tri, mk = m.export()
        return xy, tri, mk, g.cpu().numpy()
    finally:
        m.close()


def test_every_allocation_failure_reports_oom_and_leaves_the_library_usable(fem):
    f = torch.from_numpy(S.make_image(129, 4)).cuda()
    n0 = fem.fem_debug_alloc_fault(-1)
    ref = _job(fem, f)
    n_allocs = fem.fem_debug_alloc_fault(-1) - n0
    assert n_allocs > 10
    for k in range(n_allocs):
        fem.fem_debug_alloc_fault(k)
        try:
            with pytest.raises(fem.FemError) as ei:
                _job(fem, f)
            assert ei.value.status == fem.FEM_E_OOM, (k, str(ei.value))
            assert "injected" in str(ei.value)
        finally:
            fem.fem_debug_alloc_fault(-1)
        torch.cuda.synchronize()
    # after all of that, the same job gives the same result
    out = _job(fem, f)
    for a, b in zip(ref, out):
        assert np.array_equal(a, b)


def _cudart():
    for name in ("libcudart.so.13", ctypes.util.find_library("cudart"), "/usr/local/cuda/lib64/libcudart.so"):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    pytest.skip("no shared CUDA runtime to create a memory pool with")


def test_caller_memory_pool_takes_the_allocations(fem):
    rt = _cudart()
    dev = torch.cuda.current_device()
    props = (ctypes.c_ubyte * 256)()  # cudaMemPoolProps, zeroed; the fields set below lead the struct
    ctypes.c_int.from_buffer(props, 0).value = 1    # allocType = cudaMemAllocationTypePinned
    ctypes.c_int.from_buffer(props, 8).value = 1    # location.type = cudaMemLocationTypeDevice
    ctypes.c_int.from_buffer(props, 12).value = dev  # location.id
    pool = ctypes.c_void_p()
    assert rt.cudaMemPoolCreate(ctypes.byref(pool), ctypes.byref(props)) == 0
    used = ctypes.c_uint64()
    USED_HIGH = 8  # cudaMemPoolAttrUsedMemHigh
    try:
        f = torch.from_numpy(S.make_image(129, 4)).cuda()
        ref = _job(fem, f)
        assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(used)) == 0
        assert used.value == 0  # nothing came from it yet
        fem.fem_set_mem_pool(pool.value)
        try:
            out = _job(fem, f)
        finally:
            fem.fem_set_mem_pool(None)
        torch.cuda.synchronize()
        assert rt.cudaMemPoolGetAttribute(pool, USED_HIGH, ctypes.byref(used)) == 0
        assert used.value > 0
        for a, b in zip(ref, out):
            assert np.array_equal(a, b)
    finally:
        torch.cuda.synchronize()
        rt.cudaMemPoolDestroy(pool)


def test_cancel_queued_and_running_requests(fem):
    """With one slot: a queued request is removed at once; the running
    8193^2 job (about a third of a second of work) is cancelled as soon as
    it is seen running and stops at its next round; the request behind it
    still completes, and cancelling a finished request changes nothing."""
    from paper_2105_01586_gb300.serving import Server
    big = S.make_image(8193, 3, texture=True)
    small = S.make_image(257, 2)
    with Server(slots=1) as sv:
        a = sv.submit(big, 0.02)
        b = sv.submit(small, 0.05)
        c = sv.submit(small, 0.05)
        sv.cancel(b)  # queued behind a: removed at once
        assert sv.state(b) == "finished"
        assert sv.status(b) == fem.FEM_E_CANCELLED
        t0 = time.time()
        while sv.state(a) == "queued" and time.time() - t0 < 60.0:
            time.sleep(0.0005)
        assert sv.state(a) == "running"
        sv.cancel(a)
        assert sv.wait(a, 30.0)
        assert sv.status(a) == fem.FEM_E_CANCELLED, sv.status(a)
        assert sv.wait(c, 60.0)
        r = sv.result(c)
        assert r["status"] == fem.FEM_OK and r["g"].size > 0
        sv.cancel(c)  # finished: nothing happens
        assert sv.status(c) == fem.FEM_OK
        for rid in (a, b, c):
            sv.release(rid)
