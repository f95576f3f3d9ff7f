"""The C-ABI library loads and exports every symbol include/feminpaint.h
declares; host-side argument checks work without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fem():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_01586_gb300 as fem
    return fem


def _declared():
    src = open(os.path.join(ROOT, "include", "feminpaint.h")).read()
    return sorted(set(re.findall(r"FEM_API\s+[\w\s\*]*?\b(fem_\w+)\s*\(", src)))


def test_header_declares_entry_points():
    names = _declared()
    for n in ("fem_mesh_create", "fem_inpaint", "fem_triangle_errors", "fem_spatial_refine", "fem_tonal_opt",
              "fem_adjoint"):
        assert n in names


def test_library_exports_every_declared_symbol(fem):
    out = subprocess.run(["nm", "-D", "--defined-only", fem.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (fem_\w+)$", out, flags=re.M))
    declared = set(_declared())
    assert declared <= exported, declared - exported
    for n in declared:
        assert hasattr(fem._lib, n)
    assert set(fem.EXPORTED) == declared


def test_defaults_and_host_checks(fem):
    p = fem.params()
    assert p.tol == 1e-12 and p.precision == fem.FEM_PREC_FP32_IR and p.topk_frac == 0.01
    # null handle and null arguments are rejected on the host, before any CUDA call
    assert fem._lib.fem_mesh_info(None, None, None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_inpaint(None, None, None, None, None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_spatial_refine(None, None, ctypes.c_double(0.1), None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_spatial_refine_channels(None, None, 3, ctypes.c_double(0.1), None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_mesh_size(None, None, None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_tonal_opt(None, None, None, None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_adjoint(None, None, None, None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_tonal_loss(None, None, None, None, None, None, None) == fem.FEM_E_INVALID
    assert b"null" in fem._lib.fem_last_error()
    h = ctypes.c_void_p()
    for bad in ((1, 5), (5, 1), (0, 0), (-3, 9), (40000, 3), (3, 40000)):  # sides must be 2..32769
        assert fem._lib.fem_mesh_create(bad[0], bad[1], None, ctypes.byref(h)) == fem.FEM_E_SHAPE
    assert fem.fem_launch_count() == 0


def test_product_path_does_not_import_oracle():
    """The binding, build and CUDA sources never reference the oracle."""
    pkg = os.path.join(ROOT, "paper_2105_01586_gb300")
    for dp, _, fns in os.walk(pkg):
        for fn in fns:
            if fn.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dp, fn)).read()
                assert "import oracle" not in txt and "oracle." not in txt, fn


def test_server_entry_points_reject_bad_handles_on_the_host(fem):
    """The serving calls marshal their arguments and reject a null server
    before any CUDA work (runs without a GPU)."""
    import numpy as np
    sizes = np.zeros(4, np.int32)
    f = np.zeros((5, 5), np.float32)
    rid = ctypes.c_longlong()
    done = ctypes.c_int()
    assert fem._lib.fem_server_submit(None, 5, f.ctypes.data, 0.5, None, ctypes.byref(rid)) == fem.FEM_E_INVALID
    assert fem._lib.fem_server_wait(None, 1, 0.0, ctypes.byref(done)) == fem.FEM_E_INVALID
    assert fem._lib.fem_server_result(None, 1, sizes.ctypes.data, None, None, None, None, None) == fem.FEM_E_INVALID
    assert fem._lib.fem_server_release(None, 1) == fem.FEM_E_INVALID
    assert fem._lib.fem_server_cancel(None, 1) == fem.FEM_E_INVALID
    assert fem._lib.fem_server_state(None, 1, ctypes.byref(done)) == fem.FEM_E_INVALID
    assert fem._lib.fem_server_destroy(None) == fem.FEM_OK
    out = ctypes.c_void_p()
    assert fem._lib.fem_server_create(0, 0, ctypes.byref(out)) == fem.FEM_E_INVALID


def test_noalloc_entry_point_checks_sizes_on_the_host(fem):
    """The allocation-free error pass rejects sizes beyond its fixed scratch,
    null pointers and misaligned arrays before any CUDA call (no GPU needed)."""
    L = fem._lib
    ok_ptr = 1 << 12  # aligned, never dereferenced: the checks fail first
    args = lambda w, V, T, xy=ok_ptr, tri=ok_ptr: (w, V, xy, T, tri, ok_ptr, ok_ptr, ok_ptr, None)
    assert L.fem_triangle_errors_noalloc(*args(4097, 4, 2)) == fem.FEM_E_SHAPE
    assert L.fem_triangle_errors_noalloc(*args(100, 4, 2)) == fem.FEM_E_SHAPE      # not 2^L + 1
    assert L.fem_triangle_errors_noalloc(*args(129, 4, 65537)) == fem.FEM_E_INVALID
    assert b"65536" in L.fem_last_error()
    assert L.fem_triangle_errors_noalloc(*args(129, 4, 0)) == fem.FEM_E_INVALID
    assert L.fem_triangle_errors_noalloc(*args(129, 4, 2, xy=None)) == fem.FEM_E_INVALID
    assert b"null" in L.fem_last_error()
    assert L.fem_triangle_errors_noalloc(*args(129, 4, 2, tri=ok_ptr + 4)) == fem.FEM_E_INVALID
    assert b"aligned" in L.fem_last_error()


def test_allocation_fault_hook_and_pool_setting_are_host_only(fem):
    """fem_debug_alloc_fault counts and arms on the host; fem_set_mem_pool(NULL)
    selects the device's current pool.  Neither touches a device."""
    n0 = fem.fem_debug_alloc_fault(-1)
    assert n0 >= 0
    assert fem.fem_debug_alloc_fault(5) == n0   # armed five attempts ahead; nothing allocated here
    assert fem.fem_debug_alloc_fault(-1) == n0  # disarmed
    fem.fem_set_mem_pool(None)
