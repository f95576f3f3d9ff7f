"""GB300 (sm_103a) FEM harmonic inpainting with spatial and tonal data
optimisation, after Chizhov & Weickert, "Efficient Data Optimisation for
Harmonic Inpainting with Finite Elements" (arXiv 2105.01586).

This module is a thin binding over the C ABI of ``libfeminpaint.so``
(declared in ``include/feminpaint.h``): it checks and marshals torch tensors
(device pointers and the current CUDA stream) and converts status codes to
exceptions.  Every step of the computation runs in the library's CUDA
kernels; there is no CPU fallback.  Importing this package raises if the
library has not been built (``python -m paper_2105_01586_gb300._build``).

Functions keep the C names (``fem_inpaint``, ``fem_triangle_errors``,
``fem_spatial_refine``, ``fem_tonal_opt``, ``fem_adjoint``, ...).  ``Mesh``
wraps a handle; ``FemInpaint`` / ``TonalLoss`` (in ``.autograd``) expose the
forward map u = B g and its adjoint to torch autograd.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfeminpaint.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: the CUDA library must be built first "
        "(python -m paper_2105_01586_gb300._build); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

FEM_OK = 0
FEM_E_INVALID = 1
FEM_E_SHAPE = 2
FEM_E_OOM = 3
FEM_E_NOT_CONVERGED = 4
FEM_E_TIMEOUT = 5
FEM_E_CUDA = 6
FEM_E_CANCELLED = 7
FEM_PREC_FP32_IR = 0
FEM_PREC_FP64 = 1
_STATUS = {0: "FEM_OK", 1: "FEM_E_INVALID", 2: "FEM_E_SHAPE", 3: "FEM_E_OOM", 4: "FEM_E_NOT_CONVERGED",
           5: "FEM_E_TIMEOUT", 6: "FEM_E_CUDA", 7: "FEM_E_CANCELLED"}

EXPORTED = ["fem_params_default", "fem_mesh_create", "fem_mesh_destroy", "fem_mesh_info", "fem_mesh_size",
            "fem_mesh_export",
            "fem_mesh_import", "fem_mesh_curve_order", "fem_gather_mask", "fem_inpaint", "fem_triangle_errors", "fem_triangle_error_bounds", "fem_triangle_errors_noalloc", "fem_rasterize", "fem_spatial_refine", "fem_spatial_refine_channels",
            "fem_tonal_opt", "fem_tonal_opt_l1", "fem_adjoint", "fem_tonal_loss", "fem_mesh_stats", "fem_last_error", "fem_profile_enable",
            "fem_profile_read", "fem_launch_count", "fem_selftest_wait_timeout", "fem_server_create",
            "fem_server_submit", "fem_server_wait", "fem_server_result", "fem_server_state", "fem_server_cancel", "fem_server_release",
            "fem_server_destroy", "fem_set_mem_pool", "fem_debug_alloc_fault"]


class fem_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("precision", ctypes.c_int),
                ("topk_frac", ctypes.c_double), ("max_rounds", ctypes.c_int), ("tonal_tol", ctypes.c_double),
                ("tonal_maxit", ctypes.c_int), ("inner_tol", ctypes.c_double), ("fast_keys", ctypes.c_int)]


class fem_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int), ("cg_iters", ctypes.c_longlong), ("solves", ctypes.c_int),
                ("relres", ctypes.c_double), ("tonal_iters", ctypes.c_int), ("tonal_relres", ctypes.c_double),
                ("min_margin", ctypes.c_double)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_ip = ctypes.POINTER(ctypes.c_int)
_pp = ctypes.POINTER(fem_params)
_sig = {
    "fem_params_default": (None, [_pp]),
    "fem_mesh_create": (_i, [_i, _i, _vp, ctypes.POINTER(_vp)]),
    "fem_mesh_destroy": (_i, [_vp]),
    "fem_mesh_info": (_i, [_vp, _ip, _ip, _ip]),
    "fem_mesh_size": (_i, [_vp, _ip, _ip, _ip]),
    "fem_mesh_export": (_i, [_vp, _vp, _vp, _vp]),
    "fem_mesh_import": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "fem_gather_mask": (_i, [_vp, _vp, _vp, _vp]),
    "fem_mesh_curve_order": (_i, [_vp, _vp, _ip]),
    "fem_inpaint": (_i, [_vp, _vp, _vp, _vp, _pp, _vp]),
    "fem_triangle_errors": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fem_triangle_error_bounds": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "fem_triangle_errors_noalloc": (_i, [_i, _i, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "fem_rasterize": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "fem_spatial_refine": (_i, [_vp, _vp, ctypes.c_double, _pp, _vp]),
    "fem_spatial_refine_channels": (_i, [_vp, _vp, _i, ctypes.c_double, _pp, _vp]),
    "fem_tonal_opt": (_i, [_vp, _vp, _vp, _pp, _vp]),
    "fem_tonal_opt_l1": (_i, [_vp, _vp, _vp, _i, ctypes.c_double, _pp, _vp]),
    "fem_adjoint": (_i, [_vp, _vp, _vp, _pp, _vp]),
    "fem_tonal_loss": (_i, [_vp, _vp, _vp, _vp, _vp, _pp, _vp]),
    "fem_mesh_stats": (_i, [_vp, ctypes.POINTER(fem_stats)]),
    "fem_last_error": (ctypes.c_char_p, []),
    "fem_profile_enable": (None, [_i]),
    "fem_profile_read": (_i, [_i, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_char_p)]),
    "fem_launch_count": (ctypes.c_longlong, []),
    "fem_selftest_wait_timeout": (_i, [_vp]),
    "fem_server_create": (_i, [_i, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "fem_server_submit": (_i, [_vp, _i, _vp, ctypes.c_double, _pp, ctypes.POINTER(ctypes.c_longlong)]),
    "fem_server_wait": (_i, [_vp, ctypes.c_longlong, ctypes.c_double, _ip]),
    "fem_server_result": (_i, [_vp, ctypes.c_longlong, _vp, _vp, _vp, _vp, _vp, _vp]),
    "fem_server_cancel": (_i, [_vp, ctypes.c_longlong]),
    "fem_server_state": (_i, [_vp, ctypes.c_longlong, _ip]),
    "fem_server_release": (_i, [_vp, ctypes.c_longlong]),
    "fem_set_mem_pool": (_i, [_vp]),
    "fem_debug_alloc_fault": (_i, [ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    "fem_server_destroy": (_i, [_vp]),
}
for _n, (_r, _a) in _sig.items():
    _f = getattr(_lib, _n)
    _f.restype = _r
    _f.argtypes = _a


class FemError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.fem_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")


def _check(st: int, where: str, allow=()):
    if st != FEM_OK and st not in allow:
        raise FemError(st, where)
    return st


def params(**kw) -> fem_params:
    """Default parameters (fem_params_default) with keyword overrides."""
    p = fem_params()
    _lib.fem_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _torch():
    import torch
    return torch


def _stream(stream=None) -> int:
    torch = _torch()
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtype, numel=None, name="tensor"):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    return t.data_ptr()


# ------------------------------------------------------------------ C names
def fem_mesh_create(width: int, height: int, stream=None) -> int:
    h = _vp()
    _check(_lib.fem_mesh_create(width, height, _stream(stream), ctypes.byref(h)), "fem_mesh_create")
    return h.value


def fem_mesh_destroy(h: int) -> None:
    _lib.fem_mesh_destroy(h)


def fem_mesh_info(h: int) -> tuple[int, int, int]:
    V, T, K = _i(), _i(), _i()
    _check(_lib.fem_mesh_info(h, ctypes.byref(V), ctypes.byref(T), ctypes.byref(K)), "fem_mesh_info")
    return V.value, T.value, K.value


def fem_mesh_size(h: int) -> tuple[int, int, int]:
    """(width, height, domain side N) of the mesh's image."""
    W, H, N = _i(), _i(), _i()
    _check(_lib.fem_mesh_size(h, ctypes.byref(W), ctypes.byref(H), ctypes.byref(N)), "fem_mesh_size")
    return W.value, H.value, N.value


def _pixels(h: int) -> int:
    W, H, _ = fem_mesh_size(h)
    return W * H


def fem_mesh_export(h: int):
    V, T, _ = fem_mesh_info(h)
    xy = np.zeros((V, 2), np.int32)
    tri = np.zeros((T, 3), np.int32)
    mk = np.zeros(V, np.uint8)
    _check(_lib.fem_mesh_export(h, xy.ctypes.data, tri.ctypes.data, mk.ctypes.data), "fem_mesh_export")
    return xy, tri, mk


def fem_mesh_import(h: int, xy, tri, is_mask) -> None:
    xy = np.ascontiguousarray(xy, np.int32).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, np.int32).reshape(-1, 3)
    mk = np.ascontiguousarray(is_mask, np.uint8).reshape(-1)
    _check(_lib.fem_mesh_import(h, len(xy), xy.ctypes.data, len(tri), tri.ctypes.data, mk.ctypes.data),
           "fem_mesh_import")


def fem_mesh_curve_order(h: int):
    """(order, is_curve): the triangle visiting order (see the header)."""
    V, T, _ = fem_mesh_info(h)
    order = np.zeros(T, np.int32)
    ic = _i()
    _check(_lib.fem_mesh_curve_order(h, order.ctypes.data, ctypes.byref(ic)), "fem_mesh_curve_order")
    return order, bool(ic.value)


def fem_gather_mask(h: int, f, g, stream=None):
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    _check(_lib.fem_gather_mask(h, _dev_ptr(f, torch.float32, _pixels(h), "f"), _dev_ptr(g, torch.float32, K, "g"),
                                _stream(stream)), "fem_gather_mask")


def fem_inpaint(h: int, g, u=None, uv=None, p: fem_params | None = None, stream=None, allow_not_converged=False):
    V, T, K = fem_mesh_info(h)
    st = _lib.fem_inpaint(h, _dev_ptr(g, _torch().float32, K, "g"), _dev_ptr(u, _torch().float32, _pixels(h) if u is not None else None, "u"),
                          _dev_ptr(uv, _torch().float64, V, "uv"), ctypes.byref(p or params()), _stream(stream))
    return _check(st, "fem_inpaint", (FEM_E_NOT_CONVERGED,) if allow_not_converged else ())


def fem_triangle_errors(h: int, uv, f, err, stream=None):
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    _check(_lib.fem_triangle_errors(h, _dev_ptr(uv, torch.float64, V, "uv"), _dev_ptr(f, torch.float32, _pixels(h), "f"),
                                    _dev_ptr(err, torch.float64, T, "err"), _stream(stream)), "fem_triangle_errors")


def fem_triangle_error_bounds(h: int, uv, f, lo, hi, stream=None):
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    _check(_lib.fem_triangle_error_bounds(h, _dev_ptr(uv, torch.float64, V, "uv"),
                                          _dev_ptr(f, torch.float32, _pixels(h), "f"), _dev_ptr(lo, torch.float64, T, "lo"),
                                          _dev_ptr(hi, torch.float64, T, "hi"), _stream(stream)),
           "fem_triangle_error_bounds")


def fem_triangle_errors_noalloc(width: int, xy, tri4, uv, f, err, stream=None):
    """Per-triangle errors without any device allocation (fixed library
    scratch; see include/feminpaint.h).  xy: (V, 2) int32, tri4: (T, 4)
    int32 (a, b, c, unused), uv: V float64, f: width*width float32, err: T
    float64, all CUDA tensors the caller owns."""
    torch = _torch()
    V = xy.shape[0]
    T = tri4.shape[0]
    if xy.dim() != 2 or xy.shape[1] != 2 or tri4.dim() != 2 or tri4.shape[1] != 4:
        raise ValueError("xy must be (V, 2) and tri4 (T, 4)")
    _check(_lib.fem_triangle_errors_noalloc(int(width), V, _dev_ptr(xy, torch.int32, 2 * V, "xy"), T,
                                            _dev_ptr(tri4, torch.int32, 4 * T, "tri4"),
                                            _dev_ptr(uv, torch.float64, V, "uv"),
                                            _dev_ptr(f, torch.float32, int(width) * int(width), "f"),
                                            _dev_ptr(err, torch.float64, T, "err"), _stream(stream)),
           "fem_triangle_errors_noalloc")


def fem_rasterize(h: int, uv, u=None, owner=None, stream=None):
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    _check(_lib.fem_rasterize(h, _dev_ptr(uv, torch.float64, V, "uv"), _dev_ptr(u, torch.float32, _pixels(h) if u is not None else None, "u"),
                              _dev_ptr(owner, torch.int32, _pixels(h) if owner is not None else None, "owner"), _stream(stream)), "fem_rasterize")


def fem_spatial_refine(h: int, f, density: float, p: fem_params | None = None, stream=None):
    _check(_lib.fem_spatial_refine(h, _dev_ptr(f, _torch().float32, _pixels(h), "f"), float(density),
                                   ctypes.byref(p or params()), _stream(stream)), "fem_spatial_refine")


def fem_spatial_refine_channels(h: int, f, density: float, p: fem_params | None = None, stream=None):
    """Colour spatial optimisation: f is (C, H, W) float32 on the device."""
    C = int(f.shape[0]) if f.dim() == 3 else 1
    _check(_lib.fem_spatial_refine_channels(h, _dev_ptr(f, _torch().float32, C * _pixels(h), "f"), C,
                                            float(density), ctypes.byref(p or params()), _stream(stream)),
           "fem_spatial_refine_channels")


def fem_tonal_opt(h: int, f, g, p: fem_params | None = None, stream=None, allow_not_converged=False):
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    st = _lib.fem_tonal_opt(h, _dev_ptr(f, torch.float32, _pixels(h), "f"), _dev_ptr(g, torch.float32, K, "g"),
                            ctypes.byref(p or params()), _stream(stream))
    return _check(st, "fem_tonal_opt", (FEM_E_NOT_CONVERGED,) if allow_not_converged else ())


def fem_tonal_opt_l1(h: int, f, g, irls: int = 10, eps: float = 1e-3, p: fem_params | None = None, stream=None,
                     allow_not_converged=False):
    """L1 data term by IRLS (see include/feminpaint.h); g: start and result."""
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    st = _lib.fem_tonal_opt_l1(h, _dev_ptr(f, torch.float32, _pixels(h), "f"), _dev_ptr(g, torch.float32, K, "g"),
                               int(irls), float(eps), ctypes.byref(p or params()), _stream(stream))
    return _check(st, "fem_tonal_opt_l1", (FEM_E_NOT_CONVERGED,) if allow_not_converged else ())


def fem_adjoint(h: int, r, gbar, p: fem_params | None = None, stream=None):
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    _check(_lib.fem_adjoint(h, _dev_ptr(r, torch.float32, _pixels(h), "r"), _dev_ptr(gbar, torch.float32, K, "gbar"),
                            ctypes.byref(p or params()), _stream(stream)), "fem_adjoint")


def fem_tonal_loss(h: int, g, f, loss=None, grad=None, p: fem_params | None = None, stream=None):
    """loss (0-dim float64) = 1/2 ||B g - f||^2 and grad (nmask float32) =
    B^T (B g - f), both written by the library into the given CUDA tensors."""
    V, T, K = fem_mesh_info(h)
    torch = _torch()
    _check(_lib.fem_tonal_loss(h, _dev_ptr(g, torch.float32, K, "g"), _dev_ptr(f, torch.float32, _pixels(h), "f"),
                               _dev_ptr(loss, torch.float64, 1, "loss"), _dev_ptr(grad, torch.float32, K, "grad"),
                               ctypes.byref(p or params()), _stream(stream)), "fem_tonal_loss")


def fem_mesh_stats(h: int) -> dict:
    s = fem_stats()
    _check(_lib.fem_mesh_stats(h, ctypes.byref(s)), "fem_mesh_stats")
    return {k: getattr(s, k) for k, _ in fem_stats._fields_}


FAMILIES = ["raster", "cg", "assembly", "topk", "refine", "tonal", "other", "raster_pass"]


def fem_profile_enable(mask) -> None:
    """mask: int bitmask, True (all families), False/0 (off) or a family name."""
    if isinstance(mask, str):
        mask = 1 << FAMILIES.index(mask)
    elif mask is True:
        mask = (1 << len(FAMILIES)) - 1
    _lib.fem_profile_enable(int(mask))


def fem_profile_read() -> dict:
    out = {}
    for fam in range(len(FAMILIES)):
        n = ctypes.c_longlong()
        ms = ctypes.c_double()
        by = ctypes.c_double()
        name = ctypes.c_char_p()
        _lib.fem_profile_read(fam, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(name))
        out[name.value.decode()] = {"launches": n.value, "ms": ms.value, "bytes": by.value}
    return out


def fem_selftest_wait_timeout(stream=None) -> int:
    """Status of the bounded-wait check (FEM_E_TIMEOUT expected)."""
    return int(_lib.fem_selftest_wait_timeout(_stream(stream)))


def fem_launch_count() -> int:
    return int(_lib.fem_launch_count())


def fem_set_mem_pool(pool) -> None:
    """Device allocations from now on come from `pool` (a cudaMemPool_t as an
    int or c_void_p); None returns to the device's current pool."""
    _check(_lib.fem_set_mem_pool(pool), "fem_set_mem_pool")


def fem_debug_alloc_fault(fail_after: int) -> int:
    """Arm (fail_after >= 0) or disarm (< 0) the injected allocation failure;
    returns the device allocations attempted so far."""
    n = ctypes.c_longlong()
    _check(_lib.fem_debug_alloc_fault(int(fail_after), ctypes.byref(n)), "fem_debug_alloc_fault")
    return int(n.value)


# ------------------------------------------------------------- convenience
class Mesh:
    """Owning wrapper of a mesh handle for a width x height image (height
    defaults to width).  The mesh lives on the smallest (2^L + 1)^2 domain
    that holds the image; only image pixels are data."""

    def __init__(self, width: int, height: int | None = None, stream=None):
        self.width = int(width)
        self.height = int(width if height is None else height)
        self.h = fem_mesh_create(self.width, self.height, stream)
        self.n = fem_mesh_size(self.h)[2]  # the domain side N

    def close(self):
        if getattr(self, "h", None):
            fem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return fem_mesh_info(self.h)

    @property
    def V(self):
        return self.info[0]

    @property
    def T(self):
        return self.info[1]

    @property
    def nmask(self):
        return self.info[2]

    def export(self):
        return fem_mesh_export(self.h)

    def import_(self, xy, tri, is_mask):
        fem_mesh_import(self.h, xy, tri, is_mask)

    def stats(self):
        return fem_mesh_stats(self.h)

    def inpaint(self, g, p=None, want_uv=False, stream=None, allow_not_converged=False):
        torch = _torch()
        u = torch.empty((self.height, self.width), dtype=torch.float32, device=g.device)
        uv = torch.empty(self.V, dtype=torch.float64, device=g.device) if want_uv else None
        fem_inpaint(self.h, g, u, uv, p, stream, allow_not_converged)
        return (u, uv) if want_uv else u

    def triangle_errors(self, uv, f, stream=None):
        torch = _torch()
        err = torch.empty(self.T, dtype=torch.float64, device=f.device)
        fem_triangle_errors(self.h, uv, f, err, stream)
        return err

    def triangle_error_bounds(self, uv, f, stream=None):
        """FP32 intervals [lo, hi] that contain the keys of triangle_errors."""
        torch = _torch()
        lo = torch.empty(self.T, dtype=torch.float64, device=f.device)
        hi = torch.empty(self.T, dtype=torch.float64, device=f.device)
        fem_triangle_error_bounds(self.h, uv, f, lo, hi, stream)
        return lo, hi

    def rasterize(self, uv, want_owner=False, stream=None):
        torch = _torch()
        u = torch.empty((self.height, self.width), dtype=torch.float32, device=uv.device)
        own = torch.empty((self.height, self.width), dtype=torch.int32, device=uv.device) if want_owner else None
        fem_rasterize(self.h, uv, u, own, stream)
        return (u, own) if want_owner else u

    def spatial_refine(self, f, density, p=None, stream=None):
        """f: (H, W) grey, or (C, H, W) colour (C <= 4)."""
        if f.dim() == 3:
            fem_spatial_refine_channels(self.h, f, density, p, stream)
        else:
            fem_spatial_refine(self.h, f, density, p, stream)

    def g_from_f(self, f, stream=None):
        """g = f at the mask vertices (fem_gather_mask)."""
        torch = _torch()
        g = torch.empty(self.nmask, dtype=torch.float32, device=f.device)
        fem_gather_mask(self.h, f, g, stream)
        return g

    def tonal_opt(self, f, g0=None, p=None, stream=None, allow_not_converged=False):
        g = (self.g_from_f(f) if g0 is None else g0).clone()
        fem_tonal_opt(self.h, f, g, p, stream, allow_not_converged)
        return g

    def tonal_opt_l1(self, f, g0=None, irls=10, eps=1e-3, p=None, stream=None, allow_not_converged=False):
        g = (self.g_from_f(f) if g0 is None else g0).clone()
        fem_tonal_opt_l1(self.h, f, g, irls, eps, p, stream, allow_not_converged)
        return g

    def adjoint(self, r, p=None, stream=None):
        torch = _torch()
        gbar = torch.empty(self.nmask, dtype=torch.float32, device=r.device)
        fem_adjoint(self.h, r, gbar, p, stream)
        return gbar
