"""CPU FP64 oracle for FEM harmonic inpainting with spatial and tonal data
optimisation (Chizhov & Weickert, arXiv 2105.01586).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg import this package.  The product path (the CUDA library and
its binding) never imports it; the two share no code.  The arithmetic lives
in ``oracle.c`` (plain scalar C, FP64); this module only marshals numpy arrays
and adds a few numpy conveniences (eligibility flags, g = f at the mask).

Functions and the paper passages they follow:
  mesh_init   initial two-triangle mesh (replaces the Delaunay mesh of Sec. 2.2)
  refine      one newest-vertex-bisection round (Sec. 3 as adapted: top-k)
  stiffness   the P1 FEM matrix of Sec. 2.2
  solve       the Laplace solve on the unknown vertices by CG (Sec. 2.2)
  raster      linear interpolation to all pixels (Sec. 2.2) and the per-
              triangle squared errors of Sec. 3
  scatter     the transpose of the interpolation
  select_topk descending-error order of Sec. 3, ties by triangle id
  spatial     the spatial optimisation loop (Sec. 3, adapted)
  apply_B, apply_BT, tonal   u = B g and the normal equations of Sec. 4

Images are H x W arrays.  A W x H image that is not square with side
2^L + 1 lies at the top-left of the smallest such square domain, which
carries the mesh; only image pixels are data (reading R9 of oracle.c).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "_liboracle.so")
_SO_OMP = os.path.join(_HERE, "_liboracle_omp.so")

OM_OK = 0
OM_E_INVALID = 1
OM_E_OOM = 3
OM_E_NOT_CONVERGED = 4
LOG_COLS = 8

_libs = {}
_openmp = False


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c into the oracle library used by the tests (gcc, plain
    C11).  openmp=True builds the multi-core variant (-fopenmp) used as the
    second CPU baseline; its results are bit-identical (see oracle.c)."""
    so = _SO_OMP if openmp else _SO
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(_SRC):
        tmp = so + ".tmp.%d" % os.getpid()
        extra = ["-fopenmp"] if openmp else []
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", *extra, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, so)
    return so


def use_openmp(on: bool = True) -> int:
    """Meshes created from now on use the OpenMP build (on=True) or the
    single-thread build (on=False).  Returns the thread count of that build
    (OMP_NUM_THREADS, else all host cores)."""
    global _openmp
    _openmp = bool(on)
    return int(_load().om_threads())


def _load():
    L = _libs.get(_openmp)
    if L is not None:
        return L
    so = build(openmp=_openmp)
    L = ctypes.CDLL(so)
    P = ctypes.c_void_p
    ip = ctypes.POINTER(ctypes.c_int)
    dp = ctypes.POINTER(ctypes.c_double)
    fp = ctypes.POINTER(ctypes.c_float)
    up = ctypes.POINTER(ctypes.c_ubyte)
    L.om_mesh_new.restype = P
    L.om_mesh_new.argtypes = [ctypes.c_int]
    L.om_mesh_new_image.restype = P
    L.om_mesh_new_image.argtypes = [ctypes.c_int, ctypes.c_int]
    L.om_mesh_set_image.argtypes = [P, ctypes.c_int, ctypes.c_int]
    L.om_mesh_from.restype = P
    L.om_mesh_from.argtypes = [ctypes.c_int, ctypes.c_int, ip, ip, up, ctypes.c_int, ip, ip, ip]
    L.om_mesh_free.argtypes = [P]
    for n in ("om_mesh_V", "om_mesh_T", "om_mesh_N", "om_mesh_W", "om_mesh_H"):
        getattr(L, n).argtypes = [P]
        getattr(L, n).restype = ctypes.c_int
    L.om_mesh_get.argtypes = [P, ip, ip, up, ip, ip, ip]
    L.om_refine.argtypes = [P, ip, ctypes.c_int, ip]
    L.om_refine_par.argtypes = [P, ip, ctypes.c_int, ip, ip]
    L.om_stiffness_csr.argtypes = [P, ip, ip, dp, ctypes.c_int]
    L.om_solve.argtypes = [P, dp, ctypes.c_double, ctypes.c_int, ip, dp]
    L.om_raster.argtypes = [P, dp, fp, dp, dp, ip]
    L.om_scatter.argtypes = [P, dp, dp]
    L.om_topk_count.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_long]
    L.om_topk_count.restype = ctypes.c_int
    L.om_select_topk.argtypes = [P, dp, ctypes.c_int, ip, dp]
    L.om_select_topk.restype = ctypes.c_int
    L.om_spatial.argtypes = [P, fp, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                             ctypes.c_int, dp, ctypes.c_int, ip]
    L.om_spatial_channels.argtypes = [P, fp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                      ctypes.c_double, ctypes.c_int, dp, ctypes.c_int, ip]
    L.om_apply_B.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int]
    L.om_apply_BT.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int]
    L.om_tonal.argtypes = [P, fp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int, dp]
    L.om_tonal_l1.argtypes = [P, fp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                              ctypes.c_double, ctypes.c_int, dp]
    L.om_threads.restype = ctypes.c_int
    _libs[_openmp] = L
    return L


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != OM_OK:
        raise OracleError(f"{what} failed with status {rc}")


@dataclass
class Mesh:
    """A triangle mesh on the pixel grid of the N x N domain (N = 2^L + 1)
    that holds a W x H image (W = H = N unless given).  Triangle t is
    (ta[t], tb[t], tc[t]): refinement edge (ta, tb), newest vertex tc."""
    N: int
    vx: np.ndarray
    vy: np.ndarray
    mask: np.ndarray
    ta: np.ndarray
    tb: np.ndarray
    tc: np.ndarray
    W: int = 0
    H: int = 0

    def __post_init__(self):
        self.W = int(self.W) or int(self.N)
        self.H = int(self.H) or int(self.N)

    @property
    def V(self) -> int:
        return len(self.vx)

    @property
    def T(self) -> int:
        return len(self.ta)

    @property
    def tri(self) -> np.ndarray:
        return np.stack([self.ta, self.tb, self.tc], axis=1)

    @property
    def xy(self) -> np.ndarray:
        return np.stack([self.vx, self.vy], axis=1)

    def copy(self) -> "Mesh":
        return Mesh(self.N, self.vx.copy(), self.vy.copy(), self.mask.copy(),
                    self.ta.copy(), self.tb.copy(), self.tc.copy(), self.W, self.H)

    def with_mask(self, mask) -> "Mesh":
        m = self.copy()
        m.mask = np.ascontiguousarray(mask, dtype=np.uint8)
        return m


class _CMesh:
    def __init__(self, mesh: Mesh | None = None, N: int | None = None, W: int | None = None, H: int | None = None):
        L = _load()
        if mesh is None and W is not None:
            self.p = L.om_mesh_new_image(int(W), int(H))
            if not self.p:
                raise OracleError("image sides must be at least 2")
        elif mesh is None:
            self.p = L.om_mesh_new(int(N))
            if not self.p:
                raise OracleError("image side must be 2^L + 1")
        else:
            c = [np.ascontiguousarray(a, dtype=np.int32) for a in (mesh.vx, mesh.vy, mesh.ta, mesh.tb, mesh.tc)]
            mk = np.ascontiguousarray(mesh.mask, dtype=np.uint8)
            self.p = L.om_mesh_from(int(mesh.N), len(c[0]), _ptr(c[0], ctypes.c_int), _ptr(c[1], ctypes.c_int),
                                    _ptr(mk, ctypes.c_ubyte), len(c[2]), _ptr(c[2], ctypes.c_int),
                                    _ptr(c[3], ctypes.c_int), _ptr(c[4], ctypes.c_int))
            if self.p and (mesh.W, mesh.H) != (mesh.N, mesh.N):
                _check(L.om_mesh_set_image(self.p, int(mesh.W), int(mesh.H)), "set_image")
        self.L = L

    def to_mesh(self) -> Mesh:
        L = self.L
        V, T, N = L.om_mesh_V(self.p), L.om_mesh_T(self.p), L.om_mesh_N(self.p)
        W, H = L.om_mesh_W(self.p), L.om_mesh_H(self.p)
        vx = np.empty(V, np.int32); vy = np.empty(V, np.int32); mk = np.empty(V, np.uint8)
        ta = np.empty(T, np.int32); tb = np.empty(T, np.int32); tc = np.empty(T, np.int32)
        L.om_mesh_get(self.p, _ptr(vx, ctypes.c_int), _ptr(vy, ctypes.c_int), _ptr(mk, ctypes.c_ubyte),
                      _ptr(ta, ctypes.c_int), _ptr(tb, ctypes.c_int), _ptr(tc, ctypes.c_int))
        return Mesh(N, vx, vy, mk, ta, tb, tc, W, H)

    def __del__(self):
        if getattr(self, "p", None):
            self.L.om_mesh_free(self.p)
            self.p = None


def mesh_init(N: int, H: int | None = None) -> Mesh:
    """Two triangles on the corners of the domain: of an N x N image
    (N = 2^L + 1), or with H given of an N x H (width x height) image in the
    smallest domain that holds it."""
    if H is None:
        return _CMesh(N=N).to_mesh()
    return _CMesh(W=N, H=H).to_mesh()


def refine(mesh: Mesh, selected) -> tuple[Mesh, dict]:
    """One NVB round with the given selected triangles (their refinement-edge
    midpoints become mask vertices; closure-only midpoints are unknowns).
    info["parents"][i] holds the ends of the edge new vertex V + i bisects."""
    cm = _CMesh(mesh)
    sel = np.ascontiguousarray(selected, dtype=np.int32)
    info = np.zeros(4, np.int32)
    par = np.zeros(2 * (mesh.V + mesh.T), np.int32)
    _check(cm.L.om_refine_par(cm.p, _ptr(sel, ctypes.c_int), len(sel), _ptr(info, ctypes.c_int),
                              _ptr(par, ctypes.c_int)), "refine")
    return cm.to_mesh(), {"new_vertices": int(info[0]), "new_triangles": int(info[1]),
                          "generations": int(info[2]), "new_mask": int(info[3]),
                          "parents": par[: 2 * int(info[0])].reshape(-1, 2).copy()}


def stiffness(mesh: Mesh):
    """The full V x V P1 stiffness matrix as a scipy CSR matrix."""
    import scipy.sparse as sp
    cm = _CMesh(mesh)
    cap = mesh.V * 17 + 16
    rowptr = np.zeros(mesh.V + 1, np.int32)
    col = np.zeros(cap, np.int32)
    val = np.zeros(cap, np.float64)
    _check(cm.L.om_stiffness_csr(cm.p, _ptr(rowptr, ctypes.c_int), _ptr(col, ctypes.c_int),
                                 _ptr(val, ctypes.c_double), cap), "stiffness")
    n = rowptr[-1]
    return sp.csr_matrix((val[:n], col[:n], rowptr), shape=(mesh.V, mesh.V))


def g_from_f(mesh: Mesh, f: np.ndarray) -> np.ndarray:
    """Dirichlet data g = f at the mask vertices, in ascending vertex id (a
    vertex outside the image takes the nearest image pixel)."""
    k = mesh.mask.astype(bool)
    return f[np.minimum(mesh.vy[k], mesh.H - 1), np.minimum(mesh.vx[k], mesh.W - 1)].astype(np.float64)


def vertex_values(mesh: Mesh, g: np.ndarray, start: np.ndarray | None = None) -> np.ndarray:
    v = np.zeros(mesh.V) if start is None else np.array(start, dtype=np.float64)
    v[mesh.mask.astype(bool)] = g
    return v


def solve(mesh: Mesh, g: np.ndarray, start: np.ndarray | None = None, tol: float = 1e-13,
          maxit: int = 1_000_000) -> tuple[np.ndarray, int, float]:
    """Vertex values: g at the mask vertices, the FEM Laplace solution at the
    unknown vertices.  Returns (values, CG iterations, relative residual)."""
    cm = _CMesh(mesh)
    uv = np.ascontiguousarray(vertex_values(mesh, g, start))
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    _check(cm.L.om_solve(cm.p, _ptr(uv, ctypes.c_double), tol, maxit, ctypes.byref(it), ctypes.byref(rr)), "solve")
    return uv, it.value, rr.value


def raster(mesh: Mesh, v: np.ndarray, f: np.ndarray | None = None, owner: bool = False):
    """Interpolate vertex values v to all image pixels.  Returns (u image
    (H x W), per-triangle squared errors against f (or None), owner map (or
    None))."""
    cm = _CMesh(mesh)
    vv = np.ascontiguousarray(v, dtype=np.float64)
    u = np.zeros((mesh.H, mesh.W), np.float64)
    keys = np.zeros(mesh.T, np.float64) if f is not None else None
    own = np.zeros((mesh.H, mesh.W), np.int32) if owner else None
    ff = np.ascontiguousarray(f, dtype=np.float32) if f is not None else None
    rc = cm.L.om_raster(cm.p, _ptr(vv, ctypes.c_double),
                        _ptr(ff, ctypes.c_float) if ff is not None else None,
                        _ptr(u, ctypes.c_double),
                        _ptr(keys, ctypes.c_double) if keys is not None else None,
                        _ptr(own, ctypes.c_int) if own is not None else None)
    _check(rc, "raster")
    return u, keys, own


def scatter(mesh: Mesh, r: np.ndarray) -> np.ndarray:
    """P^T r: V-vector."""
    cm = _CMesh(mesh)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    s = np.zeros(mesh.V, np.float64)
    _check(cm.L.om_scatter(cm.p, _ptr(rr, ctypes.c_double), _ptr(s, ctypes.c_double)), "scatter")
    return s


def eligible(mesh: Mesh) -> np.ndarray:
    """Triangles whose refinement-edge midpoint is a pixel and whose
    bounding box meets the image."""
    sx = mesh.vx[mesh.ta] + mesh.vx[mesh.tb]
    sy = mesh.vy[mesh.ta] + mesh.vy[mesh.tb]
    xmin = np.minimum(np.minimum(mesh.vx[mesh.ta], mesh.vx[mesh.tb]), mesh.vx[mesh.tc])
    ymin = np.minimum(np.minimum(mesh.vy[mesh.ta], mesh.vy[mesh.tb]), mesh.vy[mesh.tc])
    return ((sx % 2) == 0) & ((sy % 2) == 0) & (xmin < mesh.W) & (ymin < mesh.H)


def topk_count(T: int, frac: float, n_eligible: int, vcap: int) -> int:
    return int(_load().om_topk_count(int(T), float(frac), int(n_eligible), int(vcap)))


def select_topk(mesh: Mesh, keys: np.ndarray, k: int) -> tuple[np.ndarray, float]:
    cm = _CMesh(mesh)
    kk = np.ascontiguousarray(keys, dtype=np.float64)
    sel = np.zeros(max(1, mesh.T), np.int32)
    marg = ctypes.c_double(0)
    n = cm.L.om_select_topk(cm.p, _ptr(kk, ctypes.c_double), int(k), _ptr(sel, ctypes.c_int), ctypes.byref(marg))
    if n < 0:
        raise OracleError("select_topk failed")
    return sel[:n].copy(), marg.value


def vstar(N: int, density: float, H: int | None = None) -> int:
    """ceil(density * pixels) of an N x N image, or of an N x H one."""
    import math
    return int(math.ceil(density * float(N * (N if H is None else H))))


def spatial(f: np.ndarray, density: float, frac: float, max_rounds: int = 0, tol: float = 1e-13,
            maxit: int = 1_000_000, mesh: Mesh | None = None, log_cap: int = 100_000):
    """Spatial optimisation: refine from the two-triangle mesh (or `mesh`)
    until V >= ceil(density * W H) or max_rounds rounds (> 0); f is H x W,
    or C x H x W for C channels (colour: the channels share the mesh, each
    has its own solve, a triangle's error is the sum over the channels).
    Returns (mesh, log) with log columns V, T, k, margin, CG iterations,
    relres, new vertices, new mask vertices (one row per round)."""
    C = 1 if f.ndim == 2 else f.shape[0]
    H, W = f.shape[-2:]
    cm = _CMesh(mesh) if mesh is not None else _CMesh(W=W, H=H)
    ff = np.ascontiguousarray(f, dtype=np.float32)
    log = np.zeros((log_cap, LOG_COLS), np.float64)
    rounds = ctypes.c_int(0)
    if f.ndim == 2:
        rc = cm.L.om_spatial(cm.p, _ptr(ff, ctypes.c_float), float(density), float(frac), int(max_rounds), tol,
                             maxit, _ptr(log, ctypes.c_double), log_cap, ctypes.byref(rounds))
    else:
        rc = cm.L.om_spatial_channels(cm.p, _ptr(ff, ctypes.c_float), C, float(density), float(frac),
                                      int(max_rounds), tol, maxit, _ptr(log, ctypes.c_double), log_cap,
                                      ctypes.byref(rounds))
    _check(rc, "spatial")
    return cm.to_mesh(), log[: min(rounds.value, log_cap)].copy()


def apply_B(mesh: Mesh, g: np.ndarray, tol: float = 1e-14, maxit: int = 1_000_000) -> np.ndarray:
    cm = _CMesh(mesh)
    gg = np.ascontiguousarray(g, dtype=np.float64)
    u = np.zeros((mesh.H, mesh.W), np.float64)
    _check(cm.L.om_apply_B(cm.p, _ptr(gg, ctypes.c_double), _ptr(u, ctypes.c_double), tol, maxit), "apply_B")
    return u


def apply_BT(mesh: Mesh, r: np.ndarray, tol: float = 1e-14, maxit: int = 1_000_000) -> np.ndarray:
    cm = _CMesh(mesh)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(int(mesh.mask.sum()), np.float64)
    _check(cm.L.om_apply_BT(cm.p, _ptr(rr, ctypes.c_double), _ptr(out, ctypes.c_double), tol, maxit), "apply_BT")
    return out


def tonal(mesh: Mesh, f: np.ndarray, g0: np.ndarray | None = None, tol: float = 1e-10, maxit: int = 10_000,
          inner_tol: float = 1e-14, inner_maxit: int = 1_000_000, allow_not_converged: bool = False):
    """CGLS on the normal equations (eq. 5).  Returns (g, stats) with stats
    outer iterations, relative normal residual, inner CG iterations, SSE."""
    cm = _CMesh(mesh)
    ff = np.ascontiguousarray(f, dtype=np.float32)
    g = np.ascontiguousarray(g_from_f(mesh, f) if g0 is None else g0, dtype=np.float64).copy()
    st = np.zeros(4, np.float64)
    rc = cm.L.om_tonal(cm.p, _ptr(ff, ctypes.c_float), _ptr(g, ctypes.c_double), tol, maxit, inner_tol,
                       inner_maxit, _ptr(st, ctypes.c_double))
    if not (rc == OM_OK or (allow_not_converged and rc == OM_E_NOT_CONVERGED)):
        _check(rc, "tonal")
    return g, {"iters": int(st[0]), "relres": float(st[1]), "inner_iters": int(st[2]), "sse": float(st[3]),
               "status": int(rc)}


def tonal_l1(mesh: Mesh, f: np.ndarray, g0: np.ndarray | None = None, irls: int = 10, eps: float = 1e-3,
             tol: float = 1e-12, maxit: int = 10_000, inner_tol: float = 1e-14, inner_maxit: int = 1_000_000):
    """The L1 data term (Sec. 5): min_g sum |B g - f| by IRLS, `irls` steps of
    weighted least squares with weights 1 / max(|B g - f|, eps), each from the
    current g (start g0, default f at the mask).  Returns (g, stats) with the
    CG iterations, the last step's relative residual, inner iterations, the
    L1 objective and the Huber objective at the end."""
    cm = _CMesh(mesh)
    ff = np.ascontiguousarray(f, dtype=np.float32)
    g = np.ascontiguousarray(g_from_f(mesh, f) if g0 is None else g0, dtype=np.float64).copy()
    st = np.zeros(5, np.float64)
    _check(cm.L.om_tonal_l1(cm.p, _ptr(ff, ctypes.c_float), _ptr(g, ctypes.c_double), int(irls), float(eps), tol,
                            maxit, inner_tol, inner_maxit, _ptr(st, ctypes.c_double)), "tonal_l1")
    return g, {"iters": int(st[0]), "relres": float(st[1]), "inner_iters": int(st[2]), "l1": float(st[3]),
               "huber": float(st[4])}
