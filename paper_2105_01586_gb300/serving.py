"""Continuous-batching server over the C ABI (fem_server_*): whole data-
optimisation jobs (spatial + tonal) admitted into worker slots by device
memory, overlapping on the GPU.  See include/feminpaint.h."""
from __future__ import annotations

import ctypes

import numpy as np

from . import FEM_E_NOT_CONVERGED, FEM_OK, FemError, _check, _lib, fem_params, params


class Server:
    def __init__(self, slots: int = 8, mem_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        _check(_lib.fem_server_create(int(slots), int(mem_budget_bytes), ctypes.byref(h)), "fem_server_create")
        self.h = h.value

    def submit(self, f: np.ndarray, density: float, p: fem_params | None = None) -> int:
        f = np.ascontiguousarray(f, dtype=np.float32)
        if f.ndim != 2 or f.shape[0] != f.shape[1]:
            raise ValueError("f must be a square image")
        rid = ctypes.c_longlong()
        _check(_lib.fem_server_submit(self.h, f.shape[0], f.ctypes.data, float(density),
                                      ctypes.byref(p or params()), ctypes.byref(rid)), "fem_server_submit")
        return rid.value

    def wait(self, rid: int, timeout: float = -1.0) -> bool:
        done = ctypes.c_int()
        _check(_lib.fem_server_wait(self.h, rid, float(timeout), ctypes.byref(done)), "fem_server_wait")
        return bool(done.value)

    def result(self, rid: int) -> dict:
        sizes = np.zeros(4, np.int32)
        st = _lib.fem_server_result(self.h, rid, sizes.ctypes.data, None, None, None, None, None)
        if st not in (FEM_OK, FEM_E_NOT_CONVERGED):
            raise FemError(st, "fem_server_result")
        V, T, K, width = (int(v) for v in sizes)
        xy = np.zeros((V, 2), np.int32)
        tri = np.zeros((T, 3), np.int32)
        mk = np.zeros(V, np.uint8)
        g = np.zeros(K, np.float32)
        times = np.zeros(9, np.float64)
        st = _lib.fem_server_result(self.h, rid, sizes.ctypes.data, xy.ctypes.data, tri.ctypes.data, mk.ctypes.data,
                                    g.ctypes.data, times.ctypes.data)
        return {"status": int(st), "width": width, "xy": xy, "tri": tri, "mask": mk, "g": g,
                "t_submit": times[0], "t_start": times[1], "t_end": times[2], "rounds": int(times[3]),
                "cg_iters": int(times[4]), "tonal_iters": int(times[5]), "tonal_relres": float(times[6]),
                "mem_estimate": int(times[7]), "mem_measured": int(times[8])}

    def state(self, rid: int) -> str:
        """"queued", "running" or "finished" (fem_server_state)."""
        st = ctypes.c_int()
        _check(_lib.fem_server_state(self.h, rid, ctypes.byref(st)), "fem_server_state")
        return ("queued", "running", "finished")[st.value]

    def cancel(self, rid: int) -> None:
        """Cancel a queued or running request (fem_server_cancel); it then
        finishes with status FEM_E_CANCELLED."""
        _check(_lib.fem_server_cancel(self.h, rid), "fem_server_cancel")

    def status(self, rid: int) -> int:
        """Status of a finished request (FEM_OK, FEM_E_NOT_CONVERGED,
        FEM_E_CANCELLED, ...)."""
        sizes = np.zeros(4, np.int32)
        return int(_lib.fem_server_result(self.h, rid, sizes.ctypes.data, None, None, None, None, None))

    def release(self, rid: int) -> None:
        _check(_lib.fem_server_release(self.h, rid), "fem_server_release")

    def close(self) -> None:
        if getattr(self, "h", None):
            _lib.fem_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
