"""Thin ctypes binding of the solve service (include/ohm_server.h), same entry-point names.

Argument marshalling only: the queue, admission, batching and device work all run in the
native library; there is no Python or CPU path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import ohm as _ohm

OHM_ERR_TIMEOUT = -6


class ServerDesc(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_int64), ("max_batch", C.c_int32), ("n_workers", C.c_int32),
                ("precision", C.c_int32), ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("n_coarse", C.c_int32),
                ("max_outer", C.c_int32), ("lam", C.c_double), ("tol", C.c_double), ("use_graphs", C.c_int32),
                ("krylov", C.c_int32), ("omega", C.c_double), ("nu_coarse_pre", C.c_int32),
                ("nu_coarse_post", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("base_cells", C.c_int32 * 3), ("dx0", C.c_double), ("nlevels", C.c_int32), ("nblocks", C.c_int64),
                ("block_lijk", C.POINTER(C.c_int32)), ("B", C.POINTER(C.c_double)), ("eta", C.POINTER(C.c_double)),
                ("dt", C.c_double), ("nsteps", C.c_int32), ("B_out", C.POINTER(C.c_double))]


class RequestResult(C.Structure):
    _fields_ = [("status", C.c_int32), ("cycles", C.c_int32), ("rel_l2", C.c_double), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double), ("slot", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("requests_done", C.c_int64), ("batches_created", C.c_int64), ("batches_evicted", C.c_int64),
                ("bytes_resident", C.c_int64), ("bytes_resident_max", C.c_int64), ("steps_run", C.c_int64),
                ("mean_active_slots", C.c_double), ("kernel_launches", C.c_int64)]


_bound = False


def _lib():
    global _bound
    L = _ohm.lib()
    if not _bound:
        vp = C.c_void_p
        L.ohm_server_create.argtypes = [C.POINTER(ServerDesc), C.POINTER(vp)]
        L.ohm_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_int64)]
        L.ohm_server_wait.argtypes = [vp, C.c_int64, C.c_double, C.POINTER(RequestResult)]
        L.ohm_server_clock.argtypes = [vp]
        L.ohm_server_clock.restype = C.c_double
        L.ohm_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
        L.ohm_server_destroy.argtypes = [vp]
        L.ohm_server_destroy.restype = None
        _bound = True
    return L


class Server:
    """Owning handle of an ohm_server.  submit() keeps the request's output array alive until
    wait() returns it."""

    def __init__(self, hbm_budget_bytes: int, max_batch: int = 8, n_workers: int = 4, precision: int = 1,
                 nu_pre: int = 2, nu_post: int = 2, n_coarse: int = 16, max_outer: int = 400, lam: float = 0.5,
                 tol: float = 1e-9, use_graphs: bool = False, krylov: int = 0, omega: float = 0.0,
                 nu_coarse=(0, 0)):
        d = ServerDesc(int(hbm_budget_bytes), int(max_batch), int(n_workers), int(precision), int(nu_pre),
                       int(nu_post), int(n_coarse), int(max_outer), float(lam), float(tol), 1 if use_graphs else 0,
                       int(krylov), float(omega), int(nu_coarse[0]), int(nu_coarse[1]))
        h = C.c_void_p()
        _ohm._check(_lib().ohm_server_create(C.byref(d), C.byref(h)), "ohm_server_create")
        self._h = h
        self._out = {}

    def submit(self, hier, B: np.ndarray, eta: np.ndarray, dt: float, nsteps: int) -> int:
        blocks = np.ascontiguousarray(hier.blocks, dtype=np.int32)
        B = np.ascontiguousarray(B, dtype=np.float64)
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        nb = len(blocks)
        if B.size != nb * 1536 or eta.size != nb * 512:
            raise ValueError("B / eta do not match the block list")
        out = np.empty(nb * 1536, dtype=np.float64)
        r = Request()
        r.base_cells[:] = [int(v) for v in hier.base_cells]
        r.dx0 = float(hier.dx0)
        r.nlevels = int(blocks[:, 0].max()) + 1
        r.nblocks = nb
        dp = C.POINTER(C.c_double)
        r.block_lijk = blocks.ctypes.data_as(C.POINTER(C.c_int32))
        r.B = B.ctypes.data_as(dp)
        r.eta = eta.ctypes.data_as(dp)
        r.dt = float(dt)
        r.nsteps = int(nsteps)
        r.B_out = out.ctypes.data_as(dp)
        rid = C.c_int64()
        _ohm._check(_lib().ohm_server_submit(self._h, C.byref(r), C.byref(rid)), "ohm_server_submit")
        self._out[rid.value] = out
        return rid.value

    def wait(self, rid: int, timeout_s: float = -1.0):
        """Returns (B after the request's steps, result dict), or None on timeout."""
        res = RequestResult()
        st = _lib().ohm_server_wait(self._h, int(rid), float(timeout_s), C.byref(res))
        if st == OHM_ERR_TIMEOUT:
            return None
        _ohm._check(st, "ohm_server_wait")
        out = self._out.pop(int(rid))
        return out, {"status": res.status, "cycles": res.cycles, "rel_l2": res.rel_l2, "t_submit": res.t_submit,
                     "t_start": res.t_start, "t_done": res.t_done, "slot": res.slot}

    def clock(self) -> float:
        return _lib().ohm_server_clock(self._h)

    def stats(self) -> dict:
        s = ServerStats()
        _ohm._check(_lib().ohm_server_get_stats(self._h, C.byref(s)), "ohm_server_get_stats")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            _lib().ohm_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
