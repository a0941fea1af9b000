"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

Arrays use the block layout of the solver's C ABI: float64 [nblocks][3][8][8][8] for vector
fields and [nblocks][1][8][8][8] (or [nblocks][8][8][8]) for eta, in block-list order.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_long, ip, C.c_double,
                                 C.c_char_p, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_nmg.argtypes = [C.c_void_p]
        L.orc_mg_dims.argtypes = [C.c_void_p, C.c_int, ip]
        L.orc_set_eta.argtypes = [C.c_void_p, dp]
        L.orc_mg_eta.argtypes = [C.c_void_p, C.c_int, dp]
        L.orc_div_flux.argtypes = [C.c_void_p, dp, dp]
        L.orc_apply_L.argtypes = [C.c_void_p, dp, C.c_double, dp]
        L.orc_source.argtypes = [C.c_void_p, dp, C.c_double, dp]
        L.orc_residual.argtypes = [C.c_void_p, dp, dp, C.c_double, dp, dp]
        L.orc_vcycle.argtypes = [C.c_void_p, dp, C.c_double, ip, dp]
        L.orc_cn_step.argtypes = [C.c_void_p, dp, C.c_double, C.c_double, ip, dp, C.POINTER(C.c_int)]
        L.orc_heun_step.argtypes = [C.c_void_p, dp, C.c_double]
        L.orc_sync_down.argtypes = [C.c_void_p, dp]
        L.orc_grid_smooth.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, C.c_double, C.c_int]
        L.orc_grid_residual.argtypes = [C.c_void_p, C.c_int, dp, dp, dp, C.c_double, dp]
        L.orc_grid_restrict.argtypes = [C.c_void_p, C.c_int, dp, dp, C.c_int]
        L.orc_grid_prolong_add.argtypes = [C.c_void_p, C.c_int, dp, dp]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    """FP64 CPU reference solver on one block hierarchy (see ohm_oracle.c)."""

    def __init__(self, hier, lam: float = 0.5, eta=None):
        self.hier = hier
        self.lam = lam
        err = C.create_string_buffer(256)
        blocks = np.ascontiguousarray(hier.blocks, dtype=np.int32)
        nx, ny, nz = hier.base_cells
        self._h = lib().orc_create(nx, ny, nz, hier.dx0, hier.nlevels, len(blocks), blocks, lam, err, 256)
        if not self._h:
            raise ValueError("oracle: " + err.value.decode())
        self.nb = len(blocks)
        if eta is not None:
            self.set_eta(eta)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def _vec(self, a) -> np.ndarray:
        a = _f64(a)
        assert a.size == self.nb * 3 * 512, a.shape
        return a

    @property
    def n_mg(self) -> int:
        return lib().orc_nmg(self._h)

    def mg_dims(self, m: int) -> tuple[int, int, int]:
        d = np.zeros(3, np.int32)
        assert lib().orc_mg_dims(self._h, m, d) == 0
        return tuple(int(v) for v in d)

    def set_eta(self, eta):
        eta = _f64(eta)
        assert eta.size == self.nb * 512
        lib().orc_set_eta(self._h, eta)

    def mg_eta(self, m: int) -> np.ndarray:
        """eta of base multigrid grid m, dense [nz][ny][nx] (grid 0 is the base level)."""
        nx, ny, nz = self.mg_dims(m)
        out = np.zeros((nz, ny, nx))
        assert lib().orc_mg_eta(self._h, m, out) == 0
        return out

    def div_flux(self, B) -> np.ndarray:
        out = np.zeros((self.nb, 3, 8, 8, 8))
        lib().orc_div_flux(self._h, self._vec(B), out)
        return out

    def apply_L(self, B, dt: float) -> np.ndarray:
        out = np.zeros((self.nb, 3, 8, 8, 8))
        lib().orc_apply_L(self._h, self._vec(B), dt, out)
        return out

    def source(self, b, dt: float) -> np.ndarray:
        out = np.zeros((self.nb, 3, 8, 8, 8))
        lib().orc_source(self._h, self._vec(b), dt, out)
        return out

    def residual(self, B, S, dt: float):
        R = np.zeros((self.nb, 3, 8, 8, 8))
        norms = np.zeros(4)
        lib().orc_residual(self._h, self._vec(B), self._vec(S), dt, R, norms)
        return R, {"rel_l2": norms[0], "max_abs": norms[1], "l2_R": norms[2], "l2_S": norms[3]}

    def vcycle(self, R, dt: float, nu_pre=2, nu_post=2, n_coarse=16) -> np.ndarray:
        e = np.zeros((self.nb, 3, 8, 8, 8))
        lib().orc_vcycle(self._h, self._vec(R), dt, np.array([nu_pre, nu_post, n_coarse], np.int32), e)
        return e

    def cn_step(self, B, dt: float, tol: float, nu_pre=2, nu_post=2, n_coarse=16, max_outer=50):
        """One step; returns (B_new, info).  tol < 0 runs exactly max_outer V-cycles."""
        Bn = self._vec(B).copy()
        hist = np.zeros(max_outer + 1)
        nc = C.c_int(0)
        st = lib().orc_cn_step(self._h, Bn, dt, tol, np.array([nu_pre, nu_post, n_coarse, max_outer], np.int32),
                               hist, C.byref(nc))
        return Bn.reshape(self.nb, 3, 8, 8, 8), {"converged": st == 0, "cycles": nc.value,
                                                 "history": hist[: nc.value + 1].copy()}

    def heun_step(self, B, dt: float) -> np.ndarray:
        Bn = self._vec(B).copy()
        lib().orc_heun_step(self._h, Bn, dt)
        return Bn.reshape(self.nb, 3, 8, 8, 8)

    def sync_down(self, B) -> np.ndarray:
        Bn = self._vec(B).copy()
        lib().orc_sync_down(self._h, Bn)
        return Bn.reshape(self.nb, 3, 8, 8, 8)

    # single uniform grid pieces (dense [comp][nz][ny][nx] on base multigrid grid m)
    def grid_smooth(self, m, e, r, eta, dt, colour):
        e = _f64(e).copy()
        lib().orc_grid_smooth(self._h, m, e, _f64(r), _f64(eta), dt, colour)
        return e

    def grid_residual(self, m, e, r, eta, dt):
        t = np.zeros_like(_f64(e))
        lib().orc_grid_residual(self._h, m, _f64(e), _f64(r), _f64(eta), dt, t)
        return t

    def grid_restrict(self, m, fine, ncomp=3):
        nx, ny, nz = self.mg_dims(m + 1)
        out = np.zeros((ncomp, nz, ny, nx))
        lib().orc_grid_restrict(self._h, m, _f64(fine), out, ncomp)
        return out

    def grid_prolong_add(self, m, coarse, fine):
        fine = _f64(fine).copy()
        lib().orc_grid_prolong_add(self._h, m, _f64(coarse), fine)
        return fine
