"""Thin ctypes binding of libohm (include/ohm.h), same entry-point names.

Argument marshalling only: tensors are checked (CUDA, float64, contiguous, shape) and passed
by data_ptr(); every step of the solver runs in the library's CUDA kernels.  There is no
CPU path: if the compiled library is missing this module raises on first use.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

OHM_OK = 0
OHM_ERR_INVALID = -1
OHM_ERR_NOT_CONVERGED = -2
OHM_ERR_NONFINITE = -3
OHM_ERR_OOM = -4
OHM_ERR_CUDA = -5
OHM_FP64 = 0
OHM_MIXED = 1
OHM_MIXED_FF = 2
OHM_MIXED_FF_CHECKED = 3
OHM_K_COMPOSITE, OHM_K_SMOOTH, OHM_K_RESID_RESTRICT, OHM_K_PROLONG, OHM_K_GHOST = 0, 1, 2, 3, 4
OHM_K_SYNC_DOWN, OHM_K_UPDATE, OHM_K_BOTTOM, OHM_K_NORM, OHM_K_KRYLOV = 5, 6, 7, 8, 9

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libohm.so")


class OhmError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} (status {status})")
        self.status = status


class HierDesc(C.Structure):
    _fields_ = [("base_cells", C.c_int32 * 3), ("dx0", C.c_double), ("nlevels", C.c_int32), ("nblocks", C.c_int64),
                ("block_lijk", C.POINTER(C.c_int32)), ("lam", C.c_double), ("precision", C.c_int32),
                ("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("n_coarse", C.c_int32), ("max_outer", C.c_int32),
                ("krylov", C.c_int32), ("inner_tol", C.c_double), ("n_instances", C.c_int32),
                ("use_graphs", C.c_int32), ("stream", C.c_void_p), ("omega", C.c_double),
                ("nu_coarse_pre", C.c_int32), ("nu_coarse_post", C.c_int32)]


class StepStats(C.Structure):
    _fields_ = [("cycles", C.c_int32), ("converged", C.c_int32), ("rel_l2_initial", C.c_double),
                ("rel_l2", C.c_double), ("max_abs", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("nu_pre", C.c_int32), ("nu_post", C.c_int32), ("n_coarse", C.c_int32), ("smoother", C.c_int32),
                ("ms", C.c_double), ("candidates", C.c_int32), ("omega", C.c_double),
                ("nu_coarse_pre", C.c_int32), ("nu_coarse_post", C.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libohm.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                               "python -m paper_1009_0798_gb300.build")
        L = C.CDLL(LIB_PATH)
        vp, dp = C.c_void_p, C.c_double
        L.ohm_create_hierarchy.argtypes = [C.POINTER(HierDesc), C.POINTER(vp)]
        L.ohm_set_eta.argtypes = [vp, vp]
        L.ohm_cn_step.argtypes = [vp, vp, vp, dp, dp, C.POINTER(StepStats)]
        L.ohm_residual_norm.argtypes = [vp, vp, C.POINTER(dp), C.POINTER(dp)]
        L.ohm_destroy.argtypes = [vp]
        L.ohm_destroy.restype = None
        L.ohm_status_string.argtypes = [C.c_int]
        L.ohm_status_string.restype = C.c_char_p
        L.ohm_op_div_flux.argtypes = [vp, vp, vp]
        L.ohm_op_source.argtypes = [vp, vp, dp, vp]
        L.ohm_op_residual.argtypes = [vp, vp, vp, dp, vp, C.POINTER(dp)]
        L.ohm_op_sync_down.argtypes = [vp, vp]
        L.ohm_op_vcycle.argtypes = [vp, vp, dp, vp]
        L.ohm_mg_grid_info.argtypes = [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
        L.ohm_op_grid_smooth.argtypes = [vp, C.c_int, vp, vp, vp, dp, C.c_int]
        L.ohm_op_grid_residual.argtypes = [vp, C.c_int, vp, vp, vp, dp, vp]
        L.ohm_op_grid_restrict.argtypes = [vp, C.c_int, vp, vp, C.c_int]
        L.ohm_op_grid_prolong_add.argtypes = [vp, C.c_int, vp, vp]
        L.ohm_op_grid_sweep_f32.argtypes = [vp, C.c_int, vp, vp, vp, vp, dp, C.c_int]
        L.ohm_op_grid_resid_restrict_f32.argtypes = [vp, C.c_int, vp, vp, vp, dp, vp, vp]
        L.ohm_op_grid_prolong_add_f32.argtypes = [vp, C.c_int, vp, vp]
        L.ohm_op_apply_L_f32.argtypes = [vp, vp, dp, vp]
        L.ohm_op_coarsest_f32.argtypes = [vp, vp, vp, dp, vp]
        L.ohm_prof_enable.argtypes = [vp, C.c_int, C.c_int, C.c_int]
        L.ohm_prof_read.argtypes = [vp, C.POINTER(dp), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.ohm_launch_count.argtypes = [vp]
        L.ohm_launch_count.restype = C.c_int64
        L.ohm_cn_step_batch.argtypes = [vp, vp, C.POINTER(dp), dp, C.POINTER(C.c_uint8), C.POINTER(StepStats)]
        L.ohm_hierarchy_bytes.argtypes = [C.POINTER(HierDesc), C.POINTER(C.c_int64)]
        L.ohm_autotune.argtypes = [vp, vp, C.POINTER(dp), dp, C.POINTER(TuneResult)]
        _lib = L
    return _lib


def status_string(status: int) -> str:
    try:
        return lib().ohm_status_string(status).decode()
    except Exception:  # library not loadable: keep the numeric status
        return "status"


def _ptr(t, numel=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, expected {numel}")
    return C.c_void_p(t.data_ptr())


def _ptr32(t, name="tensor"):
    """float32 CUDA tensor (the mixed-precision inner solve's arrays) or None -> pointer."""
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _check(status: int, what: str, allow=(OHM_OK,)):
    if status not in allow:
        raise OhmError(status, what)
    return status


class Hierarchy:
    """Owning handle of an ohm_hier (ohm_create_hierarchy / ohm_destroy)."""

    def __init__(self, handle, nblocks: int, lam: float, mixed: bool, n_instances: int = 0):
        self._h = handle
        self.nblocks = nblocks  # all instances of a batch
        self.lam = lam
        self.mixed = mixed
        self.n_instances = n_instances

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib().ohm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_desc(base_cells, dx0, blocks, lam, precision, nu_pre, nu_post, n_coarse, max_outer, raw_stream, krylov,
               inner_tol, n_instances, use_graphs, omega=0.0, nu_coarse=(0, 0)):
    d = HierDesc()
    d.base_cells[:] = [int(v) for v in base_cells]
    d.dx0 = float(dx0)
    d.nlevels = int(blocks[:, 0].max()) + 1 if len(blocks) else 0
    d.nblocks = len(blocks)
    d.block_lijk = blocks.ctypes.data_as(C.POINTER(C.c_int32))
    d.lam = float(lam)
    d.precision = int(precision)
    d.nu_pre, d.nu_post, d.n_coarse, d.max_outer = int(nu_pre), int(nu_post), int(n_coarse), int(max_outer)
    d.krylov = int(krylov)
    d.inner_tol = float(inner_tol)
    d.n_instances = int(n_instances)
    d.use_graphs = 1 if use_graphs else 0
    d.stream = C.c_void_p(raw_stream)
    d.omega = float(omega)
    d.nu_coarse_pre, d.nu_coarse_post = int(nu_coarse[0]), int(nu_coarse[1])
    return d


def ohm_create_hierarchy(base_cells, dx0: float, blocks, lam: float = 0.5, precision: int = OHM_FP64,
                         nu_pre: int = 2, nu_post: int = 2, n_coarse: int = 16, max_outer: int = 50,
                         stream=None, krylov: int = 0, inner_tol: float = 0.0, n_instances: int = 0,
                         use_graphs: bool = False, omega: float = 0.0, nu_coarse=(0, 0)) -> Hierarchy:
    """blocks: int32 [nblocks, 4] rows (level, bi, bj, bk) sorted by level (one instance).
    stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None for torch's current stream.
    n_instances >= 1 makes a batch of that many independent instances (ohm_cn_step_batch).
    omega: relaxation factor of the red-black sweeps (0 = 1, the paper's Gauss-Seidel).
    nu_coarse: (pre, post) sweeps on the grids coarser than level 0; (0, 0) = nu_pre, nu_post."""
    import torch
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    if stream is None:
        stream = torch.cuda.current_stream()
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    d = _make_desc(base_cells, dx0, blocks, lam, precision, nu_pre, nu_post, n_coarse, max_outer, raw, krylov,
                   inner_tol, n_instances, use_graphs, omega, nu_coarse)
    h = C.c_void_p()
    _check(lib().ohm_create_hierarchy(C.byref(d), C.byref(h)), "ohm_create_hierarchy")
    return Hierarchy(h, len(blocks) * max(1, int(n_instances)), lam, precision != OHM_FP64, int(n_instances))


def ohm_hierarchy_bytes(base_cells, dx0: float, blocks, lam: float = 0.5, precision: int = OHM_FP64,
                        nu_pre: int = 2, nu_post: int = 2, n_coarse: int = 16, max_outer: int = 50, krylov: int = 0,
                        inner_tol: float = 0.0, n_instances: int = 0, omega: float = 0.0, nu_coarse=(0, 0)) -> int:
    """Device bytes ohm_create_hierarchy would allocate for this description (no allocation)."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32)
    d = _make_desc(base_cells, dx0, blocks, lam, precision, nu_pre, nu_post, n_coarse, max_outer, 0, krylov,
                   inner_tol, n_instances, False, omega, nu_coarse)
    out = C.c_int64()
    _check(lib().ohm_hierarchy_bytes(C.byref(d), C.byref(out)), "ohm_hierarchy_bytes")
    return int(out.value)


def ohm_cn_step_batch(h: Hierarchy, B, dt, tol: float, active=None) -> tuple[int, list]:
    """Batched step in place on B (all instances' blocks, level by level).  dt: one value per
    instance; active: optional per-instance flags.  Returns (status, per-instance stats); raises
    on statuses other than OHM_OK / OHM_ERR_NOT_CONVERGED."""
    K = h.n_instances
    dts = (C.c_double * K)(*[float(v) for v in dt])
    act = None
    if active is not None:
        act = (C.c_uint8 * K)(*[1 if a else 0 for a in active])
    st = (StepStats * K)()
    status = lib().ohm_cn_step_batch(h.handle, _ptr(B, h.nblocks * 1536, "B"), dts, float(tol), act, st)
    _check(status, "ohm_cn_step_batch", allow=(OHM_OK, OHM_ERR_NOT_CONVERGED))
    return status, [{"cycles": x.cycles, "converged": bool(x.converged), "rel_l2_initial": x.rel_l2_initial,
                     "rel_l2": x.rel_l2, "max_abs": x.max_abs} for x in st]


def ohm_autotune(h: Hierarchy, B, dt, tol: float) -> dict:
    """Times the candidate schedules on copies of B and keeps the fastest (see include/ohm.h)."""
    dts = list(dt) if hasattr(dt, "__len__") else [dt]
    arr = (C.c_double * len(dts))(*[float(v) for v in dts])
    r = TuneResult()
    _check(lib().ohm_autotune(h.handle, _ptr(B, h.nblocks * 1536, "B"), arr, float(tol), C.byref(r)), "ohm_autotune")
    return {"nu_pre": r.nu_pre, "nu_post": r.nu_post, "n_coarse": r.n_coarse, "smoother": r.smoother, "ms": r.ms,
            "candidates": r.candidates, "omega": r.omega, "nu_coarse": (r.nu_coarse_pre, r.nu_coarse_post)}


def ohm_set_eta(h: Hierarchy, eta) -> None:
    _check(lib().ohm_set_eta(h.handle, _ptr(eta, h.nblocks * 512, "eta")), "ohm_set_eta")


def ohm_cn_step(h: Hierarchy, B, eta, dt: float, tol: float) -> dict:
    """One implicit step in place on B.  Returns the step statistics; raises OhmError on any
    status other than OHM_OK and OHM_ERR_NOT_CONVERGED (reported as converged=False)."""
    st = StepStats()
    e = _ptr(eta, h.nblocks * 512, "eta") if eta is not None else None
    status = lib().ohm_cn_step(h.handle, _ptr(B, h.nblocks * 1536, "B"), e, float(dt), float(tol), C.byref(st))
    _check(status, "ohm_cn_step", allow=(OHM_OK, OHM_ERR_NOT_CONVERGED))
    return {"status": status, "cycles": st.cycles, "converged": bool(st.converged), "rel_l2_initial": st.rel_l2_initial,
            "rel_l2": st.rel_l2, "max_abs": st.max_abs}


def ohm_residual_norm(h: Hierarchy, B) -> tuple[float, float]:
    r, m = C.c_double(), C.c_double()
    _check(lib().ohm_residual_norm(h.handle, _ptr(B, h.nblocks * 1536, "B"), C.byref(r), C.byref(m)),
           "ohm_residual_norm")
    return r.value, m.value


def ohm_op_div_flux(h: Hierarchy, B, out) -> None:
    _check(lib().ohm_op_div_flux(h.handle, _ptr(B, h.nblocks * 1536, "B"), _ptr(out, h.nblocks * 1536, "out")),
           "ohm_op_div_flux")


def ohm_op_source(h: Hierarchy, b, dt: float, S) -> None:
    _check(lib().ohm_op_source(h.handle, _ptr(b, h.nblocks * 1536, "b"), float(dt), _ptr(S, h.nblocks * 1536, "S")),
           "ohm_op_source")


def ohm_op_residual(h: Hierarchy, B, S, dt: float, R) -> dict:
    n = (C.c_double * 4)()
    _check(lib().ohm_op_residual(h.handle, _ptr(B, h.nblocks * 1536, "B"), _ptr(S, h.nblocks * 1536, "S"), float(dt),
                                 _ptr(R, h.nblocks * 1536, "R"), n), "ohm_op_residual")
    return {"rel_l2": n[0], "max_abs": n[1], "l2_R": n[2], "l2_S": n[3]}


def ohm_op_sync_down(h: Hierarchy, B) -> None:
    _check(lib().ohm_op_sync_down(h.handle, _ptr(B, h.nblocks * 1536, "B")), "ohm_op_sync_down")


def ohm_op_vcycle(h: Hierarchy, R, dt: float, e) -> None:
    _check(lib().ohm_op_vcycle(h.handle, _ptr(R, h.nblocks * 1536, "R"), float(dt), _ptr(e, h.nblocks * 1536, "e")),
           "ohm_op_vcycle")


def ohm_mg_grid_info(h: Hierarchy, m: int):
    dims = (C.c_int32 * 3)()
    nb = C.c_int64()
    _check(lib().ohm_mg_grid_info(h.handle, m, dims, C.byref(nb), None), "ohm_mg_grid_info")
    ijk = np.zeros((max(nb.value, 1), 3), np.int32)
    if nb.value:
        _check(lib().ohm_mg_grid_info(h.handle, m, dims, C.byref(nb), ijk.ctypes.data_as(C.POINTER(C.c_int32))),
               "ohm_mg_grid_info")
    return tuple(dims), nb.value, ijk[: nb.value]


def ohm_op_grid_smooth(h: Hierarchy, m: int, e, r, eta, dt: float, colour: int) -> None:
    _check(lib().ohm_op_grid_smooth(h.handle, m, _ptr(e), _ptr(r), _ptr(eta), float(dt), int(colour)),
           "ohm_op_grid_smooth")


def ohm_op_grid_residual(h: Hierarchy, m: int, e, r, eta, dt: float, t) -> None:
    _check(lib().ohm_op_grid_residual(h.handle, m, _ptr(e), _ptr(r), _ptr(eta), float(dt), _ptr(t)),
           "ohm_op_grid_residual")


def ohm_op_grid_restrict(h: Hierarchy, m: int, fine, coarse, ncomp: int = 3) -> None:
    _check(lib().ohm_op_grid_restrict(h.handle, m, _ptr(fine), _ptr(coarse), int(ncomp)), "ohm_op_grid_restrict")


def ohm_op_grid_prolong_add(h: Hierarchy, m: int, coarse, fine) -> None:
    _check(lib().ohm_op_grid_prolong_add(h.handle, m, _ptr(coarse), _ptr(fine)), "ohm_op_grid_prolong_add")


def ohm_op_grid_sweep_f32(h: Hierarchy, m: int, e_in, e_out, r, eta, dt: float, variant: int = 0) -> None:
    """One float32 red-black sweep on grid m (e_in None = from zero); variant 0 fused, 1 two passes."""
    _check(lib().ohm_op_grid_sweep_f32(h.handle, m, _ptr32(e_in, "e_in"), _ptr32(e_out, "e_out"), _ptr32(r, "r"),
                                       _ptr32(eta, "eta"), float(dt), int(variant)), "ohm_op_grid_sweep_f32")


def ohm_op_grid_resid_restrict_f32(h: Hierarchy, m: int, e, r, eta, dt: float, t=None, coarse=None) -> None:
    _check(lib().ohm_op_grid_resid_restrict_f32(h.handle, m, _ptr32(e, "e"), _ptr32(r, "r"), _ptr32(eta, "eta"),
                                                float(dt), _ptr32(t, "t"), _ptr32(coarse, "coarse")),
           "ohm_op_grid_resid_restrict_f32")


def ohm_op_grid_prolong_add_f32(h: Hierarchy, m: int, coarse, fine) -> None:
    _check(lib().ohm_op_grid_prolong_add_f32(h.handle, m, _ptr32(coarse, "coarse"), _ptr32(fine, "fine")),
           "ohm_op_grid_prolong_add_f32")


def ohm_op_coarsest_f32(h: Hierarchy, r, eta, dt: float, e) -> None:
    _check(lib().ohm_op_coarsest_f32(h.handle, _ptr32(r, "r"), _ptr32(eta, "eta"), float(dt), _ptr32(e, "e")),
           "ohm_op_coarsest_f32")


def ohm_op_apply_L_f32(h: Hierarchy, X, dt: float, out) -> None:
    _check(lib().ohm_op_apply_L_f32(h.handle, _ptr32(X, "X"), float(dt), _ptr32(out, "out")), "ohm_op_apply_L_f32")


def ohm_prof_enable(h: Hierarchy, kernel: int, min_blocks: int = 0, max_launches: int = 4096) -> None:
    _check(lib().ohm_prof_enable(h.handle, int(kernel), int(min_blocks), int(max_launches)), "ohm_prof_enable")


def ohm_prof_read(h: Hierarchy) -> dict:
    ms, n, cells = C.c_double(), C.c_int64(), C.c_int64()
    _check(lib().ohm_prof_read(h.handle, C.byref(ms), C.byref(n), C.byref(cells)), "ohm_prof_read")
    return {"ms": ms.value, "launches": n.value, "cells": cells.value}


def ohm_launch_count(h: Hierarchy) -> int:
    return int(lib().ohm_launch_count(h.handle))


def ohm_fp64_fma_rate(stream=None) -> float:
    """Measured float64 FMA instructions per second of the current device (include/ohm.h)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    L = lib()
    if not getattr(L.ohm_fp64_fma_rate, "argtypes", None):
        L.ohm_fp64_fma_rate.argtypes = [C.POINTER(C.c_double), C.c_void_p]
    v = C.c_double()
    _check(L.ohm_fp64_fma_rate(C.byref(v), C.c_void_p(raw)), "ohm_fp64_fma_rate")
    return v.value


def ohm_residual_static(base_cells, dx: float, lam: float, dt: float, block_ijk, B, S, eta, R, stream=None) -> dict:
    """Allocation-free residual on one uniform periodic grid (no hierarchy needed), for
    callers that cannot allocate device memory; see include/ohm.h.  block_ijk: int32 [n, 3]."""
    import torch
    ijk = np.ascontiguousarray(block_ijk, dtype=np.int32)
    n = len(ijk)
    if stream is None:
        stream = torch.cuda.current_stream()
    raw = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    L = lib()
    if not getattr(L.ohm_residual_static, "argtypes", None):
        L.ohm_residual_static.argtypes = [C.POINTER(C.c_int32), C.c_double, C.c_double, C.c_double, C.c_int64,
                                          C.POINTER(C.c_int32), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.POINTER(C.c_double), C.c_void_p]
    cells = (C.c_int32 * 3)(*[int(v) for v in base_cells])
    out = (C.c_double * 4)()
    _check(L.ohm_residual_static(cells, float(dx), float(lam), float(dt), n, ijk.ctypes.data_as(C.POINTER(C.c_int32)),
                                 _ptr(B, n * 1536, "B"), _ptr(S, n * 1536, "S"), _ptr(eta, n * 512, "eta"),
                                 _ptr(R, n * 1536, "R"), out, C.c_void_p(raw)), "ohm_residual_static")
    return {"rel_l2": out[0], "max_abs": out[1], "l2_R": out[2], "l2_S": out[3]}
