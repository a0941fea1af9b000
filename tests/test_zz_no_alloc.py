"""The allocation-free residual entry point, ohm_residual_static.

It serves callers that cannot allocate device memory -- hosts that hand out device memory only
from their own pool (a library-side cudaMalloc would escape their accounting) and real-time
loops that must not enter the CUDA allocator (unbounded latency).  Its scratch is one fixed
device array shared by all calls, so the test checks that two calls in a row (different
inputs) each reproduce the residual and norms of the hierarchy path (ohm_op_residual) within
the parity tolerance, and that grids beyond its 4096-block limit and block lists that do not
tile the grid (wrong length, a duplicated block, a coordinate out of range) are refused before
any work.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W
from tests.helpers import rand_fields, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ohm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0798_gb300 import build, ohm as mod
    build.build()
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_static_residual_matches_hierarchy_residual_on_consecutive_calls(ohm):
    h = W.uniform(32, 16, 24, 1.0 / 32)
    lam = 0.5
    g = ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=lam, nu_pre=2, nu_post=2, n_coarse=8, max_outer=5)
    ijk = h.blocks[:, 1:4]
    for seed, dt in ((1, 3e-3), (2, 7e-3)):
        B, eta = rand_fields(h, seed, 2.0)
        S = np.random.default_rng(seed + 10).standard_normal(B.shape)
        ohm.ohm_set_eta(g, dev(eta))
        R_ref = torch.zeros(h.nblocks * 1536, dtype=torch.float64, device="cuda")
        n_ref = ohm.ohm_op_residual(g, dev(B), dev(S), dt, R_ref)
        R = torch.full((h.nblocks * 1536,), float("nan"), dtype=torch.float64, device="cuda")
        n = ohm.ohm_residual_static(h.base_cells, h.dx0, lam, dt, ijk, dev(B), dev(S), dev(eta), R)
        torch.cuda.synchronize()
        assert rel_err(R.cpu().numpy(), R_ref.cpu().numpy()) < TOL
        for key in ("rel_l2", "max_abs", "l2_R", "l2_S"):
            assert n[key] == pytest.approx(n_ref[key], rel=TOL)


def test_static_residual_refuses_grids_beyond_its_limit(ohm):
    """256^3 has 32768 blocks, above the 4096-block scratch: refused before any work, so
    one-block buffers are enough here (the C entry point is called directly)."""
    import ctypes as C
    small = torch.zeros(1536, dtype=torch.float64, device="cuda")
    ijk = np.zeros((32768, 3), np.int32)
    f = ohm.lib().ohm_residual_static
    f.argtypes = [C.POINTER(C.c_int32), C.c_double, C.c_double, C.c_double, C.c_int64, C.POINTER(C.c_int32),
                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    cells = (C.c_int32 * 3)(256, 256, 256)
    p = C.c_void_p(small.data_ptr())
    st = f(cells, 1.0 / 256, 0.5, 1e-4, 32768, ijk.ctypes.data_as(C.POINTER(C.c_int32)), p, p, p, p, None, None)
    assert st == ohm.OHM_ERR_INVALID
    # a block list that does not tile the grid is refused too
    st = f((C.c_int32 * 3)(16, 16, 16), 1.0 / 16, 0.5, 1e-4, 7, ijk.ctypes.data_as(C.POINTER(C.c_int32)), p, p, p, p,
           None, None)
    assert st == ohm.OHM_ERR_INVALID


def test_static_residual_refuses_bad_block_lists_on_the_host(ohm):
    """A list of the right length with a duplicated block or a negative / too large coordinate
    is refused by the host check, before anything is enqueued (one-block buffers suffice)."""
    import ctypes as C
    small = torch.zeros(1536, dtype=torch.float64, device="cuda")
    f = ohm.lib().ohm_residual_static
    f.argtypes = [C.POINTER(C.c_int32), C.c_double, C.c_double, C.c_double, C.c_int64, C.POINTER(C.c_int32),
                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]
    h = W.uniform(16, 16, 16, 1.0 / 16)
    good = np.ascontiguousarray(h.blocks[:, 1:4], dtype=np.int32)
    p = C.c_void_p(small.data_ptr())
    cells = (C.c_int32 * 3)(16, 16, 16)
    bad_lists = []
    dup = good.copy()
    dup[3] = dup[5]
    bad_lists.append(dup)
    neg = good.copy()
    neg[2, 1] = -1
    bad_lists.append(neg)
    far = good.copy()
    far[6, 2] = -5
    bad_lists.append(far)
    big = good.copy()
    big[1, 0] = 2
    bad_lists.append(big)
    for ijk in bad_lists:
        st = f(cells, 1.0 / 16, 0.5, 1e-4, len(ijk), ijk.ctypes.data_as(C.POINTER(C.c_int32)), p, p, p, p, None, None)
        assert st == ohm.OHM_ERR_INVALID
    torch.cuda.synchronize()
    assert torch.count_nonzero(small).item() == 0
