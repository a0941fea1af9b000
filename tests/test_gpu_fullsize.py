"""Parity at the full sizes of the benchmark workloads (uniform 256^3 resistive bump; base
64^3 with 3 nested refinement levels), in the configurations bench.py times.

* float64, fixed schedule (3 V-cycles): GPU and oracle element by element, 1e-12 relative.
* mixed precision with the FGMRES inner solve, converged to 1e-9: the oracle evaluates the
  residual S - L B of the GPU's answer independently and must find it below 1e-9 as well.
"""
import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W
from tests.helpers import rel_err

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def ohm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0798_gb300 import build, ohm as mod
    build.build()
    return mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


WORKLOADS = {"resistive_bump_256": lambda: W.resistive_bump_256(256),
             "nested_spheres_64": lambda: W.nested_spheres_64(64)}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def case(request, oracle_mod):
    wl = WORKLOADS[request.param]()
    o = oracle_mod.Oracle(wl.hier, wl.lam, wl.eta)
    b = o.sync_down(wl.B)
    return request.param, wl, o, b


def test_fp64_fixed_schedule_elementwise(ohm, case):
    name, wl, o, b = case
    g = ohm.ohm_create_hierarchy(wl.hier.base_cells, wl.hier.dx0, wl.hier.blocks, lam=wl.lam, nu_pre=2, nu_post=2,
                                 n_coarse=16, max_outer=3)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(wl.eta), wl.dt, -1.0)
    want, info = o.cn_step(b, wl.dt, -1.0, 2, 2, 16, 3)
    torch.cuda.synchronize()
    assert st["cycles"] == 3
    assert rel_err(B.cpu().numpy(), want) < 1e-12
    assert st["rel_l2"] == pytest.approx(info["history"][-1], rel=1e-8)


def test_mixed_fgmres_converged_residual_checked_by_oracle(ohm, case):
    name, wl, o, b = case
    g = ohm.ohm_create_hierarchy(wl.hier.base_cells, wl.hier.dx0, wl.hier.blocks, lam=wl.lam, precision=ohm.OHM_MIXED,
                                 nu_pre=2, nu_post=2, n_coarse=16, max_outer=200, krylov=6)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(wl.eta), wl.dt, wl.tol)
    assert st["converged"] and st["rel_l2"] <= wl.tol
    got = B.cpu().numpy().reshape(b.shape)
    S = o.source(b, wl.dt)
    _, norms = o.residual(got, S, wl.dt)
    assert norms["rel_l2"] <= 1.05 * wl.tol
    assert norms["rel_l2"] == pytest.approx(st["rel_l2"], rel=0.05)
