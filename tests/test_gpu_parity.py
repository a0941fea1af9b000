"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, element by element,
on seeded inputs: each hot-path step on its own, then whole V-cycles and CN steps.

Tolerance: 1e-12 relative L2 for FP64 (the kernels and the oracle differ only in rounding
order); mixed precision is held to 1e-9 after refinement to 1e-11.
"""
import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W
from tests.helpers import amr_three_level, amr_two_level, dense_of_grid, grid_of_dense, rand_fields, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def ohm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0798_gb300 import build, ohm as mod
    build.build()
    return mod


@pytest.fixture(scope="module")
def orc(oracle_mod):
    return oracle_mod


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def make(ohm, h, lam=0.5, precision=0, **kw):
    p = dict(nu_pre=2, nu_post=2, n_coarse=8, max_outer=50)
    p.update(kw)
    return ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=lam, precision=precision, **p)


HIERS = {
    "uniform_16x24x8": lambda: W.uniform(16, 24, 8, 1.0 / 16),
    "uniform_32": lambda: W.uniform(32, 32, 32, 1.0 / 32),
    "amr_2level": lambda: amr_two_level(16),
    "amr_3level": lambda: amr_three_level(16),
    "sinusoid_e1": lambda: W.sinusoid_half_refined(N=8).hier,
}


# ------------------------------------------------------------------ single steps
@pytest.mark.parametrize("name", list(HIERS))
def test_div_flux(ohm, orc, name):
    """a1 ghost fill + a2 face fluxes + a8 refluxing + a9 sync of covered cells."""
    h = HIERS[name]()
    B, eta = rand_fields(h, 1, 2.0)
    o = orc.Oracle(h, 0.5, eta)
    g = make(ohm, h)
    ohm.ohm_set_eta(g, dev(eta))
    out = torch.zeros(h.nblocks * 1536, dtype=torch.float64, device="cuda")
    ohm.ohm_op_div_flux(g, dev(B), out)
    assert rel_err(host(out), o.div_flux(B).ravel()) < TOL64


@pytest.mark.parametrize("name", ["uniform_16x24x8", "amr_3level"])
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_source_and_residual(ohm, orc, name, lam):
    """a3 source (Eq. 14) and a4 residual with norms (Eq. 20)."""
    h = HIERS[name]()
    b, eta = rand_fields(h, 2, 2.0)
    B = b + 0.1 * np.random.default_rng(3).standard_normal(b.shape)
    dt = 3.0 * h.dx(h.nlevels - 1) ** 2
    o = orc.Oracle(h, lam, eta)
    g = make(ohm, h, lam=lam)
    ohm.ohm_set_eta(g, dev(eta))
    S = torch.zeros(h.nblocks * 1536, dtype=torch.float64, device="cuda")
    ohm.ohm_op_source(g, dev(b), dt, S)
    S_ref = o.source(b, dt)
    assert rel_err(host(S), S_ref.ravel()) < TOL64
    R = torch.zeros_like(S)
    norms = ohm.ohm_op_residual(g, dev(B), dev(S_ref), dt, R)
    R_ref, n_ref = o.residual(B, S_ref, dt)
    assert rel_err(host(R), R_ref.ravel()) < TOL64
    assert norms["rel_l2"] == pytest.approx(n_ref["rel_l2"], rel=1e-12)
    assert norms["max_abs"] == pytest.approx(n_ref["max_abs"], rel=1e-12)


@pytest.mark.parametrize("name", ["amr_2level", "amr_3level"])
def test_sync_down(ohm, orc, name):
    """a9: covered cells become the mean of their children, finest first."""
    h = HIERS[name]()
    B, eta = rand_fields(h, 4)
    g = make(ohm, h)
    t = dev(B)
    ohm.ohm_op_sync_down(g, t)
    assert rel_err(host(t), orc.Oracle(h, 0.5, eta).sync_down(B).ravel()) < 1e-15


@pytest.mark.parametrize("m", [0, 1])
@pytest.mark.parametrize("colour", [0, 1])
def test_grid_smooth(ohm, orc, m, colour):
    """a5: one red-black colour pass on base multigrid grid m."""
    h = W.uniform(64, 32, 32, 1.0 / 64)
    o = orc.Oracle(h, 0.5)
    g = make(ohm, h)
    dims, nb, ijk = ohm.ohm_mg_grid_info(g, m)
    rng = np.random.default_rng(10 + m)
    e = rng.standard_normal((3,) + dims[::-1])
    r = rng.standard_normal((3,) + dims[::-1])
    eta = 10 ** rng.uniform(-1, 1, (1,) + dims[::-1])
    dt = 5.0 * h.dx0 ** 2
    et = dev(grid_of_dense(e, ijk))
    ohm.ohm_op_grid_smooth(g, m, et, dev(grid_of_dense(r, ijk)), dev(grid_of_dense(eta, ijk)), dt, colour)
    got = dense_of_grid(host(et).reshape(nb, 3, 8, 8, 8), ijk, dims, 3)
    want = o.grid_smooth(m, e, r, eta, dt, colour)
    assert rel_err(got, want) < TOL64


@pytest.mark.parametrize("colour", [0, 1])
def test_grid_smooth_relaxed(ohm, orc, colour):
    """A colour pass of a hierarchy with omega = 1.3 (red-black SOR) moves every cell of the
    colour 1.3 times as far as the oracle's Gauss-Seidel pass and leaves the other colour."""
    h = W.uniform(32, 32, 32, 1.0 / 32)
    o = orc.Oracle(h, 0.5)
    g = make(ohm, h, omega=1.3)
    dims, nb, ijk = ohm.ohm_mg_grid_info(g, 0)
    rng = np.random.default_rng(17)
    e = rng.standard_normal((3,) + dims[::-1])
    r = rng.standard_normal((3,) + dims[::-1])
    eta = 10 ** rng.uniform(-1, 1, (1,) + dims[::-1])
    dt = 5.0 * h.dx0 ** 2
    et = dev(grid_of_dense(e, ijk))
    ohm.ohm_op_grid_smooth(g, 0, et, dev(grid_of_dense(r, ijk)), dev(grid_of_dense(eta, ijk)), dt, colour)
    got = dense_of_grid(host(et).reshape(nb, 3, 8, 8, 8), ijk, dims, 3)
    gs = o.grid_smooth(0, e, r, eta, dt, colour)
    moved = np.abs(gs - e).max(axis=0) > 0
    assert rel_err(got, e + 1.3 * (gs - e)) < TOL64
    assert np.array_equal(got[:, ~moved], e[:, ~moved])


@pytest.mark.parametrize("m", [0, 1])
def test_grid_residual_restrict_prolong(ohm, orc, m):
    """a4 (level residual), a6 restriction, a7 prolongation on base multigrid grid m."""
    h = W.uniform(64, 32, 32, 1.0 / 64)
    o = orc.Oracle(h, 0.5)
    g = make(ohm, h)
    dims, nb, ijk = ohm.ohm_mg_grid_info(g, m)
    cdims, cnb, cijk = ohm.ohm_mg_grid_info(g, m + 1)
    rng = np.random.default_rng(20 + m)
    e = rng.standard_normal((3,) + dims[::-1])
    r = rng.standard_normal((3,) + dims[::-1])
    eta = 10 ** rng.uniform(-1, 1, (1,) + dims[::-1])
    dt = 5.0 * h.dx0 ** 2
    t = torch.zeros(nb * 1536, dtype=torch.float64, device="cuda")
    ohm.ohm_op_grid_residual(g, m, dev(grid_of_dense(e, ijk)), dev(grid_of_dense(r, ijk)), dev(grid_of_dense(eta, ijk)), dt, t)
    got = dense_of_grid(host(t).reshape(nb, 3, 8, 8, 8), ijk, dims, 3)
    assert rel_err(got, o.grid_residual(m, e, r, eta, dt)) < TOL64
    # restriction of 3 and 1 components
    for nc, f in ((3, e), (1, eta)):
        ct = torch.zeros(cnb * 512 * nc, dtype=torch.float64, device="cuda")
        ohm.ohm_op_grid_restrict(g, m, dev(grid_of_dense(f, ijk)), ct, nc)
        got = dense_of_grid(host(ct).reshape(cnb, nc, 8, 8, 8), cijk, cdims, nc)
        assert rel_err(got, o.grid_restrict(m, f, nc)) < 1e-15
    # prolongation
    c = rng.standard_normal((3,) + cdims[::-1])
    ft = dev(grid_of_dense(r, ijk))
    ohm.ohm_op_grid_prolong_add(g, m, dev(grid_of_dense(c, cijk)), ft)
    got = dense_of_grid(host(ft).reshape(nb, 3, 8, 8, 8), ijk, dims, 3)
    assert rel_err(got, o.grid_prolong_add(m, c, r)) < 1e-15


# ------------------------------------------------------------------ whole cycles
@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("nu", [(2, 2), (1, 3)])
def test_vcycle(ohm, orc, name, nu):
    """One V-cycle (a5, a6, a7, a11 and the AMR coarse-fine ghosts) from a zero guess."""
    h = HIERS[name]()
    R, eta = rand_fields(h, 5, 2.0)
    R[~h.is_leaf()] = 0.0
    dt = 8.0 * h.dx(h.nlevels - 1) ** 2
    o = orc.Oracle(h, 0.5, eta)
    g = make(ohm, h, nu_pre=nu[0], nu_post=nu[1], n_coarse=6)
    ohm.ohm_set_eta(g, dev(eta))
    e = torch.zeros(h.nblocks * 1536, dtype=torch.float64, device="cuda")
    ohm.ohm_op_vcycle(g, dev(R), dt, e)
    want = o.vcycle(R, dt, nu[0], nu[1], 6)
    assert rel_err(host(e), want.ravel()) < TOL64


@pytest.mark.parametrize("edge", [56, 104])
def test_coarse_grids_beyond_one_block(ohm, orc, edge):
    """Base grids whose first coarsening that is not a multiple of 8 has more cells than the
    one-block coarsest solver takes (56^3 -> 28^3, 104^3 -> 52^3 and 26^3): the grid-wide coarse
    steps.  A fixed-schedule FP64 step equals the oracle's to 1e-12, and a mixed-precision step
    converged to 1e-9 has an oracle-evaluated residual below 1.05e-9."""
    h = W.uniform(edge, edge, edge, 1.0 / edge)
    b, eta = rand_fields(h, 30, 2.0)
    dt = 20.0 * h.dx0 ** 2
    o = orc.Oracle(h, 0.5, eta)
    g = make(ohm, h, nu_pre=2, nu_post=2, n_coarse=6, max_outer=2)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, -1.0)
    want, _ = o.cn_step(b, dt, -1.0, 2, 2, 6, 2)
    assert st["cycles"] == 2
    assert rel_err(host(B), want.ravel()) < TOL64
    gm = make(ohm, h, precision=1, nu_pre=3, nu_post=2, n_coarse=2, max_outer=200, krylov=6, omega=1.2,
              nu_coarse=(1, 0))
    Bm = dev(b)
    sm = ohm.ohm_cn_step(gm, Bm, dev(eta), dt, 1e-9)
    assert sm["converged"]
    _, norms = o.residual(host(Bm).reshape(b.shape), o.source(b, dt), dt)
    assert norms["rel_l2"] <= 1.05e-9


@pytest.mark.parametrize("name", list(HIERS))
@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_cn_step_fixed_schedule(ohm, orc, name, lam):
    """Whole step with a fixed number of cycles: identical schedule on both sides."""
    h = HIERS[name]()
    b, eta = rand_fields(h, 6, 2.0)
    dt = 6.0 * h.dx(h.nlevels - 1) ** 2
    o = orc.Oracle(h, lam, eta)
    g = make(ohm, h, lam=lam, max_outer=4, n_coarse=6)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, -1.0)
    want, info = o.cn_step(b, dt, -1.0, 2, 2, 6, 4)
    assert st["cycles"] == 4
    assert rel_err(host(B), want.ravel()) < TOL64
    assert st["rel_l2"] == pytest.approx(info["history"][-1], rel=1e-9)


@pytest.mark.parametrize("name", ["uniform_32", "amr_3level"])
def test_cn_step_converged(ohm, orc, name):
    """Both sides converged to 1e-13 reach the same B^{n+1}."""
    h = HIERS[name]()
    b, eta = rand_fields(h, 7, 1.0)
    b = orc.Oracle(h, 0.5, eta).sync_down(b)
    dt = 3.0 * h.dx(h.nlevels - 1) ** 2
    o = orc.Oracle(h, 0.5, eta)
    g = make(ohm, h, max_outer=80)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, 1e-13)
    want, info = o.cn_step(b, dt, 1e-13, 2, 2, 8, 80)
    assert st["converged"] and info["converged"]
    assert rel_err(host(B), want.ravel()) < TOL64
    rel, mx = ohm.ohm_residual_norm(g, B)
    assert rel <= 1e-13


def test_periodic_box_32_workload(ohm, orc):
    """The 32^3 periodic workload (eta = 1, dt = 10x explicit limit): 20 CN steps to 1e-10
    on the GPU track the oracle step by step."""
    wl = W.periodic_box_32()
    o = orc.Oracle(wl.hier, 0.5, wl.eta)
    g = make(ohm, wl.hier, max_outer=60)
    B = dev(wl.B)
    ohm.ohm_set_eta(g, dev(wl.eta))
    Bo = wl.B.copy()
    for _ in range(wl.steps):
        st = ohm.ohm_cn_step(g, B, None, wl.dt, wl.tol)
        Bo, info = o.cn_step(Bo, wl.dt, wl.tol, 2, 2, 8, 60)
        assert st["converged"]
    assert rel_err(host(B), Bo.ravel()) < 1e-10


# ------------------------------------------------------------------ mixed precision
@pytest.mark.parametrize("name", ["uniform_32", "amr_3level", "sinusoid_e1"])
@pytest.mark.parametrize("krylov", [0, 4])
@pytest.mark.parametrize("precision", [1, 2, 3])
def test_mixed_precision_matches_fp64_oracle(ohm, orc, name, krylov, precision):
    """FP32 multigrid (plain or FGMRES-accelerated) inside FP64 iterative refinement reaches
    the FP64 solution.  OHM_MIXED_FF_CHECKED (3) ends the step on a float64 residual: the norm
    it reports is the float64 one of its result."""
    h = HIERS[name]()
    b, eta = rand_fields(h, 8, 1.0)
    b = orc.Oracle(h, 0.5, eta).sync_down(b)
    dt = 4.0 * h.dx(h.nlevels - 1) ** 2
    want, _ = orc.Oracle(h, 0.5, eta).cn_step(b, dt, 1e-14, 2, 2, 8, 80)
    g = make(ohm, h, precision=precision, max_outer=80, krylov=krylov)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, 1e-11)
    assert st["converged"]
    assert rel_err(host(B), want.ravel()) < 1e-9
    rel, _ = ohm.ohm_residual_norm(g, B)
    assert rel <= 1e-11
    if precision == 3:
        assert st["rel_l2"] == pytest.approx(rel, rel=1e-9)


@pytest.mark.parametrize("name", ["uniform_32", "amr_3level", "sinusoid_e1"])
def test_fp64_fgmres_matches_oracle(ohm, orc, name):
    """OHM_FP64 with FGMRES(4) right-preconditioned by the float64 V-cycle (one solve to the
    tolerance per outer iteration) reaches the oracle's converged solution, in fewer V-cycles
    than the float64 defect correction."""
    h = HIERS[name]()
    b, eta = rand_fields(h, 8, 1.0)
    b = orc.Oracle(h, 0.5, eta).sync_down(b)
    dt = 4.0 * h.dx(h.nlevels - 1) ** 2
    want, _ = orc.Oracle(h, 0.5, eta).cn_step(b, dt, 1e-14, 2, 2, 8, 80)
    cyc = {}
    for kr in (0, 4):
        g = make(ohm, h, precision=0, max_outer=80, krylov=kr)
        B = dev(b)
        st = ohm.ohm_cn_step(g, B, dev(eta), dt, 1e-12)
        assert st["converged"]
        assert rel_err(host(B), want.ravel()) < 1e-10
        rel, _ = ohm.ohm_residual_norm(g, B)
        assert rel <= 1e-12
        cyc[kr] = st["cycles"]
    print(name, cyc)
    assert cyc[4] < cyc[0]


# relative residual each mixed mode reports at the oracle's converged solution (float64: rounding;
# float-float: about 2^-48 times the operator's scale), and the accuracy of its norms
OUTER = {1: (1e-13, 1e-12), 2: (1e-12, 1e-5)}


@pytest.mark.parametrize("name", ["uniform_32", "amr_3level"])
@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_outer_residual_accuracy(ohm, orc, name, precision):
    """The outer residual of OHM_MIXED (float64) and OHM_MIXED_FF (float-float, about 48 bits).
    At the oracle's converged float64 solution both report a relative residual near their
    rounding level (a float32 evaluation reports about 1e-6 here, as does a dropped trailing
    part of a coefficient or field); on an unconverged field their norms agree with the
    oracle's (float-float accumulates them in float32)."""
    h = HIERS[name]()
    b, eta = rand_fields(h, 13, 1.0)
    o = orc.Oracle(h, 0.5, eta)
    b = o.sync_down(b)
    dt = 4.0 * h.dx(h.nlevels - 1) ** 2
    want, info = o.cn_step(b, dt, 1e-14, 2, 2, 8, 80)
    assert info["converged"]
    g = make(ohm, h, precision=precision)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, 1e30)  # stores the source S of b, B unchanged
    assert st["cycles"] == 0 and rel_err(host(B), b.ravel()) == 0.0
    rel, _ = ohm.ohm_residual_norm(g, dev(want))
    _, n_want = o.residual(want, o.source(b, dt), dt)
    assert n_want["rel_l2"] < 1e-14
    bound, norm_rel = OUTER[precision]
    assert rel < bound, rel
    rel0, mx0 = ohm.ohm_residual_norm(g, dev(b))
    _, n0 = o.residual(b, o.source(b, dt), dt)
    assert rel0 == pytest.approx(n0["rel_l2"], rel=norm_rel)
    assert mx0 == pytest.approx(n0["max_abs"], rel=max(norm_rel, 1e-6))


@pytest.mark.parametrize("precision", [1, 2, 3])
@pytest.mark.parametrize("bad", ["nan_eta", "inf_B", "huge_B"])
def test_mixed_nonfinite_inputs_report_nonfinite(ohm, bad, precision):
    """NaN, infinity and (for the float-float residual, which splits float64 values into
    float32 pairs) values beyond the float32 range end a mixed step with OHM_ERR_NONFINITE."""
    h = W.uniform(16, 16, 16, 1.0 / 16)
    g = make(ohm, h, precision=precision, max_outer=3)
    b, eta = rand_fields(h, 12)
    if bad == "nan_eta":
        eta[3, 0, 1, 2, 3] = float("nan")
    elif bad == "inf_B":
        b[5, 1, 2, 3, 4] = float("inf")
    else:
        b[5, 1, 2, 3, 4] = 1e300
    with pytest.raises(ohm.OhmError) as ei:
        ohm.ohm_cn_step(g, dev(b), dev(eta), 0.01, 1e-9)
    assert ei.value.status == ohm.OHM_ERR_NONFINITE


@pytest.mark.parametrize("precision,krylov,nu_coarse", [(0, 0, (0, 0)), (1, 0, (0, 0)), (1, 4, (0, 0)),
                                                      (0, 0, (1, 1)), (1, 4, (1, 1)), (2, 4, (1, 0))])
def test_relaxed_sweeps_reach_the_same_solution(ohm, orc, precision, krylov, nu_coarse):
    """omega = 1.25 and other sweep counts on the coarser grids change the multigrid iterates,
    not the converged solution: the step reaches the oracle's converged Gauss-Seidel V(2,2)
    solution (float64: 1e-11, both sides at 1e-13; mixed: 1e-9)."""
    h = HIERS["amr_3level"]()
    b, eta = rand_fields(h, 21, 1.0)
    o = orc.Oracle(h, 0.5, eta)
    b = o.sync_down(b)
    dt = 4.0 * h.dx(h.nlevels - 1) ** 2
    want, _ = o.cn_step(b, dt, 1e-14, 2, 2, 8, 80)
    g = make(ohm, h, precision=precision, max_outer=80, krylov=krylov, omega=1.25, nu_coarse=nu_coarse)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, 1e-13 if precision == 0 else 1e-11)
    assert st["converged"]
    assert rel_err(host(B), want.ravel()) < (1e-11 if precision == 0 else 1e-9)


@pytest.mark.parametrize("precision", [0, 1])
def test_set_eta_again_same_and_changed_values(ohm, precision):
    """Setting eta values that are already set keeps the derived data; changing a single value
    (in another buffer) re-derives everything: each step gives the bits of a fresh hierarchy
    set once with that eta."""
    h = HIERS["amr_2level"]()
    b, eta = rand_fields(h, 31, 1.0)
    eta2 = eta.copy()
    eta2[h.nblocks // 2, 0, 3, 4, 5] *= 1.5
    dt = 3.0 * h.dx(h.nlevels - 1) ** 2

    def fresh(e):
        g = make(ohm, h, precision=precision, max_outer=60)
        B = dev(b)
        ohm.ohm_cn_step(g, B, dev(e), dt, 1e-10)
        return host(B)

    g = make(ohm, h, precision=precision, max_outer=60)
    out = []
    for e in (eta, eta.copy(), eta2, eta2.copy()):
        B = dev(b)
        ohm.ohm_cn_step(g, B, dev(e), dt, 1e-10)
        out.append(host(B))
    want1, want2 = fresh(eta), fresh(eta2)
    assert np.array_equal(out[0], want1) and np.array_equal(out[1], want1)
    assert np.array_equal(out[2], want2) and np.array_equal(out[3], want2)
    assert not np.array_equal(want1, want2)


def test_fgmres_takes_fewer_cycles_than_defect_correction(ohm):
    """Same converged tolerance, fewer V-cycles with the Krylov-accelerated inner solve on a
    stiff case (3-decade eta, dt = 100x the explicit limit)."""
    wl = W.resistive_bump_256(n=32)
    counts = {}
    for krylov in (0, 6):
        g = make(ohm, wl.hier, precision=1, max_outer=200, krylov=krylov)
        B = dev(wl.B)
        st = ohm.ohm_cn_step(g, B, dev(wl.eta), wl.dt, 1e-9)
        assert st["converged"]
        counts[krylov] = st["cycles"]
    assert counts[6] < counts[0]


# ------------------------------------------------------------------ edge cases
def test_single_block_grid(ohm, orc):
    """8^3: one block whose neighbours are all itself (periodic)."""
    h = W.uniform(8, 8, 8, 0.125)
    b, eta = rand_fields(h, 9, 1.0)
    dt = 0.05
    g = make(ohm, h, max_outer=3)
    B = dev(b)
    ohm.ohm_cn_step(g, B, dev(eta), dt, -1.0)
    want, _ = orc.Oracle(h, 0.5, eta).cn_step(b, dt, -1.0, 2, 2, 8, 3)
    assert rel_err(host(B), want.ravel()) < TOL64


def test_zero_field_stays_zero_and_not_converged_status(ohm, orc):
    h = W.uniform(16, 16, 16, 1.0 / 16)
    _, eta = rand_fields(h, 10)
    g = make(ohm, h, max_outer=1)
    B = torch.zeros(h.nblocks * 1536, dtype=torch.float64, device="cuda")
    st = ohm.ohm_cn_step(g, B, dev(eta), 0.01, 1e-9)
    assert float(B.abs().max()) == 0.0
    b, _ = rand_fields(h, 11)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, None, 1.0, 1e-14)
    assert st["status"] == ohm.OHM_ERR_NOT_CONVERGED and not st["converged"] and st["cycles"] == 1


def test_invalid_calls(ohm):
    h = W.uniform(16, 16, 16, 1.0 / 16)
    with pytest.raises(ohm.OhmError):
        make(ohm, h, krylov=4, n_instances=2)  # float64 FGMRES: single problems only
    g = make(ohm, h)
    B = torch.zeros(h.nblocks * 1536, dtype=torch.float64, device="cuda")
    with pytest.raises(ohm.OhmError) as ei:
        ohm.ohm_cn_step(g, B, None, 0.1, 1e-9)  # eta never set
    assert ei.value.status == ohm.OHM_ERR_INVALID
    with pytest.raises(ohm.OhmError):
        ohm.ohm_cn_step(g, B, torch.ones(h.nblocks * 512, dtype=torch.float64, device="cuda"), -1.0, 1e-9)
    with pytest.raises(ohm.OhmError):
        ohm.ohm_residual_norm(g, B)  # no step yet


def test_nonfinite_eta_reports_nonfinite(ohm):
    h = W.uniform(16, 16, 16, 1.0 / 16)
    g = make(ohm, h, max_outer=3)
    eta = torch.ones(h.nblocks * 512, dtype=torch.float64, device="cuda")
    eta[100] = float("nan")
    b, _ = rand_fields(h, 12)
    with pytest.raises(ohm.OhmError) as ei:
        ohm.ohm_cn_step(g, dev(b), eta, 0.01, 1e-9)
    assert ei.value.status == ohm.OHM_ERR_NONFINITE


@pytest.mark.parametrize("precision", [0, 1])
def test_vanishing_dt_leaves_the_field_and_takes_no_cycle(ohm, orc, precision):
    """dt -> 0: L = I and S = b, so the first residual is already below tolerance (Eqs. 13-14):
    B is returned as b (after syncing covered cells) with zero V-cycles."""
    h = amr_two_level(16)
    b, eta = rand_fields(h, 13, 2.0)
    b = orc.Oracle(h, 0.5, eta).sync_down(b)
    g = make(ohm, h, precision=precision, max_outer=5)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), 1e-14 * h.dx(1) ** 2, 1e-9)
    assert st["converged"] and st["cycles"] == 0
    assert rel_err(host(B), b.ravel()) < 1e-12


@pytest.mark.parametrize("precision,krylov,stiff", [(0, 0, 1e3), (1, 6, 1e3), (1, 6, 1e4)])
def test_very_stiff_step_converges_to_the_oracle(ohm, orc, precision, krylov, stiff):
    """dt = 1e3 and 1e4 times the explicit limit with two decades of eta per cell: the step
    converges (the paper's defect correction takes ~125 V-cycles at 1e3 -- the oracle's count --
    and is left to FGMRES at 1e4, where it needs more than 400), and its float64 residual
    evaluated by the oracle meets the tolerance."""
    h = W.uniform(32, 32, 32, 1.0 / 32)
    b, eta = rand_fields(h, 14, 2.0)
    dt = stiff * h.dx0 ** 2 / (6.0 * float(eta.max()))
    o = orc.Oracle(h, 0.5, eta)
    g = make(ohm, h, precision=precision, krylov=krylov, max_outer=400)
    B = dev(b)
    st = ohm.ohm_cn_step(g, B, dev(eta), dt, 1e-9)
    assert st["converged"]
    _, n = o.residual(host(B).reshape(b.shape), o.source(b, dt), dt)
    assert n["rel_l2"] <= 1.05e-9


def test_fp64_fma_rate_probe(ohm):
    """The float64 FMA-rate probe returns a rate between 10 G and 100 T FMA/s on any GPU this
    library runs on (the roofline denominator of the float64 kernels)."""
    r = ohm.ohm_fp64_fma_rate()
    assert 1e10 < r < 1e14
