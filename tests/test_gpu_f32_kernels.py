"""Kernel-level parity of the float32 inner-solve kernels with the FP64 oracle.

Each test hands the same float32-representable inputs to one float32 kernel (through the
row-level entry points of include/ohm.h, which launch exactly what the V-cycle launches on
that grid) and to the oracle's FP64 restatement of the step, and compares element by element:

* the fused red+black sweep on block pairs (`k_smooth_rb2`), from a previous iterate and from
  zero (its zero-start variant), against two oracle colour passes (Sec. 2.3, Eq. 19) relaxed as
  e + omega (e_GS - e);
* the same sweep on single blocks (`k_smooth_rb`, a grid whose blocks do not pair along x) and
  as two colour passes (`k_smooth<float>`);
* residual + restriction into a blocked coarse grid (`k_pair_op` on block pairs, with the fine
  residual and, as the V-cycle runs it, without: octet means from the octets' outer faces) and
  into a lexicographic one (`k_resid_restrict<float>`), and prolongation (`k_prolong_add8<float>`,
  `k_prolong_add<float>`), Sec. 2.2;
* the float32 operator L X on a uniform hierarchy (`k_pair_op`) and on a 3-level AMR hierarchy
  (`k_composite<float,float>`, with coarse-fine ghosts and refluxing);
* the coarsest-grid solve (`k_bottom_sm`, with the grid-wide steps before it where a grid is
  large) against the same V-cycle composed from the oracle's grid passes.

Tolerance.  Inputs are O(1) normal fields and eta = 10^U(-0.5, 0.5) per cell, dt = 5 h^2 (so
1 + alpha is about 10-30).  Both sides start from the same float32 values; the oracle works in
float64, so the difference is the kernel's float32 rounding alone.  An update sums about 30
rounded terms (u = 2^-24 each) whose magnitudes are within a few times (1 + alpha) |result|, and
the division by 1 + alpha brings their rounding back to a few u of the result; the black pass
inherits the red pass's errors with a gain of order one.  Measured on GB300: at most 3.5 u in
relative L2 (2.1e-7) and 34 u (2.0e-6 x rms) in the worst element.  The tests hold the relative
L2 error to TOL32 = 2e-6 (34 u) and the worst element to 10 TOL32 x rms: ten times what the
kernels show, and far below what a dropped flux term or a wrong sign produces (>= 1e-3).
Transfers (sums of 8 positive weights, no cancellation) are held to 8 u of the inputs' scale.
"""
import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W
from tests.helpers import amr_three_level, dense_of_grid, grid_of_dense, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 2e-6
U32 = 2.0 ** -24


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


def f32(a):
    """float32 copy on the device and the same values in float64 on the host."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    return torch.from_numpy(a32).cuda(), a32.astype(np.float64)


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy().astype(np.float64)


def mixed(ohm, h, omega=0.0):
    return ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=0.5, precision=ohm.OHM_MIXED, nu_pre=2,
                                    nu_post=2, n_coarse=4, max_outer=10, krylov=0, omega=omega)


def grid_inputs(dims, seed):
    rng = np.random.default_rng(seed)
    e = rng.standard_normal((3,) + dims[::-1])
    r = rng.standard_normal((3,) + dims[::-1])
    eta = 10 ** rng.uniform(-0.5, 0.5, (1,) + dims[::-1])
    # round to float32 once so that both sides see identical values
    return (e.astype(np.float32).astype(np.float64), r.astype(np.float32).astype(np.float64),
            eta.astype(np.float32).astype(np.float64))


def last_blocked(ohm, g):
    m = 0
    while ohm.ohm_mg_grid_info(g, m + 1)[1] > 0:
        m += 1
    return m


def check32(got, want, what):
    err = rel_err(got, want)
    rms = np.sqrt(np.mean(want ** 2))
    worst = np.abs(got - want).max() / rms
    print(f"{what}: rel L2 {err:.2e}, worst {worst:.2e} x rms")
    assert err < TOL32, what
    assert worst < 10 * TOL32, what


def oracle_sweep(o, m, e, r, eta, dt, omega):
    """Red colour pass then black, each relaxed: e + omega (e_GS - e)."""
    for colour in (0, 1):
        gs = o.grid_smooth(m, e, r, eta, dt, colour)
        e = e + omega * (gs - e)
    return e


SWEEP_GRIDS = {
    # 64 x 32 x 32, Morton blocks: level 0 and grid 1 pair along x (k_smooth_rb2)
    "pairs_m0": ((64, 32, 32), 0),
    "pairs_m1": ((64, 32, 32), 1),
    # 24 x 16 x 16: 3 blocks along x, the pairs (2q, 2q+1) are not x-neighbours (k_smooth_rb)
    "single_m0": ((24, 16, 16), 0),
    # a larger grid: 512 blocks, 6 blocks along z (k_smooth_rb2)
    "pairs_large": ((128, 64, 48), 0),
}


@pytest.mark.parametrize("grid", list(SWEEP_GRIDS))
@pytest.mark.parametrize("start", ["iterate", "zero"])
@pytest.mark.parametrize("omega", [1.0, 1.2])
@pytest.mark.parametrize("variant", [0, 1])
def test_float32_sweep_matches_two_oracle_colour_passes(ohm, orc, grid, start, omega, variant):
    base, m = SWEEP_GRIDS[grid]
    h = W.uniform(*base, 1.0 / base[0])
    o = orc.Oracle(h, 0.5)
    g = mixed(ohm, h, omega)
    dims, nb, ijk = ohm.ohm_mg_grid_info(g, m)
    e, r, eta = grid_inputs(dims, 40 + m + 3 * variant)
    if start == "zero":
        e = np.zeros_like(e)
    dt = 5.0 * h.dx0 ** 2
    r_d, _ = f32(grid_of_dense(r, ijk))
    eta_d, _ = f32(grid_of_dense(eta, ijk))
    e_in = None if start == "zero" else f32(grid_of_dense(e, ijk))[0]
    out = torch.full((nb * 1536,), float("nan"), dtype=torch.float32, device="cuda")
    ohm.ohm_op_grid_sweep_f32(g, m, e_in, out, r_d, eta_d, dt, variant)
    got = dense_of_grid(host(out).reshape(nb, 3, 8, 8, 8), ijk, dims, 3)
    want = oracle_sweep(o, m, e, r, eta, dt, omega)
    check32(got, want, f"sweep {grid} {start} omega={omega} variant={variant}")


@pytest.mark.parametrize("to_lex", [False, True])
def test_float32_residual_restriction_and_prolongation(ohm, orc, to_lex):
    h = W.uniform(64, 32, 32, 1.0 / 64)
    o = orc.Oracle(h, 0.5)
    g = mixed(ohm, h)
    m = last_blocked(ohm, g) if to_lex else 0
    dims, nb, ijk = ohm.ohm_mg_grid_info(g, m)
    cdims, cnb, cijk = ohm.ohm_mg_grid_info(g, m + 1)
    assert (cnb == 0) == to_lex
    e, r, eta = grid_inputs(dims, 50 + m)
    dt = 5.0 * h.dx0 ** 2
    e_d, _ = f32(grid_of_dense(e, ijk))
    r_d, _ = f32(grid_of_dense(r, ijk))
    eta_d, _ = f32(grid_of_dense(eta, ijk))
    t = torch.full((nb * 1536,), float("nan"), dtype=torch.float32, device="cuda")
    ncoarse = 3 * cdims[0] * cdims[1] * cdims[2]
    c = torch.full((ncoarse,), float("nan"), dtype=torch.float32, device="cuda")
    ohm.ohm_op_grid_resid_restrict_f32(g, m, e_d, r_d, eta_d, dt, t, c)
    t_want = o.grid_residual(m, e, r, eta, dt)
    check32(dense_of_grid(host(t).reshape(nb, 3, 8, 8, 8), ijk, dims, 3), t_want, f"residual m={m}")
    c_got = host(c).reshape((3,) + cdims[::-1]) if to_lex else \
        dense_of_grid(host(c).reshape(cnb, 3, 8, 8, 8), cijk, cdims, 3)
    check32(c_got, o.grid_restrict(m, t_want, 3), f"restriction m={m}")
    # prolongation of a float32 coarse field into a float32 fine field
    rng = np.random.default_rng(60 + m)
    cf = rng.standard_normal((3,) + cdims[::-1]).astype(np.float32).astype(np.float64)
    ff = rng.standard_normal((3,) + dims[::-1]).astype(np.float32).astype(np.float64)
    c_dev = f32(cf.ravel() if to_lex else grid_of_dense(cf, cijk))[0]
    f_dev = f32(grid_of_dense(ff, ijk))[0]
    ohm.ohm_op_grid_prolong_add_f32(g, m, c_dev, f_dev)
    got = dense_of_grid(host(f_dev).reshape(nb, 3, 8, 8, 8), ijk, dims, 3)
    want = o.grid_prolong_add(m, cf, ff)
    scale = np.abs(cf).max() + np.abs(ff).max()
    print(f"prolongation m={m}: worst {np.abs(got - want).max() / scale:.2e} of scale")
    assert np.abs(got - want).max() <= 8 * U32 * scale


@pytest.mark.parametrize("base", [(64, 32, 32), (128, 64, 48)])
def test_float32_restricted_residual_without_fine_output(ohm, orc, base):
    """Residual + restriction as the V-cycle launches it, with no fine residual requested: on
    block pairs each octet's mean is formed from the fluxes through the octet's outer faces (the
    fluxes through its inner faces cancel in the conservative form).  The coarse values must
    equal the oracle's restriction of its residual (Sec. 2.2, Eq. 20)."""
    h = W.uniform(*base, 1.0 / base[0])
    o = orc.Oracle(h, 0.5)
    g = mixed(ohm, h)
    dims, nb, ijk = ohm.ohm_mg_grid_info(g, 0)
    cdims, cnb, cijk = ohm.ohm_mg_grid_info(g, 1)
    assert cnb > 0
    e, r, eta = grid_inputs(dims, 55)
    dt = 5.0 * h.dx0 ** 2
    e_d, _ = f32(grid_of_dense(e, ijk))
    r_d, _ = f32(grid_of_dense(r, ijk))
    eta_d, _ = f32(grid_of_dense(eta, ijk))
    c = torch.full((cnb * 1536,), float("nan"), dtype=torch.float32, device="cuda")
    ohm.ohm_op_grid_resid_restrict_f32(g, 0, e_d, r_d, eta_d, dt, None, c)
    want = o.grid_restrict(0, o.grid_residual(0, e, r, eta, dt), 3)
    check32(dense_of_grid(host(c).reshape(cnb, 3, 8, 8, 8), cijk, cdims, 3), want, f"octet restriction {base}")


@pytest.mark.parametrize("name", ["uniform_32", "amr_3level"])
def test_float32_operator_matches_oracle(ohm, orc, name):
    h = W.uniform(32, 32, 32, 1.0 / 32) if name == "uniform_32" else amr_three_level(16)
    rng = np.random.default_rng(70)
    X = rng.standard_normal((h.nblocks, 3, 8, 8, 8)).astype(np.float32).astype(np.float64)
    eta = (10 ** rng.uniform(-0.5, 0.5, (h.nblocks, 1, 8, 8, 8))).astype(np.float32).astype(np.float64)
    dt = 5.0 * h.dx(h.nlevels - 1) ** 2
    o = orc.Oracle(h, 0.5, eta)
    g = mixed(ohm, h)
    ohm.ohm_set_eta(g, torch.from_numpy(eta).cuda())
    out = torch.full((h.nblocks * 1536,), float("nan"), dtype=torch.float32, device="cuda")
    ohm.ohm_op_apply_L_f32(g, f32(X)[0], dt, out)
    got = host(out).reshape(X.shape)
    want = o.apply_L(X, dt)
    leaf = h.is_leaf()
    assert np.all(got[~leaf] == 0.0)
    check32(got[leaf], want[leaf], f"operator {name}")


def oracle_coarse_vcycle(o, m0, r, eta0, dt, nu1, nu2, nc, omega):
    """The V-cycle of the coarsest-grid solver over oracle grids m0 .. n_mg - 1 (Sec. 2.2):
    from e = 0, nu1 relaxed red-black sweeps, residual restricted to the next grid, nc sweeps on
    the coarsest, trilinear prolongation and nu2 sweeps on the way up; eta of each coarser grid
    the mean of its 8 children."""
    last = o.n_mg - 1
    etas = {m0: eta0}
    for m in range(m0, last):
        etas[m + 1] = o.grid_restrict(m, etas[m], 1)
    es, rs = {}, {m0: r}
    for m in range(m0, last):
        e = np.zeros_like(rs[m])
        for _ in range(nu1):
            e = oracle_sweep(o, m, e, rs[m], etas[m], dt, omega)
        es[m] = e
        rs[m + 1] = o.grid_restrict(m, o.grid_residual(m, e, rs[m], etas[m], dt), 3)
    e = np.zeros_like(rs[last])
    for _ in range(nc):
        e = oracle_sweep(o, last, e, rs[last], etas[last], dt, omega)
    for m in range(last - 1, m0 - 1, -1):
        e = o.grid_prolong_add(m, e, es[m])
        for _ in range(nu2):
            e = oracle_sweep(o, m, e, rs[m], etas[m], dt, omega)
    return e


# 32^3: power-of-two grids 16^3 .. 2^3 in the shared-memory solver; 48 x 24 x 24: 24 x 12 x 12,
# 12 x 6 x 6 and 6 x 3 x 3 (other extents); 56^3: 28^3 stepped grid-wide (more than 16384 cells),
# then 14^3 and 7^3 in shared memory
COARSE_BASES = [(32, 32, 32), (48, 24, 24), (56, 56, 56)]


@pytest.mark.parametrize("base", COARSE_BASES)
@pytest.mark.parametrize("omega", [1.0, 1.2])
def test_float32_coarsest_grid_solve_matches_oracle_vcycle(ohm, orc, base, omega):
    """`ohm_op_coarsest_f32` (the coarsest-grid solver of the float32 inner solve, V(2,2) with 4
    coarsest sweeps here) against the same V-cycle composed from the oracle's grid passes, at the
    single-pass tolerance (measured: about 5e-8 relative L2, 4e-7 x rms in the worst element)."""
    h = W.uniform(*base, 1.0 / base[0])
    o = orc.Oracle(h, 0.5)
    g = mixed(ohm, h, omega)
    m0 = last_blocked(ohm, g) + 1
    dims, nb, _ = ohm.ohm_mg_grid_info(g, m0)
    assert nb == 0
    _, r, eta = grid_inputs(dims, 90 + base[1])
    dt = 5.0 * h.dx0 ** 2
    e = torch.full((3 * dims[0] * dims[1] * dims[2],), float("nan"), dtype=torch.float32, device="cuda")
    ohm.ohm_op_coarsest_f32(g, f32(r)[0], f32(eta)[0], dt, e)
    got = host(e).reshape(r.shape)
    want = oracle_coarse_vcycle(o, m0, r, eta[0], dt, 2, 2, 4, omega if omega else 1.0)
    check32(got, want, f"coarsest solve {base} omega={omega}: grid {dims}")
