"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's stencil: each compares it with an independent fact --
an exact discrete eigen-decay, the operator's Fourier symbol (derived by hand from
Eqs. 4-11, evaluated with numpy's FFT), the continuous operator curl(eta curl B)
(spectral derivatives), the exact diagonal of the assembled matrix, a dense direct solve,
conservation of sum B dV, and the temporal/spatial orders and printed values of Sec. 3.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def dense_grid(n, dx=None):
    nx, ny, nz = n
    return W.uniform(nx, ny, nz, dx if dx else 1.0 / nx)


def ones_eta(h, v=1.0):
    return np.full((h.nblocks, 1, 8, 8, 8), v)


# --------------------------------------------------------------------------- closed forms
@pytest.mark.parametrize("lam", [0.5, 1.0])
@pytest.mark.parametrize("axis,comp", [(0, 2), (1, 0), (2, 1)])
def test_plane_wave_exact_decay(oracle_mod, lam, axis, comp):
    """A single-direction mode B_c = sin(k x_a) (c != a) under constant eta is an eigenvector
    of the discrete operator with eigenvalue eta s^2, s = 2 sin(k h/2)/h, so one theta-step
    multiplies it by g = (1 - (1-lam) dt eta s^2) / (1 + lam dt eta s^2)  (Eq. 7)."""
    dims = [16, 8, 24]
    h = dense_grid(dims, 1.0 / 16)
    dx = h.dx0
    eta = 0.7
    o = oracle_mod.Oracle(h, lam, ones_eta(h, eta))
    L = dims[axis] * dx
    kk = 2 * math.pi * 2 / L
    coords = [(np.arange(d) + 0.5) * dx for d in dims]
    B = np.zeros((3, dims[2], dims[1], dims[0]))
    shape = [1, 1, 1]
    shape[2 - axis] = dims[axis]
    B[comp] = np.sin(kk * coords[axis]).reshape(shape)
    dt = 7.0 * dx * dx
    Bn, info = o.cn_step(W.dense_to_blocks(h, B), dt, 1e-14, max_outer=60)
    s2 = (2 * math.sin(kk * dx / 2) / dx) ** 2
    g = (1 - (1 - lam) * dt * eta * s2) / (1 + lam * dt * eta * s2)
    got = W.blocks_to_dense(h, Bn)
    assert info["converged"]
    assert np.abs(got - g * B).max() < 1e-13


def symbol_apply(R, dx, eta):
    """eta M(theta) R-hat with M_aa = sum_{c != a} s_c^2 and M_ab = -sigma_a sigma_b, where
    s_c = 2 sin(theta_c/2)/h and sigma_c = sin(theta_c)/h: the Fourier symbol of Eqs. 4-11
    for constant eta (normal differences give s^2, the four-point transverse differences
    combined with the flux divergence give -sigma_a sigma_b)."""
    nz, ny, nx = R.shape[1:]
    tz, ty, tx = np.meshgrid(2 * np.pi * np.fft.fftfreq(nz), 2 * np.pi * np.fft.fftfreq(ny),
                             2 * np.pi * np.fft.fftfreq(nx), indexing="ij")
    th = [tx, ty, tz]
    s = [2 * np.sin(t / 2) / dx for t in th]
    sg = [np.sin(t) / dx for t in th]
    Rh = [np.fft.fftn(R[c]) for c in range(3)]
    out = np.empty_like(R)
    for a in range(3):
        acc = sum(s[c] ** 2 for c in range(3) if c != a) * Rh[a]
        for b in range(3):
            if b != a:
                acc = acc - sg[a] * sg[b] * Rh[b]
        out[a] = eta * np.real(np.fft.ifftn(acc))
    return out


def test_fourier_symbol_constant_eta(oracle_mod):
    dims = [16, 8, 24]
    h = dense_grid(dims, 0.05)
    o = oracle_mod.Oracle(h, 0.5, ones_eta(h, 1.3))
    R = np.random.default_rng(3).standard_normal((3, dims[2], dims[1], dims[0]))
    got = W.blocks_to_dense(h, o.div_flux(W.dense_to_blocks(h, R)))
    want = symbol_apply(R, 0.05, 1.3)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_cn_step_matches_fft_solution(oracle_mod):
    """Constant eta, periodic: the exact discrete CN step is (I + lam dt eta M)^-1 (I - (1-lam) dt eta M)
    applied mode by mode; the oracle's multigrid must reach it."""
    n = 16
    h = dense_grid([n, n, n], 1.0 / n)
    dx, eta, lam = 1.0 / n, 1.0, 0.5
    dt = 10 * dx * dx / 6
    o = oracle_mod.Oracle(h, lam, ones_eta(h, eta))
    B = W.random_potential_field((n, n, n), dx, 11, 0.5)
    Bn, info = o.cn_step(W.dense_to_blocks(h, B), dt, 1e-14, max_outer=60)
    tz, ty, tx = np.meshgrid(*(2 * np.pi * np.fft.fftfreq(n),) * 3, indexing="ij")
    th = [tx, ty, tz]
    s = [2 * np.sin(t / 2) / dx for t in th]
    sg = [np.sin(t) / dx for t in th]
    Bh = np.array([np.fft.fftn(B[c]) for c in range(3)])
    M = np.zeros((3, 3) + Bh.shape[1:], dtype=complex)
    for a in range(3):
        for b in range(3):
            M[a, b] = sum(s[c] ** 2 for c in range(3) if c != a) if a == b else -sg[a] * sg[b]
    Mt = np.moveaxis(M, (0, 1), (-2, -1))
    I = np.eye(3)
    rhs = np.einsum("...ab,b...->...a", I - (1 - lam) * dt * eta * Mt, Bh)
    sol = np.linalg.solve(I + lam * dt * eta * Mt, rhs[..., None])[..., 0]
    want = np.real(np.array([np.fft.ifftn(np.moveaxis(sol, -1, 0)[c]) for c in range(3)]))
    got = W.blocks_to_dense(h, Bn)
    assert info["converged"]
    assert np.abs(got - want).max() < 1e-12 * np.abs(want).max()


def spectral_curl_eta_curl(B, eta, L):
    """curl(eta curl B) for band-limited periodic fields, exact with FFT derivatives."""
    n = B.shape[1]
    k = 2 * np.pi * np.fft.fftfreq(n, d=L / n)
    kz, ky, kx = np.meshgrid(k, k, k, indexing="ij")
    K = [kx, ky, kz]

    def d(f, a):
        return np.real(np.fft.ifftn(1j * K[a] * np.fft.fftn(f)))

    def curl(V):
        return np.array([d(V[2], 1) - d(V[1], 2), d(V[0], 2) - d(V[2], 0), d(V[1], 0) - d(V[0], 1)])

    return curl(eta * curl(B))


def smooth_fields(n, L=1.0):
    x = (np.arange(n) + 0.5) * L / n
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    p = 2 * np.pi / L
    B = np.array([np.sin(p * y) * np.cos(p * z) + 0.3 * np.cos(2 * p * xx),
                  np.cos(p * xx + 0.3) * np.sin(p * z) + 0.2 * np.sin(p * (xx + y)),
                  np.sin(p * (xx - y)) + 0.5 * np.cos(p * z) * np.cos(p * xx)])
    eta = 1.0 + 0.5 * np.sin(p * xx) * np.cos(p * y) + 0.3 * np.cos(p * z)
    return B, eta


def test_variable_eta_second_order_to_continuous_operator(oracle_mod):
    """(div F)(B) of Eqs. 4-11 approximates curl(eta curl B) to second order (Sec. 2.1)."""
    errs = []
    for n in (16, 32):
        h = dense_grid([n, n, n], 1.0 / n)
        B, eta = smooth_fields(n)
        o = oracle_mod.Oracle(h, 0.5, W.dense_to_blocks(h, eta[None]))
        got = W.blocks_to_dense(h, o.div_flux(W.dense_to_blocks(h, B)))
        want = spectral_curl_eta_curl(B, eta, 1.0)
        errs.append(np.abs(got - want).max() / np.abs(want).max())
    assert errs[1] < 0.01
    assert 3.5 < errs[0] / errs[1] < 4.6, errs


def test_alpha_is_exact_diagonal(oracle_mod):
    """1 + alpha_c of Eqs. 21-23 is the diagonal of L: one smoothing pass from e = 0 with a
    unit right-hand side at one cell returns 1 / L_diag there."""
    n = 8
    h = dense_grid([n, n, n], 0.1)
    rng = np.random.default_rng(5)
    eta_d = np.exp(rng.uniform(-2, 2, (1, n, n, n)))
    dt = 0.013
    o = oracle_mod.Oracle(h, 0.5, W.dense_to_blocks(h, eta_d))
    for (i, j, k, c) in [(0, 0, 0, 0), (3, 5, 7, 1), (7, 2, 4, 2), (1, 6, 3, 0)]:
        unit = np.zeros((3, n, n, n))
        unit[c, k, j, i] = 1.0
        diag = W.blocks_to_dense(h, o.apply_L(W.dense_to_blocks(h, unit), dt))[c, k, j, i]
        e = o.grid_smooth(0, np.zeros_like(unit), unit, eta_d, dt, (i + j + k) % 2)
        assert e[c, k, j, i] == pytest.approx(1.0 / diag, rel=1e-14)


def test_colour_pass_is_jacobi_within_colour(oracle_mod):
    """One colour pass: cells of that colour get e + (r - L e)/L_diag from the pre-pass state
    (residual from the independently assembled operator), the other colour is untouched."""
    n = 8
    h = dense_grid([n, n, n], 0.1)
    rng = np.random.default_rng(6)
    eta_d = np.exp(rng.uniform(-1, 1, (1, n, n, n)))
    dt = 0.02
    o = oracle_mod.Oracle(h, 0.5, W.dense_to_blocks(h, eta_d))
    e = rng.standard_normal((3, n, n, n))
    r = rng.standard_normal((3, n, n, n))
    Le = W.blocks_to_dense(h, o.apply_L(W.dense_to_blocks(h, e), dt))
    # diagonal of L from unit responses on combs of stride 4 (stencils of probed cells do not overlap)
    diag = np.empty_like(e)
    for c in range(3):
        for oi in range(4):
            for oj in range(4):
                for ok in range(4):
                    probe = np.zeros_like(e)
                    probe[c, ok::4, oj::4, oi::4] = 1.0
                    resp = W.blocks_to_dense(h, o.apply_L(W.dense_to_blocks(h, probe), dt))
                    diag[c, ok::4, oj::4, oi::4] = resp[c, ok::4, oj::4, oi::4]
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    for colour in (0, 1):
        got = o.grid_smooth(0, e, r, eta_d, dt, colour)
        want = e.copy()
        sel = ((ii + jj + kk) % 2) == colour
        for c in range(3):
            want[c][sel] = e[c][sel] + (r[c][sel] - Le[c][sel]) / diag[c][sel]
        assert np.abs(got - want).max() < 1e-12


# --------------------------------------------------------------------------- conservation
def amr_small(base=(16, 8, 8)):
    nx, ny, nz = base
    return W.refined(nx, ny, nz, 1.0 / nx, [lambda lo, hi: lo[0] < 0.45])


def test_reflux_conserves_flux_on_amr(oracle_mod):
    """Refluxing (Sec. 4): the volume-weighted sum of div F over leaf cells vanishes to
    round-off for any B and eta on an AMR hierarchy."""
    h = amr_small()
    rng = np.random.default_rng(7)
    B = rng.standard_normal((h.nblocks, 3, 8, 8, 8))
    eta = np.exp(rng.uniform(-1, 1, (h.nblocks, 1, 8, 8, 8)))
    o = oracle_mod.Oracle(h, 0.5, eta)
    div = o.div_flux(B)
    leaf = h.is_leaf()
    dv = np.array([h.dx(l) ** 3 for l in h.blocks[:, 0]])
    tot = (div * (dv * leaf)[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))
    scale = (np.abs(div) * (dv * leaf)[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))
    assert np.all(np.abs(tot) < 1e-13 * scale)


@pytest.mark.parametrize("amr", [False, True])
def test_cn_step_conserves_sum_B(oracle_mod, amr):
    h = amr_small() if amr else dense_grid([16, 16, 8], 1.0 / 16)
    rng = np.random.default_rng(8)
    B = rng.standard_normal((h.nblocks, 3, 8, 8, 8))
    eta = np.exp(rng.uniform(-1, 1, (h.nblocks, 1, 8, 8, 8)))
    o = oracle_mod.Oracle(h, 0.5, eta)
    B = o.sync_down(B)
    dx = h.dx(h.nlevels - 1)
    Bn, info = o.cn_step(B, 4 * dx * dx, 1e-13, max_outer=80)
    leaf = h.is_leaf()
    dv = np.array([h.dx(l) ** 3 for l in h.blocks[:, 0]]) * leaf
    s0 = (B * dv[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))
    s1 = (Bn * dv[:, None, None, None, None]).sum(axis=(0, 2, 3, 4))
    assert info["converged"]
    assert np.abs(s1 - s0).max() < 1e-11 * (np.abs(B) * dv[:, None, None, None, None]).sum(axis=(0, 2, 3, 4)).max()


def test_constant_field_is_steady_on_amr(oracle_mod):
    h = amr_small()
    B = np.zeros((h.nblocks, 3, 8, 8, 8))
    B[:, 0], B[:, 1], B[:, 2] = 0.3, -1.2, 2.0
    eta = np.exp(np.random.default_rng(9).uniform(-1, 1, (h.nblocks, 1, 8, 8, 8)))
    o = oracle_mod.Oracle(h, 0.5, eta)
    assert np.abs(o.div_flux(B)).max() < 1e-12


# --------------------------------------------------------------------------- direct solve
def test_multigrid_reaches_dense_lu_solution(oracle_mod):
    """The defect-correction multigrid (Eqs. 16-18) converges to L^-1 S; L assembled column by
    column from unit vectors and solved with LAPACK (8^3 cells, 1536 unknowns)."""
    n = 8
    h = dense_grid([n, n, n], 1.0 / n)
    rng = np.random.default_rng(10)
    eta = np.exp(rng.uniform(-1.5, 1.5, (h.nblocks, 1, 8, 8, 8)))
    dt = 5.0 / n ** 2 / 6.0
    o = oracle_mod.Oracle(h, 0.5, eta)
    N = 3 * n ** 3
    A = np.empty((N, N))
    for col in range(N):
        u = np.zeros(N)
        u[col] = 1.0
        A[:, col] = o.apply_L(u.reshape(1, 3, 8, 8, 8), dt).ravel()
    b = rng.standard_normal((1, 3, 8, 8, 8))
    S = o.source(b, dt)
    want = np.linalg.solve(A, S.ravel())
    got, info = o.cn_step(b, dt, 1e-14, max_outer=60)
    assert info["converged"]
    assert np.abs(got.ravel() - want).max() < 1e-12 * np.abs(want).max()


def test_fully_refined_hierarchy_equals_uniform_fine_grid(oracle_mod):
    """With every base block refined, the composite operator is the uniform operator at the
    fine resolution (no coarse-fine interface is left)."""
    hc = W.refined(16, 16, 16, 1.0 / 16, [lambda lo, hi: True])
    hf = dense_grid([32, 32, 32], 1.0 / 32)
    B, eta = smooth_fields(32)
    rng = np.random.default_rng(12)
    B = B + 0.1 * rng.standard_normal(B.shape)
    fine = hc.blocks[:, 0] == 1
    Bc = np.zeros((hc.nblocks, 3, 8, 8, 8))
    Ec = np.ones((hc.nblocks, 1, 8, 8, 8))
    Bc[fine] = W.dense_to_blocks(hc, B, level=1)
    Ec[fine] = W.dense_to_blocks(hc, eta[None], level=1)
    oc = oracle_mod.Oracle(hc, 0.5, Ec)
    of = oracle_mod.Oracle(hf, 0.5, W.dense_to_blocks(hf, eta[None]))
    dc = W.blocks_to_dense(hc, oc.div_flux(Bc), level=1)
    df = W.blocks_to_dense(hf, of.div_flux(W.dense_to_blocks(hf, B)))
    assert np.abs(dc - df).max() < 1e-12 * np.abs(df).max()


def test_amr_operator_consistent_with_continuous(oracle_mod):
    """On an AMR hierarchy the composite operator still approximates curl(eta curl B): the
    worst leaf-cell error (at the coarse-fine interface, where the quadratic ghost
    interpolation leaves an O(h) truncation error) halves when the hierarchy is refined by 2."""
    p = 2 * np.pi

    def fB(x, y, z):
        return (np.sin(p * y) * np.cos(p * z) + 0.3 * np.cos(2 * p * x),
                np.cos(p * x + 0.3) * np.sin(p * z) + 0.2 * np.sin(p * (x + y)),
                np.sin(p * (x - y)) + 0.5 * np.cos(p * z) * np.cos(p * x))

    def fE(x, y, z):
        return (1.0 + 0.5 * np.sin(p * x) * np.cos(p * y) + 0.3 * np.cos(p * z),)

    errs = []
    for n in (16, 32):
        h = W.refined(n, n, n, 1.0 / n, [lambda lo, hi: lo[0] < 0.45])
        o = oracle_mod.Oracle(h, 0.5, W.sample_blocks(h, fE, 1))
        got = o.div_flux(W.sample_blocks(h, fB, 3))
        refs = []
        for l in (0, 1):
            Bd, etad = smooth_fields(n << l)
            refs.append(spectral_curl_eta_curl(Bd, etad, 1.0))
        err = 0.0
        for b in np.nonzero(h.is_leaf())[0]:
            l, bi, bj, bk = h.blocks[b]
            ref = refs[l][:, bk * 8:(bk + 1) * 8, bj * 8:(bj + 1) * 8, bi * 8:(bi + 1) * 8]
            err = max(err, np.abs(got[b] - ref).max())
        errs.append(err / np.abs(refs[1]).max())
    assert errs[1] < errs[0] / 1.6, errs


# --------------------------------------------------------------------------- Sec. 3 tests
def test_sinusoid_setup_matches_printed_values():
    """Sec. 3.1: exp(-eta |k|^2 t) at t = 4e-3 for k = 2pi(1,2,0) is the printed 0.45, and the
    fine-grid eta dt/dx^2 of Fig. 6 follow from dx_fine = 1/(8N)."""
    k2 = (2 * math.pi) ** 2 * 5
    assert round(math.exp(-k2 * 4e-3), 2) == GOLD["sinusoid_amplitude_t4e-3"]["value"]
    for (dt, N), want in zip(GOLD["sinusoid_eta_dt_over_dx2"]["cases"], GOLD["sinusoid_eta_dt_over_dx2"]["value"]):
        assert dt * (8 * N) ** 2 == pytest.approx(want, rel=0.01)


@pytest.mark.slow
def test_sinusoid_temporal_orders_on_amr(oracle_mod):
    """Sec. 3.1, Fig. 2: on the half-refined AMR grid, lambda = 1/2 is second order and
    lambda = 1 first order in dt (temporal error measured against a dt = 5e-5 run, t = 2e-3)."""
    t_end = 2e-3
    orders = {}
    for lam in (0.5, 1.0):
        sols = {}
        for dt in (4e-4, 2e-4, 5e-5):
            wl = W.sinusoid_half_refined(N=8, lam=lam, dt=dt, t_end=t_end)
            o = oracle_mod.Oracle(wl.hier, lam, wl.eta)
            B = o.sync_down(wl.B)
            for _ in range(wl.steps):
                B, info = o.cn_step(B, dt, 1e-13, nu_pre=4, nu_post=4, max_outer=60)
                assert info["converged"]
            sols[dt] = B
        e1 = np.abs(sols[4e-4] - sols[5e-5]).max()
        e2 = np.abs(sols[2e-4] - sols[5e-5]).max()
        orders[lam] = math.log2(e1 / e2)
    assert orders[0.5] == pytest.approx(GOLD["cn_temporal_order"]["value"], abs=0.25)
    assert orders[1.0] == pytest.approx(GOLD["be_temporal_order"]["value"], abs=0.25)


@pytest.mark.slow
def test_sinusoid_amplitude_and_coarse_fine_errors(oracle_mod):
    """Sec. 3.1: amplitude 0.45 at t = 4e-3, and the CN error on the coarse half exceeds the
    error on the refined half (Fig. 3)."""
    dt = 2e-4
    wl = W.sinusoid_half_refined(N=8, lam=0.5, dt=dt, t_end=4e-3)
    o = oracle_mod.Oracle(wl.hier, 0.5, wl.eta)
    B = o.sync_down(wl.B)
    for _ in range(wl.steps):
        B, info = o.cn_step(B, dt, 1e-13, nu_pre=4, nu_post=4, max_outer=60)
    k = 2 * np.pi * np.array([1.0, 2.0, 0.0])
    decay = math.exp(-float(k @ k) * 4e-3)
    exact = W.sample_blocks(wl.hier, lambda x, y, z: (0 * x, 0 * x, decay * np.sin(k[0] * x + k[1] * y)), 3)
    leaf = wl.hier.is_leaf()
    lev = wl.hier.blocks[:, 0]
    err_f = np.abs(B - exact)[leaf & (lev == 1)][:, 2].mean()
    err_c = np.abs(B - exact)[leaf & (lev == 0)][:, 2].mean()
    assert round(np.abs(B[leaf][:, 2]).max() / 1.0, 2) == pytest.approx(GOLD["sinusoid_amplitude_t4e-3"]["value"], abs=0.02)
    assert err_c > 1.5 * err_f


@pytest.mark.slow
def test_implicit_agrees_with_explicit_at_second_order(oracle_mod):
    """Sec. 3.3 (scaled to 32^3, t = 0.2): eta = exp(-r^2), B_z = exp(-(x^2+y^2)) on [-4,4]^3.
    CN with dt = 0.05 and 0.025 against the explicit predictor-corrector with dt = 1e-3: the
    gap shrinks about 4x when dt halves (second order in time)."""
    n, L = 32, 8.0
    dx = L / n
    h = W.uniform(n, n, n, dx, origin=(-4.0, -4.0, -4.0))
    eta = W.sample_blocks(h, lambda x, y, z: (np.exp(-(x * x + y * y + z * z)),), 1)
    B0 = W.sample_blocks(h, lambda x, y, z: (0 * x, 0 * x, np.exp(-(x * x + y * y))), 3)
    o = oracle_mod.Oracle(h, 0.5, eta)
    t_end = 0.2
    Be = B0.copy()
    for _ in range(200):
        Be = o.heun_step(Be, 1e-3)
    gaps = []
    for dt in (0.05, 0.025):
        B = B0.copy()
        for _ in range(int(round(t_end / dt))):
            B, info = o.cn_step(B, dt, 1e-13, max_outer=60)
            assert info["converged"]
        gaps.append(np.abs(B - Be).max())
    assert gaps[0] / gaps[1] == pytest.approx(4.0, rel=0.25)
    assert gaps[1] < 1e-3 * np.abs(B0).max()


# --------------------------------------------------------------------------- multigrid transfers
# Sec. 2.2 names averaging restriction and full-weight prolongation; these pins hold the
# oracle's two transfers and the coarse-grid eta to properties that fix them: exactness on
# the data each must reproduce, conservation, and commutation with periodic shifts (which
# sends data across the periodic seam).
TDIMS = (32, 16, 24)  # base multigrid grid 0; grid 1 is 16 x 8 x 12


def transfer_oracle(oracle_mod):
    h = dense_grid(list(TDIMS), 0.05)
    return h, oracle_mod.Oracle(h, 0.5)


def centres(dims, dx):
    """Cell-centre coordinates (x, y, z), each of shape [nz][ny][nx]."""
    nx, ny, nz = dims
    z, y, x = np.meshgrid((np.arange(nz) + 0.5) * dx, (np.arange(ny) + 0.5) * dx, (np.arange(nx) + 0.5) * dx,
                          indexing="ij")
    return x, y, z


def test_prolongation_exact_for_linear_fields_away_from_seam(oracle_mod):
    """Trilinear cell-centred interpolation reproduces a field linear in x, y and z exactly at
    every fine cell whose 2x2x2 coarse stencil does not wrap around the periodic box; swapped
    3/4 and 1/4 weights, or a child taking its neighbour on the wrong side, fail this."""
    h, o = transfer_oracle(oracle_mod)
    dx = h.dx0
    cdims = o.mg_dims(1)
    a0, a = 0.7, np.array([1.3, -2.1, 0.45])
    cx = centres(cdims, 2 * dx)
    coarse = np.stack([a0 + c + a[0] * cx[0] + a[1] * cx[1] + a[2] * cx[2] for c in range(3)])
    got = o.grid_prolong_add(0, coarse, np.zeros((3,) + TDIMS[::-1]))
    fx = centres(TDIMS, dx)
    want = np.stack([a0 + c + a[0] * fx[0] + a[1] * fx[1] + a[2] * fx[2] for c in range(3)])
    inner = (slice(None), slice(1, -1), slice(1, -1), slice(1, -1))
    assert np.abs(got[inner] - want[inner]).max() < 1e-13 * np.abs(want).max()
    # a constant coarse field is reproduced everywhere, the seam included
    got_c = o.grid_prolong_add(0, np.full((3,) + cdims[::-1], 2.5), np.zeros((3,) + TDIMS[::-1]))
    assert np.abs(got_c - 2.5).max() < 1e-14


def test_prolongation_adds_and_commutes_with_periodic_shifts(oracle_mod):
    """fine += P coarse (the fine field is added to, not replaced), and P commutes with periodic
    translation: shifting the coarse field by one coarse cell shifts P coarse by two fine cells."""
    h, o = transfer_oracle(oracle_mod)
    rng = np.random.default_rng(31)
    cdims = o.mg_dims(1)
    coarse = rng.standard_normal((3,) + cdims[::-1])
    fine = rng.standard_normal((3,) + TDIMS[::-1])
    P0 = o.grid_prolong_add(0, coarse, np.zeros_like(fine))
    assert np.abs(o.grid_prolong_add(0, coarse, fine) - (fine + P0)).max() < 1e-14 * np.abs(fine + P0).max()
    for ax in (1, 2, 3):  # z, y, x of the dense layout
        shifted = o.grid_prolong_add(0, np.roll(coarse, 1, axis=ax), np.zeros_like(fine))
        assert np.abs(shifted - np.roll(P0, 2, axis=ax)).max() < 1e-14 * np.abs(P0).max()


def test_restriction_octet_constant_linear_and_conservative(oracle_mod):
    """Averaging restriction maps a field constant on each 2x2x2 octet to that constant, a
    linear field to its values at the coarse centres, and keeps sum f dV; it commutes with
    periodic shifts (two fine cells = one coarse cell)."""
    h, o = transfer_oracle(oracle_mod)
    dx = h.dx0
    cdims = o.mg_dims(1)
    rng = np.random.default_rng(32)
    c = rng.standard_normal((3,) + cdims[::-1])
    octet = np.repeat(np.repeat(np.repeat(c, 2, axis=1), 2, axis=2), 2, axis=3)
    assert np.abs(o.grid_restrict(0, octet, 3) - c).max() < 1e-15 * np.abs(c).max() + 1e-300
    fx, cx = centres(TDIMS, dx), centres(cdims, 2 * dx)
    lin = 0.3 + 1.7 * fx[0] - 0.6 * fx[1] + 2.2 * fx[2]
    want = 0.3 + 1.7 * cx[0] - 0.6 * cx[1] + 2.2 * cx[2]
    assert np.abs(o.grid_restrict(0, lin[None], 1)[0] - want).max() < 1e-14 * np.abs(want).max()
    f = rng.standard_normal((3,) + TDIMS[::-1])
    R = o.grid_restrict(0, f, 3)
    for comp in range(3):
        assert abs(R[comp].sum() * (2 * dx) ** 3 - f[comp].sum() * dx ** 3) < 1e-13 * np.abs(f[comp]).sum() * dx ** 3
    for ax in (1, 2, 3):
        assert np.abs(o.grid_restrict(0, np.roll(f, 2, axis=ax), 3) - np.roll(R, 1, axis=ax)).max() < 1e-15 * np.abs(R).max()


def test_coarse_grid_eta_is_mean_of_children(oracle_mod):
    """The multigrid eta (Sec. 2.2 coarse operator reading): on every coarser grid it equals the
    mean of the fine cells it covers.  Checked on eta constant on each 2^m cube (grid m then holds
    exactly those constants) and on a positive linear eta (reproduced at the coarse centres)."""
    h = dense_grid(list(TDIMS), 0.05)
    o = oracle_mod.Oracle(h, 0.5)
    nmg = o.n_mg
    assert nmg >= 3
    rng = np.random.default_rng(33)
    d2 = o.mg_dims(2)
    vals = 10 ** rng.uniform(-1, 1, d2[::-1])
    eta = np.repeat(np.repeat(np.repeat(vals, 4, axis=0), 4, axis=1), 4, axis=2)
    o.set_eta(W.dense_to_blocks(h, eta[None]))
    assert np.array_equal(o.mg_eta(0), eta)
    assert np.abs(o.mg_eta(2) - vals).max() <= 1e-15 * vals.max()
    assert np.abs(o.mg_eta(1) - np.repeat(np.repeat(np.repeat(vals, 2, axis=0), 2, axis=1), 2, axis=2)).max() <= 1e-15 * vals.max()
    fx = centres(TDIMS, h.dx0)
    lin = 2.0 + fx[0] + 0.5 * fx[1] + 0.25 * fx[2]
    o.set_eta(W.dense_to_blocks(h, lin[None]))
    for m in range(1, nmg):
        cx = centres(o.mg_dims(m), h.dx0 * 2 ** m)
        want = 2.0 + cx[0] + 0.5 * cx[1] + 0.25 * cx[2]
        assert np.abs(o.mg_eta(m) - want).max() < 1e-14 * want.max()


def test_residual_norms_are_leaf_only_and_volume_weighted(oracle_mod):
    """The stopping norm (Sec. 3.1 uses max |R|; the solver also reports the volume-weighted
    L2 ratio): on a 3-level hierarchy, ||R||^2 = sum over leaf cells of R^2 h_l^3, likewise
    ||S||, and max |R| over leaf cells, with S made nonzero and large on covered blocks (which
    must not count) and scaled per level (so a missing volume weight changes the ratio)."""
    c = np.array([0.5, 0.5, 0.5])

    def sphere(r):
        return lambda lo, hi: float(np.sum((np.clip(c, lo, hi) - c) ** 2)) < r * r

    h = W.refined(16, 16, 16, 1.0 / 16, [sphere(0.3), sphere(0.12)])
    assert h.nlevels == 3
    rng = np.random.default_rng(34)
    B = rng.standard_normal((h.nblocks, 3, 8, 8, 8))
    S = rng.standard_normal((h.nblocks, 3, 8, 8, 8)) * (1.0 + 3.0 * h.blocks[:, 0])[:, None, None, None, None]
    leaf = h.is_leaf()
    S[~leaf] *= 1e3
    eta = np.exp(rng.uniform(-1, 1, (h.nblocks, 1, 8, 8, 8)))
    o = oracle_mod.Oracle(h, 0.5, eta)
    dt = 2.0 * h.dx(2) ** 2
    R, n = o.residual(B, S, dt)
    assert np.all(R[~leaf] == 0.0)
    dv = np.array([h.dx(l) ** 3 for l in h.blocks[:, 0]])[leaf]
    sr = float((R[leaf] ** 2).sum(axis=(1, 2, 3, 4)) @ dv)
    ss = float((S[leaf] ** 2).sum(axis=(1, 2, 3, 4)) @ dv)
    assert n["l2_R"] == pytest.approx(math.sqrt(sr), rel=1e-13)
    assert n["l2_S"] == pytest.approx(math.sqrt(ss), rel=1e-13)
    assert n["rel_l2"] == pytest.approx(math.sqrt(sr / ss), rel=1e-13)
    assert n["max_abs"] == np.abs(R[leaf]).max()
    # R itself on leaf cells is S - B - lambda dt div F(B) with the oracle's own flux divergence
    # (pinned above by the Fourier symbol, refluxing and the continuous operator)
    div = o.div_flux(o.sync_down(B))
    assert np.abs(R[leaf] - (S - B - 0.5 * dt * div)[leaf]).max() < 1e-12 * np.abs(S[leaf]).max()
