"""The seeded input generators (shared by the CUDA path and the oracle, no solver arithmetic)
produce what their recipes state: divergence-free fields of the requested rms, the resistivity
ranges and time steps of the configurations, reproducible seeds, block layouts that round-trip.
CPU only."""
import math

import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W


def d0_div(B, dx):
    """Central-difference divergence of a dense periodic [3][z][y][x] field."""
    def d0(f, axis):
        return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2.0 * dx)
    return d0(B[0], 2) + d0(B[1], 1) + d0(B[2], 0)


def test_random_potential_field_is_solenoidal_with_requested_rms():
    n, dx = 16, 1.0 / 16
    B = W.random_potential_field((n, n, n), dx, seed=5, rms=0.7)
    rms = math.sqrt(float(np.mean(np.sum(B * B, axis=0))))
    assert rms == pytest.approx(0.7, rel=1e-12)
    # the central-difference curl has zero central-difference divergence (the difference
    # operators commute on a periodic grid)
    assert np.abs(d0_div(B, dx)).max() < 1e-12 * np.abs(B).max() / dx
    again = W.random_potential_field((n, n, n), dx, seed=5, rms=0.7)
    other = W.random_potential_field((n, n, n), dx, seed=6, rms=0.7)
    assert np.array_equal(B, again) and not np.array_equal(B, other)


def test_resistive_bump_recipe():
    n = 32
    wl = W.resistive_bump_256(n)
    eta = W.blocks_to_dense(wl.hier, wl.eta)[0]
    dx = 1.0 / n
    # eta = 1e-3 (1 + 999 exp(-|x-c|^2/0.05^2)): three decades, the peak at the centre cells
    assert eta.min() == pytest.approx(1e-3, rel=1e-9)
    r2 = 3 * (0.5 * dx) ** 2  # the eight cells around the centre
    assert eta.max() == pytest.approx(1e-3 * (1 + 999 * math.exp(-r2 / 0.05 ** 2)), rel=1e-12)
    assert wl.dt == pytest.approx(100.0 * dx * dx / (6.0 * 1.0), rel=1e-12)
    assert wl.steps == 10 and wl.tol == 1e-9
    B = W.blocks_to_dense(wl.hier, wl.B)
    assert math.sqrt(float(np.mean(np.sum(B * B, axis=0)))) == pytest.approx(1.0, rel=1e-12)


def test_periodic_box_recipe():
    wl = W.periodic_box_32()
    n, dx = 32, 1.0 / 32
    B = W.blocks_to_dense(wl.hier, wl.B)
    x = (np.arange(n) + 0.5) * dx
    noise = B.copy()
    noise[1] -= np.sin(2 * np.pi * x)[None, None, :]
    noise[2] -= np.cos(2 * np.pi * x)[None, None, :]
    assert math.sqrt(float(np.mean(np.sum(noise * noise, axis=0)))) == pytest.approx(0.1, rel=1e-9)
    assert np.all(wl.eta == 1.0)
    assert wl.dt == pytest.approx(10.0 * dx * dx / 6.0) and wl.steps == 20 and wl.tol == 1e-10


def test_blocks_round_trip_and_morton_layout():
    h = W.uniform(32, 16, 24, 1.0 / 32)
    rng = np.random.default_rng(3)
    dense = rng.standard_normal((3, 24, 16, 32))
    blk = W.dense_to_blocks(h, dense)
    assert blk.shape == (h.nblocks, 3, 8, 8, 8)
    assert np.array_equal(W.blocks_to_dense(h, blk), dense)
    # block b holds the 8^3 cells at its (bi, bj, bk)
    lv, bi, bj, bk = h.blocks[5]
    assert np.array_equal(blk[5, 2], dense[2, 8 * bk:8 * bk + 8, 8 * bj:8 * bj + 8, 8 * bi:8 * bi + 8])


def test_smooth_lognormal_eta_spans_two_decades():
    eta = W.smooth_lognormal_eta(16, seed=9)[0]
    assert eta.min() == pytest.approx(1e-3, rel=1e-12)
    assert eta.max() == pytest.approx(1e-1, rel=1e-12)
    # smooth: neighbouring cells differ far less than the full range (sigma = 2 cells)
    step = np.abs(np.diff(np.log10(eta), axis=2)).max()
    assert step < 0.5


def test_batched_instances_recipe_and_prefix_reproducibility():
    inst = W.batched_instances(count=40, seed=4)
    assert {i.n for i in inst} <= set(W.BATCH_EDGES)
    for i in inst[:6]:
        eta = W.blocks_to_dense(i.hier, i.eta)
        lim = (1.0 / i.n) ** 2 / (6.0 * float(eta.max()))
        assert 10.0 * lim * (1 - 1e-12) <= i.dt <= 100.0 * lim * (1 + 1e-12)
        B = W.blocks_to_dense(i.hier, i.B)
        assert np.abs(d0_div(B, 1.0 / i.n)).max() < 1e-10 * np.abs(B).max() * i.n
    # instance q depends on (seed, q) only: a shorter list gives the same first instances
    short = W.batched_instances(count=5, seed=4)
    for a, b in zip(short, inst[:5]):
        assert a.n == b.n and a.dt == b.dt and np.array_equal(a.B, b.B) and np.array_equal(a.eta, b.eta)
