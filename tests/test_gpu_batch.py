"""Batched hierarchies (n_instances = K): K independent instances of one block structure,
stepped together by ohm_cn_step_batch, each instance against the FP64 oracle run on that
instance alone with its own eta and dt.

Tolerances: FP64 fixed schedules 1e-12 relative L2 (the batch folds dt into eta, so it differs
from the oracle in rounding only); mixed precision 1e-9 after refinement to 1e-11.  An instance
must give the same bits alone (K = 1) as in a batch, with or without CUDA graphs.
"""
import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W
from tests.helpers import amr_two_level, rand_fields, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def level_ranges(h):
    lv = h.blocks[:, 0]
    return [(int(np.searchsorted(lv, l, "left")), int(np.searchsorted(lv, l, "right"))) for l in range(h.nlevels)]


def stack(h, per_instance):
    """Batch layout: level by level, the instances' blocks of that level one after another."""
    parts = []
    for lo, hi in level_ranges(h):
        for a in per_instance:
            parts.append(a[lo:hi])
    return np.concatenate(parts)


def unstack(h, arr, K):
    out = [[] for _ in range(K)]
    pos = 0
    for lo, hi in level_ranges(h):
        n = hi - lo
        for q in range(K):
            out[q].append(arr[pos:pos + n])
            pos += n
    return [np.concatenate(o) for o in out]


def make(ohm, h, K, precision=0, stream=None, **kw):
    p = dict(nu_pre=2, nu_post=2, n_coarse=8, max_outer=60)
    p.update(kw)
    return ohm.ohm_create_hierarchy(h.base_cells, h.dx0, h.blocks, lam=0.5, precision=precision, n_instances=K,
                                    stream=stream, **p)


def instances(h, K, seed0):
    bs, etas = [], []
    for q in range(K):
        b, eta = rand_fields(h, seed0 + q, 1.0)
        bs.append(b)
        etas.append(eta)
    return bs, etas


@pytest.mark.parametrize("name", ["uniform_16", "amr_2level"])
def test_fp64_batch_fixed_schedule_matches_oracle(ohm, orc, name):
    """Every launch covers all instances; each instance equals its own oracle run (Eqs. 16-18,
    3 V-cycles), with its own eta and dt."""
    h = W.uniform(16, 16, 16, 1.0 / 16) if name == "uniform_16" else amr_two_level(16)
    K = 3
    bs, etas = instances(h, K, 40)
    dts = [(2.0 + 3.0 * q) * h.dx(h.nlevels - 1) ** 2 for q in range(K)]
    bs = [orc.Oracle(h, 0.5, etas[q]).sync_down(bs[q]) for q in range(K)]
    g = make(ohm, h, K, max_outer=3)
    ohm.ohm_set_eta(g, dev(stack(h, etas)))
    B = dev(stack(h, bs))
    status, st = ohm.ohm_cn_step_batch(g, B, dts, -1.0)
    got = unstack(h, host(B).reshape(-1, 1536), K)
    for q in range(K):
        want, _ = orc.Oracle(h, 0.5, etas[q]).cn_step(bs[q], dts[q], -1.0, 2, 2, 8, 3)
        assert st[q]["cycles"] == 3
        assert rel_err(got[q], want.reshape(-1, 1536)) < 1e-12, q


@pytest.mark.parametrize("name", ["uniform_16", "amr_2level"])
@pytest.mark.parametrize("precision", [1, 2])
def test_mixed_batch_converges_to_oracle(ohm, orc, name, precision):
    h = W.uniform(16, 16, 16, 1.0 / 16) if name == "uniform_16" else amr_two_level(16)
    K = 4
    bs, etas = instances(h, K, 50)
    bs = [orc.Oracle(h, 0.5, etas[q]).sync_down(bs[q]) for q in range(K)]
    dts = [(3.0 + q) * h.dx(h.nlevels - 1) ** 2 for q in range(K)]
    g = make(ohm, h, K, precision=precision, max_outer=120)
    ohm.ohm_set_eta(g, dev(stack(h, etas)))
    B = dev(stack(h, bs))
    status, st = ohm.ohm_cn_step_batch(g, B, dts, 1e-11)
    assert status == ohm.OHM_OK, st
    got = unstack(h, host(B).reshape(-1, 1536), K)
    for q in range(K):
        assert st[q]["converged"] and st[q]["rel_l2"] <= 1e-11
        want, _ = orc.Oracle(h, 0.5, etas[q]).cn_step(bs[q], dts[q], 1e-14, 2, 2, 8, 120)
        assert rel_err(got[q], want.reshape(-1, 1536)) < 1e-9, q


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("sched", ["paper", "relaxed"])
def test_instance_same_bits_alone_and_in_batch(ohm, graphs, precision, sched):
    """An instance stepped alone (K = 1) and inside a batch of 5 with other eta, dt and data,
    some of them inactive, gives identical bits; inactive instances are left untouched.  Also
    with omega 1.3, V(3,2) on level 0 and V(1,0) on the coarser grids."""
    h = amr_two_level(16)
    K = 5
    bs, etas = instances(h, K, 60)
    dts = [(2.0 + q) * h.dx(1) ** 2 for q in range(K)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        kw = {} if sched == "paper" else dict(omega=1.3, nu_pre=3, nu_post=2, nu_coarse=(1, 0))
        g1 = make(ohm, h, 1, precision=precision, stream=stream, use_graphs=graphs, **kw)
        ohm.ohm_set_eta(g1, dev(etas[2]))
        B1 = dev(bs[2])
        s1, st1 = ohm.ohm_cn_step_batch(g1, B1, [dts[2]], 1e-9)
        s1b, st1b = ohm.ohm_cn_step_batch(g1, B1, [dts[2]], 1e-9)  # second step: graph replay
        gK = make(ohm, h, K, precision=precision, stream=stream, use_graphs=graphs, **kw)
        ohm.ohm_set_eta(gK, dev(stack(h, etas)))
        BK = dev(stack(h, bs))
        active = [1, 0, 1, 1, 0]
        sK, stK = ohm.ohm_cn_step_batch(gK, BK, dts, 1e-9, active=active)
        sKb, stKb = ohm.ohm_cn_step_batch(gK, BK, dts, 1e-9, active=active)
    stream.synchronize()
    got = unstack(h, host(BK).reshape(-1, 1536), K)
    assert st1[0]["converged"] and stK[2]["converged"]
    assert st1[0]["cycles"] == stK[2]["cycles"] and st1b[0]["cycles"] == stKb[2]["cycles"]
    assert np.array_equal(got[2], host(B1).reshape(-1, 1536))
    lv = h.blocks[:, 0]
    leaf_fine = lv == 1  # level-1 blocks are leaves; level-0 covered cells may be re-synced
    for q in (1, 4):
        assert stK[q]["cycles"] == 0
        assert np.array_equal(got[q][leaf_fine], bs[q].reshape(-1, 1536)[leaf_fine])


@pytest.mark.parametrize("graphs", [False, True])
def test_grid_wide_coarse_grids_same_bits_alone_and_in_batch(ohm, graphs):
    """A 56^3 base grid: its first coarsening that is not a multiple of 8 (28^3, 21952 cells) is
    stepped by the grid-wide coarse-grid kernels, the rest by the one-block solver.  An instance
    gives the same bits alone and in a batch of 3 with another instance inactive."""
    h = W.uniform(56, 56, 56, 1.0 / 56)
    K = 3
    bs, etas = instances(h, K, 90)
    dts = [(4.0 + q) * h.dx0 ** 2 for q in range(K)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g1 = make(ohm, h, 1, precision=1, stream=stream, use_graphs=graphs, max_outer=200)
        ohm.ohm_set_eta(g1, dev(etas[1]))
        B1 = dev(bs[1])
        s1, st1 = ohm.ohm_cn_step_batch(g1, B1, [dts[1]], 1e-9)
        gK = make(ohm, h, K, precision=1, stream=stream, use_graphs=graphs, max_outer=200)
        ohm.ohm_set_eta(gK, dev(stack(h, etas)))
        BK = dev(stack(h, bs))
        sK, stK = ohm.ohm_cn_step_batch(gK, BK, dts, 1e-9, active=[1, 1, 0])
    stream.synchronize()
    got = unstack(h, host(BK).reshape(-1, 1536), K)
    assert st1[0]["converged"] and stK[1]["converged"] and stK[0]["converged"]
    assert st1[0]["cycles"] == stK[1]["cycles"]
    assert np.array_equal(got[1], host(B1).reshape(-1, 1536))
    assert stK[2]["cycles"] == 0 and np.array_equal(got[2], bs[2].reshape(-1, 1536))


def test_graphs_give_same_bits(ohm):
    h = W.uniform(16, 16, 16, 1.0 / 16)
    K = 3
    bs, etas = instances(h, K, 70)
    dts = [8.0 * h.dx0 ** 2] * K
    outs = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            g = make(ohm, h, K, precision=1, stream=stream, use_graphs=graphs)
            ohm.ohm_set_eta(g, dev(stack(h, etas)))
            B = dev(stack(h, bs))
            for _ in range(3):
                ohm.ohm_cn_step_batch(g, B, dts, 1e-9)
        stream.synchronize()
        outs.append(host(B))
    assert np.array_equal(outs[0], outs[1])


def test_batch_of_mixed_sizes_by_class(ohm, orc):
    """Two size classes (16^3 and 24^3: blocked and lexicographic coarsest grids) as two
    batches; the 24^3 class goes through a 12^3 lexicographic grid per instance."""
    for n in (16, 24):
        h = W.uniform(n, n, n, 1.0 / n)
        K = 2
        bs, etas = instances(h, K, 80 + n)
        dts = [10.0 * h.dx0 ** 2, 40.0 * h.dx0 ** 2]
        g = make(ohm, h, K, max_outer=2)
        ohm.ohm_set_eta(g, dev(stack(h, etas)))
        B = dev(stack(h, bs))
        ohm.ohm_cn_step_batch(g, B, dts, -1.0)
        got = unstack(h, host(B).reshape(-1, 1536), K)
        for q in range(K):
            want, _ = orc.Oracle(h, 0.5, etas[q]).cn_step(bs[q], dts[q], -1.0, 2, 2, 8, 2)
            assert rel_err(got[q], want.reshape(-1, 1536)) < 1e-12


def test_autotune_picks_a_converging_schedule(ohm):
    wl = W.resistive_bump_256(n=32)
    g = ohm.ohm_create_hierarchy(wl.hier.base_cells, wl.hier.dx0, wl.hier.blocks, lam=wl.lam, precision=1,
                                 max_outer=200)
    ohm.ohm_set_eta(g, dev(wl.eta))
    B0 = dev(wl.B)
    r = ohm.ohm_autotune(g, B0, wl.dt, 1e-9)
    # 24 schedules at the hierarchy's omega (1), then V(1,1) and V(1,0) on the coarser grids, then
    # omega 1.15, 1.3 and 1.45 on the best one
    assert r["candidates"] == 29 and r["ms"] > 0
    assert r["nu_coarse"] in [(0, 0), (1, 1), (1, 0)]
    assert (r["nu_pre"], r["nu_post"]) in [(1, 1), (2, 1), (2, 2), (3, 2), (3, 3), (4, 4)]
    assert r["omega"] in (1.0, 1.15, 1.3, 1.45)
    assert np.array_equal(host(B0).reshape(-1), wl.B.reshape(-1))  # the input is not modified
    st = ohm.ohm_cn_step(g, B0, None, wl.dt, 1e-9)
    assert st["converged"]


def test_batch_rejects_single_entry_points_and_bad_args(ohm):
    h = W.uniform(16, 16, 16, 1.0 / 16)
    g = make(ohm, h, 2)
    eta = dev(np.ones(2 * h.nblocks * 512))
    ohm.ohm_set_eta(g, eta)
    B = dev(np.zeros(2 * h.nblocks * 1536))
    with pytest.raises(ohm.OhmError):
        ohm.ohm_cn_step(g, B, None, 0.1, 1e-9)
    with pytest.raises(ohm.OhmError):
        ohm.ohm_cn_step_batch(g, B, [0.1, -1.0], 1e-9)
    status, st = ohm.ohm_cn_step_batch(g, B, [0.1, -1.0], 1e-9, active=[1, 0])  # inactive dt unused
    assert status == ohm.OHM_OK and st[1]["cycles"] == 0


@pytest.mark.parametrize("name", ["uniform_16", "amr_2level"])
def test_fgmres_batch_converges_to_oracle(ohm, orc, name):
    """Per-instance FGMRES(4) inner solves in one batch reach each instance's FP64 solution."""
    h = W.uniform(16, 16, 16, 1.0 / 16) if name == "uniform_16" else amr_two_level(16)
    K = 4
    bs, etas = instances(h, K, 90)
    bs = [orc.Oracle(h, 0.5, etas[q]).sync_down(bs[q]) for q in range(K)]
    dts = [(3.0 + 2.0 * q) * h.dx(h.nlevels - 1) ** 2 for q in range(K)]
    g = make(ohm, h, K, precision=1, max_outer=120, krylov=4)
    ohm.ohm_set_eta(g, dev(stack(h, etas)))
    B = dev(stack(h, bs))
    status, st = ohm.ohm_cn_step_batch(g, B, dts, 1e-11)
    assert status == ohm.OHM_OK, st
    got = unstack(h, host(B).reshape(-1, 1536), K)
    for q in range(K):
        assert st[q]["converged"] and st[q]["rel_l2"] <= 1e-11
        want, _ = orc.Oracle(h, 0.5, etas[q]).cn_step(bs[q], dts[q], 1e-14, 2, 2, 8, 120)
        assert rel_err(got[q], want.reshape(-1, 1536)) < 1e-9, q


@pytest.mark.parametrize("graphs", [False, True])
@pytest.mark.parametrize("precision", [1, 2])
def test_fgmres_batch_same_bits_alone_and_in_batch(ohm, precision, graphs):
    """Per-instance FGMRES(4): an instance gives the same bits alone and in a batch, with the
    restart cycles run eagerly or replayed from a CUDA graph (two steps: the second replays)."""
    h = amr_two_level(16)
    K = 4
    bs, etas = instances(h, K, 95)
    dts = [(2.0 + q) * h.dx(1) ** 2 for q in range(K)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g1 = make(ohm, h, 1, precision=precision, krylov=4, stream=stream, use_graphs=graphs)
        ohm.ohm_set_eta(g1, dev(etas[1]))
        B1 = dev(bs[1])
        _, st1 = ohm.ohm_cn_step_batch(g1, B1, [dts[1]], 1e-9)
        _, st1b = ohm.ohm_cn_step_batch(g1, B1, [dts[1]], 1e-9)
        gK = make(ohm, h, K, precision=precision, krylov=4, stream=stream, use_graphs=graphs)
        ohm.ohm_set_eta(gK, dev(stack(h, etas)))
        BK = dev(stack(h, bs))
        _, stK = ohm.ohm_cn_step_batch(gK, BK, dts, 1e-9, active=[1, 1, 0, 1])
        _, stKb = ohm.ohm_cn_step_batch(gK, BK, dts, 1e-9, active=[1, 1, 0, 1])
    stream.synchronize()
    got = unstack(h, host(BK).reshape(-1, 1536), K)
    assert st1[0]["converged"] and stK[1]["converged"] and st1[0]["cycles"] == stK[1]["cycles"]
    assert st1b[0]["converged"] and st1b[0]["cycles"] == stKb[1]["cycles"]
    assert np.array_equal(got[1], host(B1).reshape(-1, 1536))
    assert stK[2]["cycles"] == 0 and stKb[2]["cycles"] == 0


def test_fgmres_batch_graphs_give_same_bits(ohm):
    """The batched FGMRES restart cycle replayed from a CUDA graph gives the bits of the eager
    launches (three steps of a 3-instance batch)."""
    h = W.uniform(16, 16, 16, 1.0 / 16)
    K = 3
    bs, etas = instances(h, K, 97)
    dts = [(4.0 + q) * h.dx0 ** 2 for q in range(K)]
    outs = []
    for graphs in (False, True):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            g = make(ohm, h, K, precision=1, krylov=5, stream=stream, use_graphs=graphs)
            ohm.ohm_set_eta(g, dev(stack(h, etas)))
            B = dev(stack(h, bs))
            for _ in range(3):
                status, st = ohm.ohm_cn_step_batch(g, B, dts, 1e-9)
                assert status == ohm.OHM_OK
        stream.synchronize()
        outs.append(host(B))
    assert np.array_equal(outs[0], outs[1])


def test_fgmres_batch_takes_fewer_cycles(ohm):
    """On the stiff 32^3 resistive bump (3-decade eta, dt = 100x the explicit limit), batched
    FGMRES(6) needs fewer V-cycles per instance than batched defect correction."""
    wl = W.resistive_bump_256(n=32)
    K = 3
    cyc = {}
    for kr in (0, 6):
        g = make(ohm, wl.hier, K, precision=1, max_outer=300, krylov=kr, n_coarse=16)
        ohm.ohm_set_eta(g, dev(np.concatenate([wl.eta] * K)))
        B = dev(np.concatenate([wl.B] * K))
        status, st = ohm.ohm_cn_step_batch(g, B, [wl.dt, 0.5 * wl.dt, 2.0 * wl.dt], 1e-9)
        assert status == ohm.OHM_OK
        cyc[kr] = [x["cycles"] for x in st]
    assert all(a < b for a, b in zip(cyc[6], cyc[0])), cyc
