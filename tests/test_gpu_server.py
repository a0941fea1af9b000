"""Continuous-batching solve service (include/ohm_server.h): each request's result is the same
bits alone and in a mix of requests of several classes arriving together, matches the FP64
oracle (1e-9 relative after refinement to 1e-11), and admission stays within the HBM budget.
"""
import time

import numpy as np
import pytest

from paper_1009_0798_gb300 import workloads as W
from tests.helpers import amr_two_level, rand_fields, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def srv():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_0798_gb300 import build, server
    build.build()
    torch.cuda.init()
    return server


def request(h, seed, q):
    b, eta = rand_fields(h, seed, 1.0)
    dt = (3.0 + q) * h.dx(h.nlevels - 1) ** 2
    return h, b, eta, dt


CLASSES = {
    "u16": lambda: W.uniform(16, 16, 16, 1.0 / 16),
    "u24": lambda: W.uniform(24, 24, 24, 1.0 / 24),
    "amr": lambda: amr_two_level(16),
}


def test_same_bits_alone_and_in_a_mix(srv):
    h = CLASSES["amr"]()
    _, b, eta, dt = request(h, 101, 0)
    with srv.Server(hbm_budget_bytes=4 << 30, max_batch=4, n_workers=2, tol=1e-9) as s:
        alone, r_alone = s.wait(s.submit(h, b, eta, dt, 2))
    mix = []
    for i in range(12):
        name = ["u16", "u24", "amr"][i % 3]
        hh = CLASSES[name]()
        mix.append(request(hh, 200 + i, i % 5) + (1 + i % 3,))
    with srv.Server(hbm_budget_bytes=4 << 30, max_batch=4, n_workers=3, tol=1e-9, use_graphs=True) as s:
        ids = [s.submit(hh, bb, ee, dd, ns) for hh, bb, ee, dd, ns in mix[:5]]
        rid = s.submit(h, b, eta, dt, 2)
        ids += [s.submit(hh, bb, ee, dd, ns) for hh, bb, ee, dd, ns in mix[5:]]
        in_mix, r_mix = s.wait(rid)
        others = [s.wait(i) for i in ids]
        stats = s.stats()
    assert r_alone["status"] == 0 and r_mix["status"] == 0
    assert r_alone["cycles"] == r_mix["cycles"]
    assert np.array_equal(alone, in_mix)
    assert all(o[1]["status"] == 0 for o in others)
    assert stats["requests_done"] == 13 and stats["mean_active_slots"] > 1.0


def test_results_match_oracle(srv, oracle_mod):
    reqs = [request(CLASSES[n](), 300 + i, i) for i, n in enumerate(["u16", "u24", "amr", "u16"])]
    with srv.Server(hbm_budget_bytes=2 << 30, max_batch=2, n_workers=2, tol=1e-11) as s:
        ids = [s.submit(h, b, e, dt, 1) for h, b, e, dt in reqs]
        outs = [s.wait(i) for i in ids]
    for (h, b, e, dt), (out, res) in zip(reqs, outs):
        assert res["status"] == 0 and res["rel_l2"] <= 1e-11
        o = oracle_mod.Oracle(h, 0.5, e)
        want, _ = o.cn_step(o.sync_down(b), dt, 1e-14, 2, 2, 16, 200)
        assert rel_err(out, want) < 1e-9


def test_admission_within_budget_evicts_idle_batches(srv):
    from paper_1009_0798_gb300 import ohm
    hs = [CLASSES[n]() for n in ("u16", "u24", "amr")]
    need = max(ohm.ohm_hierarchy_bytes(h.base_cells, h.dx0, h.blocks, precision=1, n_instances=2)
               + 2 * h.nblocks * 2048 * 8 for h in hs)
    budget = int(need * 1.2)  # one batch of any class at a time
    with srv.Server(hbm_budget_bytes=budget, max_batch=2, n_workers=3, tol=1e-9) as s:
        ids = []
        for i in range(9):
            h = hs[i % 3]
            _, b, e, dt = request(h, 400 + i, i % 4)
            ids.append(s.submit(h, b, e, dt, 1))
        res = [s.wait(i, 300.0) for i in ids]
        stats = s.stats()
    assert all(r is not None and r[1]["status"] == 0 for r in res)
    assert stats["bytes_resident_max"] <= budget
    assert stats["batches_evicted"] >= 1


def test_requests_join_running_batches(srv):
    """Requests that arrive while a batch steps are admitted at its next step boundary."""
    h = CLASSES["u16"]()
    with srv.Server(hbm_budget_bytes=2 << 30, max_batch=4, n_workers=1, tol=1e-9) as s:
        _, b, e, dt = request(h, 500, 0)
        first = s.submit(h, b, e, dt, 40)
        time.sleep(0.05)
        late = [s.submit(h, *request(h, 501 + i, i)[1:], 2) for i in range(3)]
        r_late = [s.wait(i) for i in late]
        r_first = s.wait(first)
    assert all(r[1]["status"] == 0 for r in r_late)
    # the late requests finished while the long one was still running in the same batch
    assert max(r[1]["t_done"] for r in r_late) < r_first[1]["t_done"]
    assert len({r[1]["slot"] for r in r_late} | {r_first[1]["slot"]}) >= 2


def test_oversized_request_is_rejected(srv):
    from paper_1009_0798_gb300 import ohm
    h = CLASSES["u16"]()
    with srv.Server(hbm_budget_bytes=1 << 16, max_batch=2, n_workers=1) as s:
        _, b, e, dt = request(h, 600, 0)
        with pytest.raises(ohm.OhmError):
            s.submit(h, b, e, dt, 1)


@pytest.mark.slow
def test_serving_sizes_converge_and_pass_oracle(srv, oracle_mod):
    """Requests of the serving workload's largest uniform class (128^3) and its AMR class (base
    32^3, sphere r < 0.2 refined), with the service configuration bench.py times: each converges
    and the oracle re-evaluates its residual."""
    import bench
    reqs = bench.serving_requests(40, 200.0)
    pick = [next(r for r in reqs if r["key"] == 128), next(r for r in reqs if r["key"] == "amr")]
    cfg = dict(hbm_budget_bytes=60 << 30, max_batch=8, n_workers=2, precision=1, tol=1e-9, use_graphs=True,
               nu_pre=4, nu_post=4, n_coarse=4, max_outer=400)
    with srv.Server(**cfg) as s:
        ids = [s.submit(r["hier"], r["B"] * r["fb"], r["eta"] * r["fe"], r["dt"], 1) for r in pick]
        outs = [s.wait(i) for i in ids]
    for r, (out, res) in zip(pick, outs):
        assert res["status"] == 0 and res["rel_l2"] <= 1e-9
        o = oracle_mod.Oracle(r["hier"], 0.5, r["eta"] * r["fe"])
        b = o.sync_down(r["B"] * r["fb"])
        S = o.source(b, r["dt"])
        _, norms = o.residual(out.reshape(b.shape), S, r["dt"])
        assert norms["rel_l2"] <= 1.05e-9, norms
