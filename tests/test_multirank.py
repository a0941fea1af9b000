"""The benchmark's multi-GPU mode is replicas only: each rank solves its own copy and the job
throughput is all ranks' cell-steps over the slowest rank's time.  Checked here with two gloo
ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    import torch.distributed as td

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=ws)
    elapsed = [120.0, 300.0][rank]  # ms per rank
    v = bench.job_throughput(ws, 1000, 10, elapsed)
    m = bench.barrier_max(ws, elapsed)
    out.put((rank, v, m))
    td.destroy_process_group()


def test_replica_throughput_uses_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, m in res:
        assert m == 300.0
        assert v == pytest.approx(2 * 1000 * 10 / 0.3)
