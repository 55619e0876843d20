"""The multi-rank benchmark path on CPU: two gloo ranks, each running its own
replica, agree on the job time (maximum over ranks) and the whole-job rate."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import sys
    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=ws)
    t = bench.max_over_ranks(1.5 + rank, ws, torch.device("cpu"))
    rate = bench.whole_job_rate(20000, ws, t)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, rate))


def test_two_gloo_ranks_max_time_and_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.5, 2.5]           # both ranks see the slowest rank's time
    assert res[0][2] == pytest.approx(2 * 20000 / 2.5)  # units of both replicas / max time
