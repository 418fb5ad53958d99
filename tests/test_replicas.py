"""Replica bookkeeping of bench.py for runs on several GPUs (the hot path does
not shard: ranks render independently; only the barrier, the slowest rank's
time and the unit sum cross ranks).  Run as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2406_06963_b300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, lr = replicas.dist_env()
        assert (w, r, lr) == (ws, rank, rank)
        replicas.barrier(ws)
        # rank k processed 1000 (k + 1) units in 0.5 (k + 1) s
        thr, total, tmax = replicas.job_throughput(ws, 1000.0 * (rank + 1), 0.5 * (rank + 1))
        mx = replicas.max_over_ranks(ws, float(rank))
        sm = replicas.sum_over_ranks(ws, 1.0)
        replicas.barrier(ws)
        out.put((rank, thr, total, tmax, mx, sm))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, PORT, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, thr, total, tmax, mx, sm in res:
        assert total == 3000.0                 # units of both ranks
        assert tmax == 1.0                     # the slower rank's time
        assert thr == pytest.approx(3000.0)    # whole-job units / slowest time
        assert mx == 1.0 and sm == 2.0


def test_single_process_is_identity(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert replicas.dist_env() == (1, 0, 0)
    replicas.barrier(1)
    assert replicas.job_throughput(1, 500.0, 0.25) == (2000.0, 500.0, 0.25)


PORT = _free_port()
