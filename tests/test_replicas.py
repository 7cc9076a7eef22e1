"""The multi-GPU host logic (independent replicas, timing reductions) with two
gloo ranks on CPU: the slowest replica sets the job time, the whole-job
throughput counts every replica's snapshots, replicas get distinct streams."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2108_08845_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world_size, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        ws, r, local = replicas.world()
        ms_local = 100.0 + 25.0 * rank       # rank 1 is the slow replica
        e2e_local = 5000.0 - 1000.0 * rank   # and the one with the lower end-to-end rate
        ms_max, e2e_min = replicas.reduce_timing(ms_local, e2e_local, ws)
        out[rank] = (ws, r, local, ms_max, e2e_min, replicas.stream_seed(1236, r))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_reduce_timing():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        ws, rr, local, ms_max, e2e_min, seed = res[r]
        assert (ws, rr, local) == (2, r, r)
        assert ms_max == 125.0 and e2e_min == 4000.0   # every rank sees the job's values
    assert res[0][5] != res[1][5]                        # distinct snapshot streams
    assert replicas.job_throughput(2, 8, 128, 125.0) == pytest.approx(2 * 8 * 128 / 0.125)


def test_single_replica_passthrough():
    assert replicas.reduce_timing(12.5, None, 1) == (12.5, None)
    assert replicas.reduce_timing(12.5, 3.0, 1) == (12.5, 3.0)
