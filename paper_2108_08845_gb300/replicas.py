"""Host logic of a multi-GPU run: one independent replica of the streaming
update per GPU (Sec. 4.2's row partitions live inside one GPU's launches, so a
single GPU's path has no exchange step; several GPUs process independent
snapshot streams).  The only collectives are the timing reductions of a run:
the slowest replica's device time and the whole-job throughput."""
import os

import torch


def world():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def stream_seed(base_seed: int, rank: int) -> int:
    """Seed of replica `rank`'s snapshot stream: replicas process different data."""
    return int(base_seed) + 1000 * int(rank)


def reduce_timing(ms_local: float, e2e_local, world_size: int, device="cpu"):
    """(max over ranks of the timed region in ms, min over ranks of the end-to-end
    throughput or None).  With one rank the inputs are returned unchanged."""
    if world_size <= 1:
        return float(ms_local), (None if e2e_local is None else float(e2e_local))
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    e2e = None
    if e2e_local is not None:
        u = torch.tensor([float(e2e_local)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(u, op=torch.distributed.ReduceOp.MIN)
        e2e = float(u.item())
    return float(t.item()), e2e


def job_throughput(world_size: int, steps: int, batch: int, ms_max: float) -> float:
    """Whole-job snapshots/s: every replica processed steps * batch snapshots in at
    most ms_max milliseconds."""
    return world_size * steps * batch / (ms_max * 1e-3)
