"""Host-side logic of the multi-GPU forms: one process per GPU, no exchange on
the data path.

Independent work (replicas of one workload, or whole jobs of a batch or of a
served arrival stream) is dealt to the ranks; the only collectives are the
barrier around the timed region and the reductions of the reported numbers
(the slowest rank's time, the sum of all ranks' work).  The same functions run
under NCCL on GPUs and under gloo on the CPU.
"""
from __future__ import annotations

import os


def world():
    """(rank, world_size, local_rank) from the launcher's environment."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, ws, local


def init(backend="nccl"):
    """Join the process group when launched with WORLD_SIZE > 1.  With NCCL
    each rank binds the GPU of its local rank.  Returns world()."""
    import torch
    rank, ws, local = world()
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return rank, ws, local


def finish(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def deal(items, rank, ws):
    """Round-robin share of `items` for `rank` (item k goes to rank k mod ws)."""
    return [x for k, x in enumerate(items) if k % ws == rank]


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    import torch.distributed as dist
    return x if ws == 1 else _reduce(x, ws, dist.ReduceOp.MAX)


def sum_over_ranks(x, ws):
    import torch.distributed as dist
    return x if ws == 1 else _reduce(x, ws, dist.ReduceOp.SUM)


def aggregate_rate(local_units, local_seconds, ws):
    """Whole-job throughput: the units all ranks processed / the slowest
    rank's time (weak scaling: each rank's share is fixed as ws grows)."""
    return sum_over_ranks(local_units, ws) / max_over_ranks(local_seconds, ws)
