"""Multi-GPU runs of the solve as independent replicas: one process per GPU
(launched by torchrun), no collective on the data path.  The only
communication is around the timed region: a barrier before and after, and
the maximum of the per-rank elapsed times, which is the whole job's time;
the job's throughput is the units all ranks processed divided by it.
"""

import os


def world():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def setup(backend: str = "nccl"):
    """Join the process group (world size > 1) and select this rank's GPU
    (NCCL).  Returns (world size, rank, local rank)."""
    import torch
    ws, rank, local = world()
    if backend == "nccl":
        torch.cuda.set_device(local if ws > 1 else 0)
    if ws > 1:
        import torch.distributed as dist
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x: float, ws: int, device: str = "cuda") -> float:
    """The maximum of x over the ranks (x on a single rank)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ws: int, max_ms: float) -> float:
    """Units of all ranks per second of the slowest rank (weak scaling)."""
    return ws * units_per_rank / (max_ms / 1e3)


def teardown(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
