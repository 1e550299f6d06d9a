"""Independent replicas across GPUs (one process per GPU, no data exchange).

The solve of one lattice does not shard across GPUs in this library; with
N processes each rank solves its own lattice and only the timing is
combined: the job time is the maximum over ranks and the throughput is
the units of work of all ranks divided by that time.
"""
import os


def world():
    """(rank, world_size, local_rank) from the torchrun environment (1 process when absent)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend):
    """Initialise torch.distributed when launched with more than one process."""
    rank, size, _ = world()
    if size > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend, rank=rank, world_size=size)
    return rank, size


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def combine(seconds, units, device=None):
    """(max seconds over ranks, total units over ranks)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(seconds), float(units)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
