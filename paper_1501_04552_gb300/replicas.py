"""Independent replicas on several GPUs of one node.

The step of the method is not sharded here: one field fits one GPU, so N GPUs run N
independent replicas (the ensemble's instances are independent too).  Throughput is
whole-job: the units all ranks processed divided by the slowest rank's time, which
needs the maximum of the per-rank times across ranks.
"""


def max_over_ranks(value, device="cpu"):
    """maximum of a float over all ranks of the default process group (the value itself
    when torch.distributed is not initialised)"""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank, world, slowest_seconds):
    """whole-job units per second for weak scaling (every rank processed units_per_rank)"""
    return world * units_per_rank / slowest_seconds
