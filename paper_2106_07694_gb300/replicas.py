"""Independent replicas across ranks (one simulation per GPU, no data-path collective).

The coupled step shards by slabs, but every run of this library uses one GPU per
process; N processes advance N independent simulations.  The job's time is the
slowest rank's time (max over ranks) and its throughput counts the nodes of every rank.
"""


def job_time_ms(local_ms, device=None):
    """Max over ranks of local_ms (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_glups(local_ms, nodes_per_rank, steps, device=None):
    """(GLUPS of the whole job, job time in ms) for `steps` steps of `nodes_per_rank`
    lattice nodes on every rank."""
    import torch.distributed as dist
    world = dist.get_world_size() if (dist.is_available() and dist.is_initialized()) else 1
    t = job_time_ms(local_ms, device)
    return world * nodes_per_rank * steps / (t * 1e-3) / 1e9, t
