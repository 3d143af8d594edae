"""Work division over ranks (one process per GPU).

Every part of the hot path shards without an exchange: the d = 27 chain runs
as one independent replica per rank (weak scaling), and a list of
independent problems (lb_run_instances) is divided between ranks by cost.
The only collective is the maximum over ranks of a timed region.
"""

import os


def dist_env():
    """(rank, world, local_rank) from the launcher's environment."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def instance_cost(d, nslices, B, steps_per_slice=1):
    """Arithmetic of one problem in units of complex multiply-adds: the
    builds (about 19 n^3 each for the six products, the LU and the solve, at
    one squaring) plus the propagation (n^2 per state-step), n = d^2."""
    n = d * d
    return nslices * (19.0 * n ** 3 + steps_per_slice * B * n ** 2)


def partition(costs, world):
    """Split item indices into `world` lists with near-equal total cost:
    largest first, each to the currently lightest rank (ties to the lower
    rank).  Deterministic, so every rank computes the same split."""
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    for p in parts:
        p.sort()
    return parts


def max_over_ranks(x, device=None):
    """Maximum of a float over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
