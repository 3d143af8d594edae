"""Work division over ranks on CPU: two gloo processes compute the instance
split and the max-over-ranks timing reduction the benchmark uses."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

from paper_2603_18052_gb300 import ranks  # noqa: E402


def test_partition_is_complete_disjoint_and_balanced():
    from workloads.configs import make_instances

    inst, models = make_instances(256)
    costs = [ranks.instance_cost(x["d"], len(x["u"]), x["states"].shape[0]) for x in inst]
    for world in (1, 2, 3, 8):
        parts = ranks.partition(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        # largest-first greedy: no rank exceeds the mean by more than the largest item
        assert max(loads) - sum(loads) / world <= max(costs) + 1e-9
    assert ranks.partition(costs, 4) == ranks.partition(list(costs), 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = ranks.dist_env()
    mine = ranks.partition(costs, w)[r]
    got = [None] * w
    dist.all_gather_object(got, mine)
    t = ranks.max_over_ranks(10.0 * (r + 1))
    out.put((r, got, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_split_and_max():
    costs = [float((7 * k) % 13 + 1) for k in range(40)]
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, got, t in res:
        assert t == 20.0
        flat = sorted(i for part in got for i in part)
        assert flat == list(range(len(costs)))
        assert got == ranks.partition(costs, world)
