"""The N > 1 host logic on CPU: two gloo ranks on 127.0.0.1 split a batch of uneven
grids without overlap and combine their timings (slowest rank, total work)."""
import os
import socket

import pytest

from paper_1909_00709_gb300 import inputs, replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        shapes = inputs.batch_shapes(40, seed=3)
        mine = replicas.assign_grids(shapes, world)[rank]
        pts = sum(shapes[i][0] * shapes[i][1] * shapes[i][2] for i in mine)
        slow = replicas.slowest(10.0 + rank)
        tot = replicas.total(pts)
        q.put((rank, mine, pts, slow, tot))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_split_and_combine():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shapes = inputs.batch_shapes(40, seed=3)
    (_, m0, p0, s0, t0), (_, m1, p1, s1, t1) = res
    assert sorted(m0 + m1) == list(range(40)) and not set(m0) & set(m1)
    assert s0 == s1 == 11.0
    assert t0 == t1 == p0 + p1 == sum(a * b * c for a, b, c in shapes)
    assert max(p0, p1) <= 1.34 * (p0 + p1) / 2


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_assignment_is_a_balanced_partition(world):
    shapes = inputs.batch_shapes(256, seed=3)
    parts = replicas.assign_grids(shapes, world)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(256))
    loads = [sum(shapes[i][0] * shapes[i][1] * shapes[i][2] for i in p) for p in parts]
    big = max(a * b * c for a, b, c in shapes)
    assert max(loads) - min(loads) <= big  # LPT: the spread is at most the largest unit
