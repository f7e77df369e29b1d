"""Host logic of the multi-rank (replicas only) path on CPU with gloo,
world_size 2: case partition, max over ranks, aggregate throughput."""
import os
import socket

import pytest

from paper_2102_01366_gb300 import replicas


def test_assign_cases_balances_and_covers():
    cells = [6 * n ** 3 for n in (8, 40, 12, 33, 20, 9, 27, 16)]
    parts = replicas.assign_cases(cells, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(cells)))
    loads = [sum(cells[i] for i in p) for p in parts]
    # LPT bound: no rank exceeds the ideal share by more than the largest case
    assert max(loads) <= sum(cells) / 3 + max(cells)
    assert replicas.assign_cases(cells, 3) == parts  # deterministic
    assert replicas.assign_cases([5, 5], 4)[2:] == [[], []]
    with pytest.raises(ValueError):
        replicas.assign_cases([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, r, lr = replicas.world()
        slowest = replicas.max_over_ranks(1.0 + rank)       # rank 1 is slower
        tput = replicas.aggregate(100.0 * (rank + 1), 2.0 + rank)
        out.put((r, ws, slowest, tput))
    finally:
        dist.destroy_process_group()


def test_max_and_aggregate_over_two_gloo_ranks():
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
    for r, (rank, ws, slowest, tput) in enumerate(res):
        assert rank == r and ws == 2
        assert slowest == 2.0
        assert tput == pytest.approx((100.0 + 200.0) / 3.0)


def test_single_process_is_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate(10.0, 2.0) == 5.0


def _split_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    from paper_2102_01366_gb300 import inputs as I
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, W, dW, desc, meshes = I.batch_cases(n_cases=6, n_range=(2, 4), seed=3)
        mine, my_meshes, Wr, dWr = replicas.rank_batch(meshes, W, dW, world, rank)
        got = [None] * world
        dist.all_gather_object(got, (mine, Wr.sum(), Wr.shape[1], dWr.shape[1]))
        out.put((rank, got, W.sum(), W.shape[1]))
    finally:
        dist.destroy_process_group()


def test_batched_cases_split_over_two_gloo_ranks():
    """The batched workload's cases split over 2 ranks: every case on exactly
    one rank, each rank's state the columns of its cases."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, got, wsum, ncells = res[0]
    cases = sorted(k for mine, _, _, _ in got for k in mine)
    assert cases == list(range(6))
    assert sum(n for _, _, n, _ in got) == ncells
    assert all(n == m for _, _, n, m in got)
    assert abs(sum(s for _, s, _, _ in got) - wsum) < 1e-9 * abs(wsum)
    assert all(len(mine) > 0 for mine, _, _, _ in got)
