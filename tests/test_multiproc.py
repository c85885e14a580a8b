"""The multi-GPU path partitions images across ranks (no data-path
collective); its host logic is tested with world_size 2 over gloo on CPU."""
import os
import socket

import gs_synthetic as S
from paper_2501_06838_gb300.shard import image_costs, shard_images


def test_shard_images_cover_and_balance():
    _, views = S.config3()
    costs = image_costs(views)
    for world in (1, 2, 3, 4, 8, 16, 20):
        parts = shard_images(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(views)))            # disjoint cover
        loads = [sum(costs[i] for i in p) for p in parts]
        # LPT bound: max load <= mean + largest single image
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
    assert shard_images([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2501_06838_gb300.shard import image_costs, max_over_ranks, shard_images
        _, views = S.config3()
        parts = shard_images(image_costs(views), world)
        mine = parts[rank]
        # every rank computes the same partition without communicating
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        t = max_over_ranks(10.0 + rank)
        q.put((rank, mine, gathered, t))
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    (r0, m0, g0, t0), (r1, m1, g1, t1) = res
    assert g0 == g1 == [m0, m1]
    assert sorted(m0 + m1) == list(range(16)) and not set(m0) & set(m1)
    assert t0 == t1 == 11.0
