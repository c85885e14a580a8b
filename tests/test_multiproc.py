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


def _bench_worker(rank, world, port, q):
    """The benchmark's own sharding code (bench.shard_workload) on two gloo
    ranks: each rank takes its part; the band adjoints are summed with the
    same all-reduce the benchmark runs (shard.allreduce_band_grads)."""
    import argparse

    import numpy as np
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2501_06838_gb300.shard import allreduce_band_grads
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out = {}
        # config 3: its 16 images partitioned, no collective
        g3, v3 = S.config3()
        a = argparse.Namespace(shard="auto", tile=0, workload="c3")
        _, mv, info = bench.shard_workload(a, g3, v3, rank, world)
        out["c3"] = (info["rank_images"], info["scaling"], info["job_hr_pixels"], len(mv))
        # a single-image workload: a batch of one image per rank
        g1, v1 = S.config1()
        a = argparse.Namespace(shard="auto", tile=0, workload="c1")
        mg, _, info = bench.shard_workload(a, g1, v1, rank, world)
        out["c1"] = (float(mg[0].sigma.sum()), info["scaling"], info["job_hr_pixels"])
        # row bands of one image: the bands' adjoints sum to the image's
        a = argparse.Namespace(shard="bands", tile=16, workload="c1")
        mg, mv, info = bench.shard_workload(a, g1, v1, rank, world)
        r0, rows = info["band"]
        assert (mv[0].row0, mv[0].out_h) == (r0, rows)
        go = S.grad_out(5, v1[0].out_h, v1[0].out_w)
        # a band's adjoint is the image's adjoint of the upstream gradient
        # restricted to the band's rows (the oracle renders whole images)
        gb = np.zeros_like(go)
        gb[:, r0:r0 + rows] = go[:, r0:r0 + rows]
        gr = torch.from_numpy(oracle.adjoint(mg[0], v1[0], gb))
        allreduce_band_grads(gr)
        whole = oracle.adjoint(g1[0], v1[0], go)
        err = float(np.abs(gr.numpy() - whole).max() / np.abs(whole).max())
        out["bands"] = (r0, rows, info["scaling"], info["job_hr_pixels"], err)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_bench_sharding_two_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_bench_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    a, b = res[0], res[1]
    # images partitioned: disjoint cover, each rank fewer than all, same job size
    assert sorted(a["c3"][0] + b["c3"][0]) == list(range(16)) and a["c3"][3] + b["c3"][3] == 16
    assert a["c3"][1] == "strong" and a["c3"][2] == b["c3"][2]
    # one image per rank: different draws, job = two images
    assert a["c1"][0] != b["c1"][0] and a["c1"][1] == "weak"
    assert a["c1"][2] == b["c1"][2] == 2 * 192 * 192
    # bands partition the rows on tile rows; the summed adjoint is the image's
    (r0a, na, sa, ja, ea), (r0b, nb, _, _, eb) = a["bands"], b["bands"]
    assert r0a == 0 and r0b == na and na + nb == 192 and na % 16 == 0
    assert sa == "strong" and ja == 192 * 192
    assert ea < 1e-12 and eb < 1e-12
