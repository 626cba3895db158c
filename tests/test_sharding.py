"""Sharding of independent realizations across ranks, on CPU: the LPT
partition, and a world_size-2 gloo run in which each rank advances only its
shard (with the oracle standing in for the GPU) and the gathered results equal
a single-process run."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1803_02977_gb300 import sharding, synth


def test_lpt_partition_is_complete_disjoint_and_balanced():
    b = synth.batch_workload(count=512)
    sizes = [s * s for s in b.sides]
    for n in (1, 2, 3, 4, 8):
        parts = sharding.lpt_partition(sizes, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = sharding.shard_loads(sizes, parts)
        # LPT bound: makespan <= 4/3 OPT, and OPT >= max(mean load, largest item)
        opt_lb = max(sum(sizes) / n, max(sizes))
        assert max(loads) <= 4 / 3 * opt_lb + 1
    assert sharding.lpt_partition(sizes, 4) == sharding.lpt_partition(sizes, 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _tiny_batch():
    sides = [7, 12, 9, 15, 5, 11, 8, 6]
    return [synth.noise_surface(s, s + 1, 1000 + r) for r, s in enumerate(sides)]


def _worker(rank, world, port, out):
    import torch
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    surfaces = _tiny_batch()
    parts = sharding.lpt_partition([s.size for s in surfaces], world)
    mine = parts[rank]
    p = oracle.params(K=2e-5)
    sums = torch.zeros(len(surfaces), dtype=torch.float64)
    for i in mine:
        sums[i] = float(oracle.run(surfaces[i], p, 3).sum())
    dist.all_reduce(sums)  # host-side gather of results: each slot written by one rank
    if rank == 0:
        out.put(sums.numpy().tolist())
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_process():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = q.get(timeout=120)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = oracle.params(K=2e-5)
    want = [float(oracle.run(s, p, 3).sum()) for s in _tiny_batch()]
    assert np.allclose(got, want, rtol=0, atol=0)
