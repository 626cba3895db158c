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
    return synth.batch_workload(count=9, side_lo=5, side_hi=17, seed=11)


def _oracle_advance(surfaces, pars, steps):
    # the oracle stands in for the GPU step on a CPU-only run
    import oracle
    return [oracle.run(s.astype(np.float64), oracle.params(**p), steps).astype(np.float32)
            for s, p in zip(surfaces, pars)]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bw = _tiny_batch()
    parts = sharding.lpt_partition([s * s for s in bw.sides], world)
    res = sharding.run_shard(None, bw, parts[rank], 3, advance=_oracle_advance)
    full = sharding.gather_surfaces(res["surfaces"], bw.count, rank, world)
    if rank == 0:
        out.put([np.asarray(s).tolist() for s in full])
    else:
        assert full is None
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_process():
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
    bw = _tiny_batch()
    single = sharding.run_shard(None, bw, list(range(bw.count)), 3, advance=_oracle_advance)
    want = sharding.gather_surfaces(single["surfaces"], bw.count, 0, 1)
    assert len(got) == bw.count
    for r in range(bw.count):
        g = np.asarray(got[r], np.float32)
        assert g.shape == want[r].shape
        assert np.array_equal(g, want[r]), f"realization {r} differs"
        # each realization really advanced
        assert not np.array_equal(g, bw.initial(r).astype(np.float32))


def test_gather_rejects_missing_or_duplicate_realizations():
    with pytest.raises(KeyError):
        sharding.gather_surfaces({0: 1, 2: 3}, 3, 0, 1)
