"""Sharding of independent simulations across ranks: partition properties
and a 2-rank gloo run (CPU) whose per-simulation results equal a
single-process run."""
import os
import socket

import numpy as np

from paper_2503_10796_gb300 import sharding, workloads


def test_lpt_partition_properties():
    rng = np.random.default_rng(0)
    sizes = rng.integers(1000, 200000, 256)
    for n in (1, 2, 3, 4, 8):
        parts = sharding.lpt_partition(sizes, n)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [int(sum(sizes[i] for i in p)) for p in parts]
        # LPT bound: max load <= 4/3 optimum, optimum >= mean and >= max item
        opt_lb = max(sum(sizes) / n, max(sizes))
        assert max(loads) <= 4.0 / 3.0 * opt_lb + 1
    assert sharding.lpt_partition([5, 5, 5], 2) == [[0, 2], [1]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    pops = workloads.batched_sweep(n_sims=6, lo=40, hi=400, seed=2)
    idx, mine = sharding.shard(pops, [p.n for p in pops], rank, world)
    res = {}
    for i, p in zip(idx, mine):
        s = oracle.Sim(p.xyz, p.diameter, p.params)
        s.step(2)
        res[i] = s.get()[0]
    gathered = [None] * world
    dist.all_gather_object(gathered, res)
    if rank == 0:
        merged = {}
        for g in gathered:
            merged.update(g)
        out.put(merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gloo_shards_match_single_process(orc):
    import multiprocessing as mp
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pops = workloads.batched_sweep(n_sims=6, lo=40, hi=400, seed=2)
    assert sorted(merged) == list(range(6))
    for i, p in enumerate(pops):
        s = oracle.Sim(p.xyz, p.diameter, p.params)
        s.step(2)
        assert np.array_equal(merged[i], s.get()[0])
