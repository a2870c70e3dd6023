"""Slab decomposition with halo exchange and migration (host side): the
pack/unpack and halo rules by hand, and 2- and 3-rank gloo runs (CPU) whose
positions after several iterations equal a single-domain run bit for bit
(the oracle steps every rank's agents; each sum over neighbours runs in
ascending ID order on every rank, as in one domain)."""
import os
import socket

import numpy as np
import pytest

from paper_2503_10796_gb300 import halo, workloads


def test_pack_unpack_and_owner_rules():
    ids = np.array([7, 2, 2 ** 40])
    xyz = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, -6.5], [0.1, 0.2, 0.3]])
    d = np.array([10.0, 9.0, 8.5])
    i2, x2, d2 = halo.unpack(halo.pack(ids, xyz, d))
    assert np.array_equal(i2, ids) and np.array_equal(x2, xyz) and np.array_equal(d2, d)
    s = halo.Slabs(0.0, 30.0, 3)  # edges 0, 10, 20, 30; outer slabs open
    assert s.owner([-5.0, 0.0, 9.99, 10.0, 19.0, 20.0, 45.0]).tolist() == [0, 0, 0, 1, 1, 2, 2]
    z = np.array([10.5, 12.0, 17.9, 18.0, 19.5])
    down, up = halo.halo_masks(z, s, 1, 2.0)
    assert down.tolist() == [True, False, False, False, False]
    assert up.tolist() == [False, False, False, True, True]
    down0, up0 = halo.halo_masks(np.array([1.0, 9.0]), s, 0, 2.0)
    assert down0.tolist() == [False, False] and up0.tolist() == [False, True]
    with pytest.raises(ValueError):
        halo.pack([2 ** 53], np.zeros((1, 3)), [1.0])


def _free_port():
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    return port


def _population():
    # a dense uniform cube: contacts across every slab face, and agents that
    # the forces push across faces
    xyz, d = workloads.uniform_cube(2500, 70.0, seed=4)
    return workloads.Population(xyz, d, workloads.SimParams(precision=0))


def _rank_main(rank, world, port, iters, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    pop = _population()

    def engine(xyz, d, ghost):
        s = oracle.Sim(xyz, d, pop.params)
        s.step(1)
        return s.get()[0]

    z = pop.xyz[:, 2]
    slabs = halo.Slabs(float(z.min()), float(z.max()), world)
    dom = halo.SlabDomain(slabs, rank, np.arange(pop.n), pop.xyz, pop.diameter)
    halo_in = moved = 0
    for _ in range(iters):
        c = dom.step(dist, engine)
        halo_in += c["halo_in"]
        moved += c["migrated_out"]
    gathered = [None] * world
    dist.all_gather_object(gathered, (dom.ids, dom.xyz, halo_in, moved))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slab_ranks_match_one_domain(orc, world):
    import multiprocessing as mp

    import oracle
    iters = 4
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, iters, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    pop = _population()
    ids = np.concatenate([g[0] for g in gathered])
    xyz = np.concatenate([g[1] for g in gathered])
    assert np.array_equal(np.sort(ids), np.arange(pop.n))  # every agent on exactly one rank
    assert all(g[2] > 0 for g in gathered)  # every rank received halo agents
    assert sum(g[3] for g in gathered) > 0  # and agents changed owner
    got = np.empty_like(xyz)
    got[ids] = xyz
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    s.step(iters)
    assert np.array_equal(got, s.get()[0])


def oracle_engine(params):
    import oracle

    def engine(xyz, d, ghost):
        s = oracle.Sim(xyz, d, params)
        s.step(1)
        x = s.get()[0]
        x[ghost] = xyz[ghost]  # ghosts stay (their results are not the rank's)
        return x
    return engine


def run_local(pop, world, iters, engine):
    z = pop.xyz[:, 2]
    slabs = halo.Slabs(float(z.min()), float(z.max()), world)
    doms = [halo.SlabDomain(slabs, r, np.arange(pop.n), pop.xyz, pop.diameter) for r in range(world)]
    halo_in = moved = 0
    for _ in range(iters):
        for c in halo.step_local(doms, engine):
            halo_in += c["halo_in"]
            moved += c["migrated_out"]
    ids = np.concatenate([dm.ids for dm in doms])
    xyz = np.concatenate([dm.xyz for dm in doms])
    assert np.array_equal(np.sort(ids), np.arange(pop.n))
    got = np.empty_like(xyz)
    got[ids] = xyz
    return got, halo_in, moved


@pytest.mark.parametrize("world", [2, 3])
def test_local_exchange_matches_one_domain(orc, world):
    """The in-process exchange (every slab stepped by one process) equals a
    single domain bit for bit, with ghosts left in place."""
    import oracle
    pop = _population()
    got, halo_in, moved = run_local(pop, world, 4, oracle_engine(pop.params))
    assert halo_in > 0 and moved > 0
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    s.step(4)
    assert np.array_equal(got, s.get()[0])
