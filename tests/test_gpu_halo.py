"""The library under the slab decomposition: halo agents as ghosts
(bdm_set_ghosts), read-only neighbours that bdm_step does not move, grow or
divide.

- Every slab of a domain stepped by its own context (halo.LibraryEngine,
  the messages handed over in this process by halo.step_local) equals one
  domain run by the oracle, bit for bit in the FP64 path.
- Ghost semantics on one context against the oracle with the ghosts put back
  after each iteration; growth leaves ghosts alone; flags survive a
  checkpoint and are reset by bdm_set_agents.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import halo, workloads

pytestmark = pytest.mark.gpu


def population(precision=0):
    xyz, d = workloads.uniform_cube(2500, 70.0, seed=4)
    return workloads.Population(xyz, d, workloads.SimParams(precision=precision))


def run_slabs(pop, world, iters):
    z = pop.xyz[:, 2]
    slabs = halo.Slabs(float(z.min()), float(z.max()), world)
    doms = [halo.SlabDomain(slabs, r, np.arange(pop.n), pop.xyz, pop.diameter) for r in range(world)]
    engines = [halo.LibraryEngine(pop.params, pop.n + 16) for _ in range(world)]
    halo_in = moved = 0
    for _ in range(iters):
        # each rank with its own context
        counts = halo.step_local(doms, _per_rank(engines))
        halo_in += sum(c["halo_in"] for c in counts)
        moved += sum(c["migrated_out"] for c in counts)
    ids = np.concatenate([dm.ids for dm in doms])
    xyz = np.concatenate([dm.xyz for dm in doms])
    assert np.array_equal(np.sort(ids), np.arange(pop.n))  # every agent on exactly one rank
    got = np.empty_like(xyz)
    got[ids] = xyz
    return got, halo_in, moved


def _per_rank(engines):
    """An engine that hands the k-th call of an iteration to rank k's context
    (step_local advances the ranks in order)."""
    calls = iter(engines)

    def engine(xyz, d, ghost):
        return next(calls)(xyz, d, ghost)
    return engine


@pytest.mark.parametrize("world", [2, 3])
def test_library_slabs_match_one_domain_bit_exact(orc, world):
    import oracle
    pop = population(0)
    got, halo_in, moved = run_slabs(pop, world, 4)
    assert halo_in > 0 and moved > 0
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    s.step(4)
    assert np.array_equal(got, s.get()[0])


def test_library_slabs_fp32_within_tolerance(orc):
    import oracle
    pop = population(1)
    got, _, _ = run_slabs(pop, 3, 4)
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    s.step(4)
    assert np.abs(got - s.get()[0]).max() <= 1e-4 * pop.diameter.max()


def test_ghosts_stay_and_others_match_oracle(orc):
    """With a third of the agents as ghosts, ten iterations equal the oracle
    stepping everything and putting the ghosts back after each iteration."""
    import oracle
    from paper_2503_10796_gb300 import binding
    pop = population(0)
    ghost = np.random.default_rng(5).random(pop.n) < 1 / 3
    ctx = binding.Context(binding.make_params(pop.params), pop.n + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    ctx.set_ghosts(0, ghost)
    x_o = pop.xyz.copy()
    for t in range(10):
        ctx.step(1)
        s = oracle.Sim(x_o, pop.diameter, pop.params)
        s.step(1)
        x_new = s.get()[0]
        x_new[ghost] = x_o[ghost]
        x_o = x_new
        x, _ = ctx.get_agents(0)
        assert np.array_equal(x, x_o), t
    assert np.array_equal(x[ghost], pop.xyz[ghost])
    assert not np.array_equal(x[~ghost], pop.xyz[~ghost])
    # the flags travel with a checkpoint, and bdm_set_agents clears them
    state = ctx.get_state(0)
    b = binding.Context(binding.make_params(pop.params), pop.n + 16)
    b.set_state(0, state)
    b.step(1)
    ctx.step(1)
    assert np.array_equal(b.get_agents(0)[0], ctx.get_agents(0)[0])
    ctx.set_agents(0, pop.xyz, pop.diameter)
    ctx.step(1)
    assert not np.array_equal(ctx.get_agents(0)[0][ghost], pop.xyz[ghost])


def test_ghosts_neither_grow_nor_divide(orc):
    from paper_2503_10796_gb300 import binding
    pop = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)
    ghost = np.zeros(pop.n, bool)
    ghost[::2] = True
    ctx = binding.Context(binding.make_params(pop.params), pop.params.capacity + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    ctx.set_ghosts(0, ghost)
    ctx.step(16)  # past the first division round (iteration 14)
    x, d = ctx.get_agents(0)
    assert ctx.count(0) == pop.n + int((~ghost).sum())  # only the ordinary agents divided
    assert np.array_equal(d[: pop.n][ghost], pop.diameter[ghost])
    assert np.array_equal(x[: pop.n][ghost], pop.xyz[ghost])


def test_ghost_mask_errors(orc):
    from paper_2503_10796_gb300 import binding
    pop = workloads.plain_fp64(n=100, precision=0)
    ctx = binding.Context(binding.make_params(pop.params), 128)
    with pytest.raises(binding.BdmError) as e:
        ctx.set_ghosts(0, np.zeros(100, bool))  # no agents set yet
    assert e.value.code == -7
    ctx.set_agents(0, pop.xyz, pop.diameter)
    with pytest.raises(binding.BdmError) as e:
        ctx.set_ghosts(0, np.zeros(99, bool))
    assert e.value.code == -1
