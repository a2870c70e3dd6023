"""The in-place execution context (§5.2) on the GPU against the oracle.

The kernel runs one launch per box colour and a group of lanes per box (8
for large populations, forced here by a test hook, or a whole warp), and
commits each agent's displacement before the box's next agent.  It follows the
oracle's order (colour, box index, agent ID) and evaluates every definition
in FP64 in the oracle's order of operations, so positions, forces and nnz
equal the oracle's bit for bit at every iteration: in open space, on an odd
torus (a third colour at the seam), in a closed box, for a crowd beyond the
kernel's sorted partner list, with growth and division, and in a context of
several simulations.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu


def ctx_for(pops, narrow=False, **kw):
    """narrow: the boxes on groups of 8 lanes (the form for large
    populations; a test hook) instead of a warp per box."""
    from paper_2503_10796_gb300 import binding
    pops = pops if isinstance(pops, list) else [pops]
    ctx = binding.Context([binding.make_params(p.params, execution_context=1, **kw) for p in pops],
                          sum(max(p.n, p.params.capacity) for p in pops) + 16)
    for s, p in enumerate(pops):
        ctx.set_agents(s, p.xyz, p.diameter)
    if narrow:
        t = ctx.get_tuning()
        t.update(test_flags=2)
        ctx.set_tuning(**t)
    return ctx


def orc_for(pop):
    import oracle
    return oracle.Sim(pop.xyz, pop.diameter, pop.params, execution_context=1)


def scenes():
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    rng = np.random.default_rng(3)
    txyz = rng.uniform(0.0, 90.0, (2500, 3))
    td = rng.uniform(8.0, 12.0, 2500)
    cxyz = rng.uniform(0.0, 90.0, (2500, 3))
    cd = rng.uniform(8.0, 12.0, 2500)
    clump = rng.uniform(0.0, 20.0, (300, 3))
    clump_d = rng.uniform(8.0, 12.0, 300)
    base = workloads.clustered(n_clusters=5, per_cluster=700, side=600.0, sigma=25.0, seed=2)
    return [
        ("perturbed", workloads.Population(xyz, d, workloads.SimParams(dt=0.05, precision=0))),
        ("clusters", workloads.Population(base.xyz, base.diameter, workloads.SimParams(precision=0))),
        ("torus_odd", workloads.Population(txyz, td, workloads.SimParams(precision=0, boundary=2, bound_min=0.0,
                                                                        bound_max=90.0))),
        ("closed", workloads.Population(cxyz, cd, workloads.SimParams(precision=0, boundary=1, bound_min=0.0,
                                                                     bound_max=90.0, dt=0.05))),
        ("dense_clump", workloads.Population(clump, clump_d, workloads.SimParams(precision=0))),
    ]


@pytest.mark.parametrize("narrow", [False, True])
@pytest.mark.parametrize("sort_interval", [0, 3])
@pytest.mark.parametrize("scene", range(5))
def test_inplace_trajectory_bit_exact(orc, scene, sort_interval, narrow):
    name, pop = scenes()[scene]
    ctx = ctx_for(pop, narrow=narrow, sort_interval=sort_interval)
    o = orc_for(pop)
    for t in range(10):
        ctx.step(1)
        o.step(1)
        x, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        assert np.array_equal(x, x_o), (name, t, np.abs(x - x_o).max())
        F, nnz, st = ctx.forces(0)
        F_o, _, nnz_o, _, _ = o.last()
        assert np.array_equal(F, F_o), (name, t)
        assert np.array_equal(nnz, np.minimum(nnz_o, 255)), (name, t)
        assert not st.any()
    # the in-place trajectory is not the copy context's
    import oracle
    c = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    c.step(10)
    assert not np.array_equal(c.get()[0], x), name


@pytest.mark.parametrize("narrow,n", [(True, 8), (True, 9), (True, 40), (True, 100), (True, 200),
                                      (False, 32), (False, 33), (False, 100), (False, 300), (False, 600)])
def test_inplace_crowd_beyond_the_partner_list(orc, narrow, n):
    """Every agent of a tight clump overlaps all others.  With groups of 8
    lanes per box: up to 8 agents of a box keep their IDs in the group's
    lanes (9 take the loop over the box); up to 64 overlapping partners are
    sorted in shared memory (40); beyond that (100), or beyond the 128
    candidates the filter keeps (200), the selection loop adds the partners
    one ID after the other.  With a warp per box the limits are 32 IDs, 256
    partners and 512 candidates (32, 33, 100, 300, 600)."""
    rng = np.random.default_rng(9)
    pop = workloads.Population(100.0 + rng.uniform(0.0, 5.0, (n, 3)), rng.uniform(9.5, 10.5, n),
                               workloads.SimParams(precision=0, dt=0.01))
    ctx = ctx_for(pop, narrow=narrow)
    o = orc_for(pop)
    for t in range(3):
        ctx.step(1)
        o.step(1)
        assert np.array_equal(ctx.get_agents(0)[0], o.get()[0]), (n, t)
        F, nnz, _ = ctx.forces(0)
        F_o, _, nnz_o, _, _ = o.last()
        assert np.array_equal(F, F_o) and np.array_equal(nnz, np.minimum(nnz_o, 255)), (n, t)
        if t == 0:  # the first agent of the iteration met the whole clump unmoved
            _, _, _, ov = ctx.forces(0, overlaps=True)
            assert ov.max() == n - 1, (n, ov.max())


@pytest.mark.parametrize("narrow", [False, True])
def test_inplace_growth_and_batched_sims_bit_exact(orc, narrow):
    pop = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)
    ctx = ctx_for(pop, narrow=narrow)
    o = orc_for(pop)
    for t in range(30):
        ctx.step(1)
        o.step(1)
        assert ctx.count(0) == o.n, t
    x, d = ctx.get_agents(0)
    x_o, d_o, _ = o.get()
    assert np.array_equal(d, d_o) and np.array_equal(x, x_o)
    pops = workloads.batched_sweep(n_sims=4, lo=50, hi=2000, seed=11, precision=0)
    ctx = ctx_for(pops, narrow=narrow)
    ctx.step(6)
    for s, p in enumerate(pops):
        o = orc_for(p)
        o.step(6)
        assert np.array_equal(ctx.get_agents(s)[0], o.get()[0]), s


def test_inplace_parameters_are_checked(orc):
    from paper_2503_10796_gb300 import binding
    pop = workloads.plain_fp64(n=100, precision=0)
    for kw in (dict(precision=1), dict(detect_static=1), dict(execution_context=2)):
        p = dict(execution_context=1)
        p.update(kw)
        with pytest.raises(binding.BdmError) as e:
            binding.Context(binding.make_params(pop.params, **p), 128)
        assert e.value.code == -1
    with pytest.raises(binding.BdmError) as e:
        binding.Context([binding.make_params(pop.params, execution_context=1), binding.make_params(pop.params)], 256)
    assert e.value.code == -1
