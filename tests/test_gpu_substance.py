"""A substance inside bdm_step (bdm_set_substance): after the mechanical
step of every iteration the agents secrete (Algorithm 6), the substance
takes one step of Eq 4.3, and the agents follow its gradient (Algorithm 7).

Against the oracle composed in the same order (its mechanical iteration,
then secretion, diffusion and chemotaxis, the moved positions set back):
positions, forces, nnz and concentrations bit for bit in the FP64 path, with
static detection off and on, with grid reuse, and in the in-place context.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu

LO = np.array([-100.0, -100.0, -100.0])
H = np.array([10.0, 12.0, 9.0])
SHAPE = (90, 70, 80)  # (nz, ny, nx): the grid covers every cluster
NU, MU, Q, W = 2.0, 0.05, 1.0, 0.3


def scene(**kw):
    base = workloads.clustered(n_clusters=5, per_cluster=600, side=500.0, sigma=20.0, seed=8)
    return workloads.Population(base.xyz, base.diameter, workloads.SimParams(precision=0, **kw))


def oracle_iteration(o, u, dt):
    import oracle
    o.step(1)
    x, _, _ = o.get()
    oracle.secrete(u, LO, H, x, Q)
    oracle.diffuse(u, H, NU, MU, dt, 1)
    o.set_positions(oracle.chemotaxis(u, LO, H, x, W))


@pytest.mark.parametrize("mode", ["copy", "static", "reuse", "inplace"])
def test_substance_in_step_bit_exact(orc, mode):
    import oracle
    from paper_2503_10796_gb300 import binding
    kw = {"static": dict(detect_static=1), "inplace": dict(execution_context=1)}.get(mode, {})
    pop = scene(**kw)
    ctx = binding.Context(binding.make_params(pop.params), pop.n + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    if mode == "reuse":
        t = ctx.get_tuning()
        t.update(box_scale_pct=150, grid_reuse=1)
        ctx.set_tuning(**t)
    u0 = np.random.default_rng(3).uniform(0.0, 1.0, SHAPE)
    ctx.set_substance(0, u0, LO, H, NU, MU, Q, W)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    u = u0.copy()
    for t in range(8):
        ctx.step(1)
        oracle_iteration(o, u, pop.params.dt)
        x, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        assert np.array_equal(x, x_o), (mode, t, np.abs(x - x_o).max())
        assert np.array_equal(ctx.get_substance(0), u), (mode, t)
        F, nnz, st = ctx.forces(0)
        F_o, _, nnz_o, st_o, _ = o.last()
        assert np.array_equal(F, F_o) and np.array_equal(nnz, np.minimum(nnz_o, 255)), (mode, t)
        assert np.array_equal(st, st_o), (mode, t)
    assert not np.array_equal(x, pop.xyz)
    # removed again: the next iteration is the mechanical step alone
    ctx.clear_substance(0)
    ctx.step(1)
    o.step(1)
    assert np.array_equal(ctx.get_agents(0)[0], o.get()[0])


def test_substance_errors(orc):
    from paper_2503_10796_gb300 import binding
    pop = scene()
    ctx = binding.Context(binding.make_params(pop.params), pop.n + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    with pytest.raises(binding.BdmError) as e:
        ctx.get_substance(0)
    assert e.value.code in (-7, -1)
    with pytest.raises(binding.BdmError) as e:
        ctx.set_substance(0, np.zeros(SHAPE), LO, H, -1.0, MU, Q, W)
    assert e.value.code == -1
    closed = workloads.Population(np.array([[5.0, 5.0, 5.0]]), np.array([1.0]),
                                  workloads.SimParams(precision=0, boundary=1, bound_min=0.0, bound_max=10.0))
    c2 = binding.Context(binding.make_params(closed.params), 8)
    c2.set_agents(0, closed.xyz, closed.diameter)
    with pytest.raises(binding.BdmError) as e:
        c2.set_substance(0, np.zeros((2, 2, 2)), [0, 0, 0], [5, 5, 5], NU, MU, Q, W)
    assert e.value.code == -1


def oracle_kinds_iteration(o, us, kinds, dt):
    """The oracle's iteration with a substance per kind (each kind's agents
    secrete into and follow their own substance)."""
    import oracle
    o.step(1)
    x, _, _ = o.get()
    for k, u in us.items():
        m = kinds == k
        oracle.secrete(u, LO, H, x[m], Q)
        oracle.diffuse(u, H, NU, MU, dt, 1)
        x[m] = oracle.chemotaxis(u, LO, H, x[m], W)
    o.set_positions(x)


def test_two_kinds_soma_clustering_bit_exact(orc):
    """Two cell kinds at random, each secreting its own substance and
    following it (the soma-clustering benchmark of §4.6)."""
    import oracle
    from paper_2503_10796_gb300 import binding
    rng = np.random.default_rng(12)
    xyz = rng.uniform(0.0, 500.0, (3000, 3))
    d = rng.uniform(8.0, 12.0, 3000)
    pop = workloads.Population(xyz, d, workloads.SimParams(precision=0))
    kinds = (rng.random(pop.n) < 0.5).astype(np.uint8)
    ctx = binding.Context(binding.make_params(pop.params), pop.n + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    ctx.set_agent_kinds(0, kinds)
    us = {k: rng.uniform(0.0, 1.0, SHAPE) for k in (0, 1)}
    for k, u in us.items():
        ctx.set_substance(0, u, LO, H, NU, MU, Q, W, kind=k)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    for t in range(6):
        ctx.step(1)
        oracle_kinds_iteration(o, us, kinds, pop.params.dt)
        assert np.array_equal(ctx.get_agents(0)[0], o.get()[0]), t
        for k, u in us.items():
            assert np.array_equal(ctx.get_substance(0, kind=k), u), (t, k)


def test_kinds_follow_division_and_removal(orc):
    import oracle
    from paper_2503_10796_gb300 import binding
    pop = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)
    kinds = (np.arange(pop.n) % 2).astype(np.uint8)
    ctx = binding.Context(binding.make_params(pop.params), pop.params.capacity + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    ctx.set_agent_kinds(0, kinds)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    ctx.step(15)  # every agent divides at iteration 14: daughter n + i of mother i
    o.step(15)
    assert ctx.count(0) == o.n == 2 * pop.n
    kinds = np.concatenate([kinds, kinds])
    # removal renumbers by the swaps of §5.3.2: track the survivors' kinds by position
    x_before, _, _ = o.get()
    gone = np.random.default_rng(2).choice(o.n, 40, replace=False)
    ctx.remove_agents(0, gone)
    o.remove(gone)
    x_after, _, _ = o.get()
    where = {tuple(p): i for i, p in enumerate(x_before)}
    kinds = kinds[[where[tuple(p)] for p in x_after]]
    us = {1: np.random.default_rng(4).uniform(0.0, 1.0, SHAPE)}
    ctx.set_substance(0, us[1], LO, H, NU, MU, Q, W, kind=1)
    for t in range(4):
        ctx.step(1)
        oracle_kinds_iteration(o, us, kinds, pop.params.dt)
        assert np.array_equal(ctx.get_agents(0)[0], o.get()[0]), t
    assert np.array_equal(ctx.get_substance(0, kind=1), us[1])
