"""Incremental grid (tuning grid_reuse): iterations keep the last build's grid
while every agent stays within the skin (L - largest diameter) / 2 of its
registered box, with the moved agents' records rewritten in place.

The pair set of every iteration is still the geometric one, so:
- FP64 trajectories, forces and nnz equal the oracle's (which rebuilds every
  iteration) bit for bit, while fewer grids are built than iterations run;
- FP32 forces of every iteration meet the parity tolerance against the
  oracle's forces on the same positions, with exact overlap counts;
- changes between steps (agents moved by the host, a neighbour query, a
  checkpoint restore) make the next iteration rebuild, and results stay exact.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads
from tests.pair_counts import overlap_counts

pytestmark = pytest.mark.gpu


def clusters(precision, seed=2, sort_interval=0):
    base = workloads.clustered(n_clusters=5, per_cluster=700, side=600.0, sigma=25.0, seed=seed)
    return workloads.Population(base.xyz, base.diameter,
                                workloads.SimParams(precision=precision, sort_interval=sort_interval))


def reuse_ctx(pops, box_scale_pct=150):
    from paper_2503_10796_gb300 import binding
    pops = pops if isinstance(pops, list) else [pops]
    ctx = binding.Context([binding.make_params(p.params) for p in pops], sum(p.n for p in pops) + 16)
    for s, p in enumerate(pops):
        ctx.set_agents(s, p.xyz, p.diameter)
    t = ctx.get_tuning()
    t.update(box_scale_pct=box_scale_pct, grid_reuse=1)
    ctx.set_tuning(**t)
    return ctx


@pytest.mark.parametrize("sort_interval", [0, 4])
def test_fp64_trajectory_bit_exact_with_fewer_builds(orc, sort_interval):
    import oracle
    pop = clusters(0, sort_interval=sort_interval)
    ctx = reuse_ctx(pop)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    b0 = ctx.counters()["grid_builds"]
    iters = 30
    for t in range(iters):
        ctx.step(1)
        o.step(1)
        x, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        assert np.array_equal(x, x_o), (t, np.abs(x - x_o).max())
        F, nnz, _ = ctx.forces(0)
        F_o, _, nnz_o, _, _ = o.last()
        assert np.array_equal(F, F_o) and np.array_equal(nnz, np.minimum(nnz_o, 255)), t
    builds = ctx.counters()["grid_builds"] - b0
    assert 1 <= builds < iters
    print(f"GRID REUSE FP64 sort={sort_interval}: {builds} builds in {iters} iterations")


def test_fp32_forces_every_iteration(orc):
    import oracle
    pop = clusters(1, seed=3)
    ctx = reuse_ctx(pop)
    b0 = ctx.counters()["grid_builds"]
    for t in range(20):
        x, d = ctx.get_agents(0)
        ref = oracle.Sim(x, d, pop.params)
        F0, _, smag = ref.forces()
        ctx.step(1)
        F, _, _, ov = ctx.forces(0, overlaps=True)
        err = np.linalg.norm(F - F0, axis=1) / np.maximum(smag, 1e-300)
        err[smag == 0] = np.linalg.norm(F[smag == 0], axis=1)
        assert err.max() <= 1e-5, (t, err.max())
        assert np.array_equal(ov, overlap_counts(pop.n, ref.neighbors(-1.0))), t
    assert ctx.counters()["grid_builds"] - b0 < 20


def test_changes_between_steps_rebuild(orc):
    import oracle
    pop = clusters(0, seed=4)
    ctx = reuse_ctx(pop)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    ctx.step(5)
    o.step(5)
    # move one agent far into another cluster, by the host
    x, _ = ctx.get_agents(0)
    x[7] = x[pop.n - 1] + 1.0
    ctx.update_agents(0, x)
    o = oracle.Sim(x, pop.diameter, pop.params)
    b = ctx.counters()["grid_builds"]
    ctx.step(1)
    o.step(1)
    assert ctx.counters()["grid_builds"] == b + 1
    assert np.array_equal(ctx.get_agents(0)[0], o.get()[0])
    # a neighbour query between steps
    ctx.neighbors(0, 20.0)
    ctx.step(3)
    o.step(3)
    assert np.array_equal(ctx.get_agents(0)[0], o.get()[0])
    # a checkpoint restore
    state = ctx.get_state(0)
    ctx.step(4)
    ctx.set_state(0, state)
    ctx.step(4)
    o.step(4)
    assert np.array_equal(ctx.get_agents(0)[0], o.get()[0])


def test_batched_simulations_bit_exact(orc):
    import oracle
    pops = workloads.batched_sweep(n_sims=4, lo=200, hi=3000, seed=13, precision=0)
    ctx = reuse_ctx(pops, box_scale_pct=125)
    ctx.step(12)
    for s, p in enumerate(pops):
        o = oracle.Sim(p.xyz, p.diameter, p.params)
        o.step(12)
        assert np.array_equal(ctx.get_agents(s)[0], o.get()[0]), s


def test_reuse_needs_eligible_simulations(orc):
    from paper_2503_10796_gb300 import binding
    for kw in (dict(detect_static=1), dict(growth_rate=4000.0, divide_volume=900.0),
               dict(boundary=2, bound_min=0.0, bound_max=200.0)):
        pop = workloads.plain_fp64(n=100, precision=0)
        ctx = binding.Context(binding.make_params(pop.params, **kw), 256)
        t = ctx.get_tuning()
        t.update(grid_reuse=1)
        with pytest.raises(binding.BdmError) as e:
            ctx.set_tuning(**t)
        assert e.value.code == -1


@pytest.mark.parametrize("precision", [0, 1])
def test_closed_box_walls_with_reuse(orc, precision):
    """Agents pushed into the walls of a closed box: clamped moves take the
    exact record path; FP64 trajectories stay bit-exact, FP32 forces of
    every iteration meet the tolerance with exact overlap counts."""
    import oracle
    rng = np.random.default_rng(17)
    xyz = rng.uniform(0.0, 90.0, (2500, 3))
    d = rng.uniform(8.0, 12.0, 2500)
    pop = workloads.Population(xyz, d, workloads.SimParams(precision=precision, boundary=1, bound_min=0.0,
                                                           bound_max=90.0, dt=0.05))
    ctx = reuse_ctx(pop)
    b0 = ctx.counters()["grid_builds"]
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    for t in range(12):
        x, dd = ctx.get_agents(0)
        if precision == 1:
            ref = oracle.Sim(x, dd, pop.params)
            F0, _, smag = ref.forces()
        ctx.step(1)
        if precision == 0:
            o.step(1)
            assert np.array_equal(ctx.get_agents(0)[0], o.get()[0]), t
        else:
            F, _, _, ov = ctx.forces(0, overlaps=True)
            err = np.linalg.norm(F - F0, axis=1) / np.maximum(smag, 1e-300)
            err[smag == 0] = np.linalg.norm(F[smag == 0], axis=1)
            assert err.max() <= 1e-5, (t, err.max())
            assert np.array_equal(ov, overlap_counts(pop.n, ref.neighbors(-1.0))), t
    x, _ = ctx.get_agents(0)
    assert (x >= 0.0).all() and (x <= 90.0).all()
    assert ctx.counters()["grid_builds"] - b0 <= 12


def test_reuse_switched_off_and_on(orc):
    """Turning grid reuse off after reused iterations (and on again) keeps the
    trajectory exact: the next iteration builds its grid."""
    import oracle
    pop = clusters(0, seed=6)
    ctx = reuse_ctx(pop)
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    for reuse in (1, 0, 1, 0):
        t = ctx.get_tuning()
        t.update(grid_reuse=reuse)
        ctx.set_tuning(**t)
        b = ctx.counters()["grid_builds"]
        ctx.step(6)
        o.step(6)
        assert np.array_equal(ctx.get_agents(0)[0], o.get()[0]), reuse
        builds = ctx.counters()["grid_builds"] - b
        assert builds == 6 if reuse == 0 else builds < 6, (reuse, builds)
