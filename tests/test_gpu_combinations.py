"""Seeded combinations of the step's options against the oracle, FP64 path
(bit for bit): space boundary (open, closed, toroidal), static detection,
re-sort interval, growth and division, the in-place context, grid reuse and
a substance inside the step, drawn within the combinations the library
accepts.  Every iteration compares positions, diameters, forces, nnz and
static flags (and the substance's concentrations)."""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu

SEEDS = range(18)


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    boundary = int(rng.integers(0, 3))
    grows = bool(rng.random() < 0.3)
    inplace = bool(rng.random() < 0.3) and not grows
    static = bool(rng.random() < 0.4) and not inplace
    if seed % 3 == 0:  # every third draw keeps the grid between builds
        boundary, grows, inplace, static = boundary % 2, False, False, False
    reuse = seed % 3 == 0
    substance = bool(rng.random() < 0.3) and boundary == 0
    sort_interval = int(rng.choice([0, 3, 5]))
    size = 90.0
    n = int(rng.integers(800, 2500))
    if grows:
        base = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)
        xyz = np.mod(base.xyz, size) if boundary else base.xyz
        d = base.diameter
        p = base.params
    else:
        xyz = rng.uniform(0.0, size, (n, 3))
        d = rng.uniform(8.0, 12.0, n)
        p = workloads.SimParams(precision=0)
    p.boundary, p.bound_min, p.bound_max = boundary, 0.0, size
    p.detect_static = int(static)
    p.sort_interval = sort_interval
    p.dt = float(rng.choice([0.01, 0.05]))
    p.execution_context = int(inplace)
    return workloads.Population(xyz, d, p), dict(boundary=boundary, grows=grows, inplace=inplace, static=static,
                                                 reuse=reuse, substance=substance, sort=sort_interval)


@pytest.mark.parametrize("seed", SEEDS)
def test_option_combinations_bit_exact(orc, seed):
    import oracle
    from paper_2503_10796_gb300 import binding
    pop, opt = draw(seed)
    ctx = binding.Context(binding.make_params(pop.params), max(pop.n, pop.params.capacity) + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    if opt["reuse"]:
        t = ctx.get_tuning()
        t.update(box_scale_pct=150, grid_reuse=1)
        ctx.set_tuning(**t)
    lo, h, shape = np.array([-20.0, -20.0, -20.0]), np.array([8.0, 8.0, 8.0]), (20, 20, 20)
    u = None
    if opt["substance"]:
        u = np.random.default_rng(seed).uniform(0.0, 1.0, shape)
        ctx.set_substance(0, u, lo, h, 1.0, 0.02, 1.0, 0.4)
        u = u.copy()
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    for t in range(8):
        ctx.step(1)
        o.step(1)
        if u is not None:
            x, _, _ = o.get()
            oracle.secrete(u, lo, h, x, 1.0)
            oracle.diffuse(u, h, 1.0, 0.02, pop.params.dt, 1)
            o.set_positions(oracle.chemotaxis(u, lo, h, x, 0.4))
        x_g, d_g = ctx.get_agents(0)
        x_o, d_o, _ = o.get()
        assert ctx.count(0) == o.n, (opt, t)
        assert np.array_equal(d_g, d_o) and np.array_equal(x_g, x_o), (opt, t, np.abs(x_g - x_o).max())
        F, nnz, st = ctx.forces(0)
        F_o, _, nnz_o, st_o, _ = o.last()
        assert np.array_equal(F, F_o), (opt, t)
        assert np.array_equal(nnz, np.minimum(nnz_o, 255)) and np.array_equal(st, st_o), (opt, t)
        if u is not None:
            assert np.array_equal(ctx.get_substance(0), u), (opt, t)
