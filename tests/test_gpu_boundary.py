"""Space boundary conditions (§4.4.11) and agent removal (§5.3.2) on the
GPU, against the oracle.

FP64 path: trajectories, static flags and nnz bit for bit (the oracle's
order of operations, minimum images on a torus, clamps and wraps included).
FP32-force path: forces within the parity tolerance, overlap counts exact.
Neighbour queries on a torus: pair sets bit-exact.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads
from tests.pair_counts import overlap_counts

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def ctx_for(pop, **kw):
    from paper_2503_10796_gb300 import binding
    ctx = binding.Context(binding.make_params(pop.params, **kw), max(pop.n, pop.params.capacity) + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    return ctx


def orc_for(pop, **kw):
    import oracle
    return oracle.Sim(pop.xyz, pop.diameter, pop.params, **kw)


def torus_pop(n=2500, size=90.0, seed=3, **kw):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, size, (n, 3))
    d = rng.uniform(8.0, 12.0, n)
    return workloads.Population(xyz, d, workloads.SimParams(boundary=2, bound_min=0.0, bound_max=size, **kw))


def closed_pop(n=2500, size=90.0, seed=4, **kw):
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, size, (n, 3))
    d = rng.uniform(8.0, 12.0, n)
    # dt 0.05: agents at the walls get pushed into them
    return workloads.Population(xyz, d, workloads.SimParams(boundary=1, bound_min=0.0, bound_max=size, dt=0.05,
                                                            **kw))


@pytest.mark.parametrize("static", [0, 1])
@pytest.mark.parametrize("make", [torus_pop, closed_pop])
def test_fp64_boundary_trajectory_bit_exact(orc, make, static):
    pop = make(precision=0, detect_static=static)
    ctx = ctx_for(pop)
    o = orc_for(pop)
    box, ol, dims = ctx.grid(0)
    obox, ool, odims = o.grid()
    assert np.array_equal(box, obox) and np.array_equal(ol, ool) and np.array_equal(dims, odims)
    for t in range(12):
        ctx.step(1)
        o.step(1)
        x, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        assert np.array_equal(x, x_o), t
        _, nnz, st = ctx.forces(0)
        _, _, nnz_o, st_o, _ = o.last()
        assert np.array_equal(st, st_o) and np.array_equal(nnz, np.minimum(nnz_o, 255)), t
    lo, hi = pop.params.bound_min, pop.params.bound_max
    assert (x >= lo).all() and ((x < hi).all() if pop.params.boundary == 2 else (x <= hi).all())


@pytest.mark.parametrize("make", [torus_pop, closed_pop])
def test_fp32_boundary_forces(orc, make):
    pop = make(precision=1)
    ctx = ctx_for(pop)
    o = orc_for(pop)
    F0, nnz0, smag = o.forces()
    ctx.step(1)
    ctx.sync()
    F, nnz, _, ov = ctx.forces(0, overlaps=True)
    err = np.linalg.norm(F - F0, axis=1) / np.maximum(smag, 1e-300)
    err[smag == 0] = np.linalg.norm(F[smag == 0], axis=1)
    assert err.max() <= TOL[1], err.max()
    assert np.array_equal(ov, overlap_counts(pop.n, o.neighbors(-1.0)))
    # several iterations stay close to the oracle
    ctx.step(9)
    o.step(10)
    x, _ = ctx.get_agents(0)
    x_o, _, _ = o.get()
    dx = np.abs(x - x_o)
    if pop.params.boundary == 2:
        dx = np.minimum(dx, pop.params.bound_max - pop.params.bound_min - dx)
    assert dx.max() <= 1e-4 * pop.diameter.max()


@pytest.mark.parametrize("radius", [-1.0, 7.5, 20.0])
def test_torus_neighbors_bit_exact(orc, radius):
    pop = torus_pop(precision=0)
    ctx = ctx_for(pop)
    assert np.array_equal(ctx.neighbors(0, radius), orc_for(pop).neighbors(radius))


def test_seam_pair_on_gpu(orc):
    for precision in (0, 1):
        pop = workloads.Population(np.array([[1.0, 50.0, 50.0], [97.0, 50.0, 50.0]]), np.array([10.0, 10.0]),
                                   workloads.SimParams(boundary=2, bound_min=0.0, bound_max=100.0, dt=1.0,
                                                       precision=precision))
        ctx = ctx_for(pop)
        ctx.step(1)
        F, nnz, _ = ctx.forces(0)
        fn = 12.0 - np.sqrt(15.0)
        assert F[0, 0] == pytest.approx(fn, rel=TOL[precision]) and nnz.tolist() == [1, 1]
        x, _ = ctx.get_agents(0)
        assert x[0, 0] == pytest.approx(4.0) and x[1, 0] == pytest.approx(94.0)


@pytest.mark.parametrize("boundary,size", [(1, 40.0), (2, 40.0)])
def test_growth_in_a_bounded_space_bit_exact(orc, boundary, size):
    base = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)
    xyz = np.mod(base.xyz, size)
    p = base.params
    p.boundary, p.bound_min, p.bound_max = boundary, 0.0, size
    pop = workloads.Population(xyz, base.diameter, p)
    ctx = ctx_for(pop)
    o = orc_for(pop)
    for t in range(30):
        ctx.step(1)
        o.step(1)
        assert ctx.count(0) == o.n, t
    x, d = ctx.get_agents(0)
    x_o, d_o, _ = o.get()
    assert np.array_equal(d, d_o) and np.array_equal(x, x_o)


def test_narrow_torus_is_reported(orc):
    from paper_2503_10796_gb300 import binding
    pop = workloads.Population(np.array([[1.0, 1.0, 1.0], [20.0, 20.0, 20.0]]), np.array([10.0, 10.0]),
                               workloads.SimParams(boundary=2, bound_min=0.0, bound_max=25.0))
    ctx = ctx_for(pop)
    ctx.step(1)
    with pytest.raises(binding.BdmError) as e:
        ctx.sync()
    assert e.value.code == -1


def test_positions_outside_the_space_are_rejected(orc):
    from paper_2503_10796_gb300 import binding
    for boundary, v in ((1, 100.5), (2, 100.0)):
        pop = workloads.Population(np.array([[v, 5.0, 5.0]]), np.array([1.0]),
                                   workloads.SimParams(boundary=boundary, bound_min=0.0, bound_max=100.0))
        ctx = binding.Context(binding.make_params(pop.params), 4)
        with pytest.raises(binding.BdmError) as e:
            ctx.set_agents(0, pop.xyz, pop.diameter)
        assert e.value.code == -1


@pytest.mark.parametrize("precision", [0, 1])
def test_removal_matches_oracle(orc, precision):
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    pop = workloads.Population(xyz, d, workloads.SimParams(dt=0.05, precision=precision, detect_static=1,
                                                           sort_interval=3))
    ctx = ctx_for(pop)
    o = orc_for(pop)
    ctx.step(5)
    o.step(5)
    rng = np.random.default_rng(8)
    gone = rng.choice(pop.n, pop.n // 3, replace=False)
    ctx.remove_agents(0, gone)
    o.remove(gone)
    assert ctx.count(0) == o.n
    x, dd = ctx.get_agents(0)
    x_o, d_o, _ = o.get()
    assert np.array_equal(dd, d_o)
    tol = 0.0 if precision == 0 else 1e-4 * d.max()
    assert np.abs(x - x_o).max() <= tol
    for t in range(8):
        ctx.step(1)
        o.step(1)
        x, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        if precision == 0:
            assert np.array_equal(x, x_o), t
            _, _, st = ctx.forces(0)
            _, _, _, st_o, _ = o.last()
            assert np.array_equal(st, st_o), t
        else:
            assert np.abs(x - x_o).max() <= 1e-3 * d.max(), t


def test_removal_edge_cases(orc):
    from paper_2503_10796_gb300 import binding
    pop = workloads.plain_fp64(n=300, precision=0)
    ctx = ctx_for(pop)
    for bad in ([300], [-1], [5, 5]):
        with pytest.raises(binding.BdmError) as e:
            ctx.remove_agents(0, bad)
        assert e.value.code == -1
    assert ctx.count(0) == 300
    ctx.remove_agents(0, [])
    assert ctx.count(0) == 300
    ctx.remove_agents(0, [6, 1, 4] + list(range(7, 300)))  # leaves 0, 2, 3, 5 -> 0, 5, 2, 3
    x, _ = ctx.get_agents(0)
    assert np.array_equal(x, pop.xyz[[0, 5, 2, 3]])
    ctx.step(2)
    ctx.remove_agents(0, [0, 1, 2, 3])
    assert ctx.count(0) == 0
    ctx.step(1)
    ctx.sync()
