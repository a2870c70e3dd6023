"""Parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times (the force kernel, sort curve and re-sort
interval its tuning picks for each workload).

The oracle computes sampled outputs one by one:

- box indices are compared for every agent where the oracle's grid over the
  whole population finishes in seconds (8.4M agents), and otherwise for the
  agents of a region;
- a region's agents plus the agents that fix the grid (the per-axis minimum
  and maximum centres, the largest diameter) form a sub-population whose grid
  has the full population's origin, box length and dimensions (§4.4.3: they
  depend on those agents only), so the oracle's box indices of that
  sub-population are the full population's;
- an agent at least one largest diameter inside the region has all its
  interaction partners (Eq. 4.1: distance below the sum of the radii) in the
  sub-population, so its overlap pairs, its force and its displacement
  (which depends on its own force only) are those of the full population.

Forces are compared per agent as |F_gpu - F_oracle| / s_i <= 1e-5 (FP32-force
path) with s_i the magnitude sum of the agent's pair forces; box indices and
pair sets bit-exact.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads
from tests.pair_counts import check_nnz, overlap_counts

pytestmark = pytest.mark.gpu

TOL32 = 1e-5


def make_ctx(pops, **tuning):
    from paper_2503_10796_gb300 import binding
    params = [binding.make_params(p.params) for p in pops]
    total = sum(max(p.n, p.params.capacity) for p in pops) + 1024
    ctx = binding.Context(params, total)
    for s, p in enumerate(pops):
        ctx.set_agents(s, p.xyz, p.diameter)
    if tuning:
        ctx.set_tuning(**tuning)
    return ctx


def region_subset(xyz, d, lo, hi):
    """Ascending IDs of the agents with centres in [lo, hi) per axis, plus the
    agents that fix the grid; and the mask (over the returned IDs) of the
    agents at least max(d) inside the region."""
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    inside = np.ones(xyz.shape[0], bool)
    for a in range(3):
        inside &= (xyz[:, a] >= lo[a]) & (xyz[:, a] < hi[a])
    extra = [int(np.argmin(xyz[:, a])) for a in range(3)] + [int(np.argmax(xyz[:, a])) for a in range(3)]
    extra.append(int(np.argmax(d)))
    inside[extra] = True
    ids = np.flatnonzero(inside)
    m = float(d.max())
    sx = xyz[ids]
    core = np.all((sx >= lo + m) & (sx < hi - m), axis=1)
    return ids, core


def report(name, err):
    print(f"PARITY {name}: agents {err.size}, max {err.max():.3e}, p99.9 {np.quantile(err, 0.999):.3e}")


def rel_err(F, F0, smag):
    err = np.linalg.norm(F - F0, axis=1) / np.maximum(smag, 1e-300)
    zero = smag == 0
    err[zero] = np.linalg.norm(F[zero], axis=1)
    return err


def check_region(name, pop, box_gpu, pairs_gpu, F_gpu, nnz_gpu, ov_gpu, x_gpu, lo, hi):
    """Everything the oracle can fix from one region of the population."""
    import oracle
    ids, core = region_subset(pop.xyz, pop.diameter, lo, hi)
    assert core.sum() >= 200, (name, core.sum())
    sub = oracle.Sim(pop.xyz[ids], pop.diameter[ids], pop.params)
    # grid: same origin, box length and dimensions as the full population
    sbox, _, _ = sub.grid()
    assert np.array_equal(box_gpu[ids], sbox), name
    # overlap pairs with an endpoint in the core
    in_core = np.zeros(pop.n, bool)
    in_core[ids[core]] = True
    want = ids[sub.neighbors(-1.0)]
    want = want[in_core[want[:, 0]] | in_core[want[:, 1]]]
    got = pairs_gpu[in_core[pairs_gpu[:, 0]] | in_core[pairs_gpu[:, 1]]]
    assert got.shape == want.shape and np.array_equal(got, want), name
    # forces of the core agents; their overlap counts from the oracle's pairs
    loc = np.flatnonzero(core)
    F0, nnz0, smag = sub.forces(loc)
    g = ids[loc]
    err = rel_err(F_gpu[g], F0, smag)
    report(name, err)
    assert err.max() <= TOL32, (name, err.max())
    sub_pairs = sub.neighbors(-1.0)
    assert np.array_equal(ov_gpu[g], overlap_counts(ids.size, sub_pairs)[loc]), name
    check_nnz(nnz_gpu[g], nnz0, loc, pop.xyz[ids], pop.diameter[ids], sub_pairs, pop.params.k, pop.params.gamma)
    # one step: positions of the core agents
    sub.step(1)
    x_o, _, _ = sub.get()
    x_o = x_o[loc]
    fn = np.linalg.norm(F0, axis=1)
    flip = np.abs(fn - pop.params.adherence) <= 4 * TOL32 * np.maximum(smag, 1e-300)
    dx = np.abs(x_gpu[g] - x_o).max(axis=1)
    bound = pop.params.dt * (4 * TOL32 * smag) + 4 * np.spacing(np.abs(x_o).max(axis=1))
    bad = (dx > bound) & ~flip
    assert not bad.any(), (name, dx[bad][:5], bound[bad][:5])


def test_clustered_8M_full_size(orc):
    """64 Gaussian clusters of 131,072 agents: every box index against the
    oracle's grid over all 8.4M agents; sampled forces over the whole
    population; pairs, forces and positions of two regions (a cluster's
    dense centre and its flank)."""
    import oracle
    pop = workloads.clustered(sort_interval=10)
    ctx = make_ctx([pop], force_variant=5, sort_interval=10, sort_curve=0)
    try:
        box_gpu, ol, dims = ctx.grid(0)
        full = oracle.Sim(pop.xyz, pop.diameter, pop.params)
        obox, ool, odims = full.grid()
        assert np.array_equal(ol, ool) and np.array_equal(dims, odims)
        assert np.array_equal(box_gpu, obox)
        pairs_gpu = ctx.neighbors(0, -1.0)
        ctx.step(1)
        ctx.sync()
        F_gpu, nnz_gpu, st, ov_gpu = ctx.forces(0, overlaps=True)
        assert not st.any()
        x_gpu, _ = ctx.get_agents(0)
        rng = np.random.default_rng(5)
        sample = np.sort(rng.choice(pop.n, 20000, replace=False))
        F0, nnz0, smag = full.forces(sample)
        del full
        err = rel_err(F_gpu[sample], F0, smag)
        report("clustered_8M sampled", err)
        assert err.max() <= TOL32
        # every agent's overlap count from the (bit-exact, region-checked)
        # pair list; nnz of the sample against the oracle
        assert np.array_equal(ov_gpu, overlap_counts(pop.n, pairs_gpu))
        check_nnz(nnz_gpu[sample], nnz0, sample, pop.xyz, pop.diameter, pairs_gpu, pop.params.k, pop.params.gamma)
        c = pop.xyz[:131072].mean(axis=0)  # the first cluster's centre
        for name, off in (("clustered_8M centre", 0.0), ("clustered_8M flank", 300.0)):
            lo = c + np.array([off, 0.0, 0.0]) - 100.0
            check_region(name, pop, box_gpu, pairs_gpu, F_gpu, nnz_gpu, ov_gpu, x_gpu, lo, lo + 200.0)
    finally:
        ctx.close()


def test_clustered_8M_grid_reuse_full_size(orc):
    """The incremental grid at full size: after 52 iterations (settling,
    re-sorts at 0, 10, ..., 50, reused iterations between), the forces of an
    iteration that kept its grid, on 20,000 sampled agents, against the
    oracle on the same positions; the overlap and non-zero counts of the
    sample exact."""
    import oracle
    pop = workloads.clustered(sort_interval=10)
    ctx = make_ctx([pop], force_variant=5, sort_interval=10, sort_curve=0, box_scale_pct=125, grid_reuse=1)
    try:
        ctx.step(52)
        x, d = ctx.get_agents(0)
        b = ctx.counters()["grid_builds"]
        ctx.step(1)
        ctx.sync()
        assert ctx.counters()["grid_builds"] == b  # this iteration kept its grid
        F_gpu, nnz_gpu, _, ov_gpu = ctx.forces(0, overlaps=True)
        full = oracle.Sim(x, d, pop.params)
        rng = np.random.default_rng(6)
        sample = np.sort(rng.choice(pop.n, 20000, replace=False))
        F0, nnz0, smag = full.forces(sample)
        err = rel_err(F_gpu[sample], F0, smag)
        report("clustered_8M grid reuse sampled", err)
        assert err.max() <= TOL32
        pairs = full.neighbors(-1.0)
        assert np.array_equal(ov_gpu[sample], overlap_counts(pop.n, pairs)[sample])
        check_nnz(nnz_gpu[sample], nnz0, sample, x, d, pairs, pop.params.k, pop.params.gamma)
    finally:
        ctx.close()


def test_uniform_200M_full_size(orc):
    """200M agents at volume fraction 0.3: box indices, pairs, forces and
    positions of a corner region (at the grid origin) and a central one."""
    pop = workloads.uniform_fraction(200_000_000, sort_interval=10)
    ctx = make_ctx([pop], force_variant=5, sort_interval=-1, sort_curve=1)
    try:
        box_gpu, ol, dims = ctx.grid(0)
        assert np.array_equal(ol[:3], pop.xyz.min(axis=0)) and ol[3] == pop.diameter.max()
        pairs_gpu = ctx.neighbors(0, -1.0)
        ctx.step(1)
        ctx.sync()
        F_gpu, nnz_gpu, st, ov_gpu = ctx.forces(0, overlaps=True)
        assert not st.any()
        assert np.array_equal(ov_gpu, overlap_counts(pop.n, pairs_gpu))
        x_gpu, _ = ctx.get_agents(0)
        side = float(pop.xyz.max())
        for name, lo in (("uniform_200M corner", ol[:3]), ("uniform_200M centre", np.full(3, side / 2 - 75.0))):
            check_region(name, pop, box_gpu, pairs_gpu, F_gpu, nnz_gpu, ov_gpu, x_gpu, lo, lo + 150.0)
    finally:
        ctx.close()


def test_batched_sweep_256_full_size(orc):
    """256 simulations in one context: six of them (the smallest, the largest
    and four seeded picks) against the oracle in full."""
    import oracle
    pops = workloads.batched_sweep()
    ctx = make_ctx(pops, force_variant=5, sort_interval=5, sort_curve=0)
    try:
        sizes = np.array([p.n for p in pops])
        rng = np.random.default_rng(7)
        picks = sorted({int(sizes.argmin()), int(sizes.argmax())} | set(rng.choice(len(pops), 4, replace=False).tolist()))
        before = {}
        for s in picks:
            box, ol, dims = ctx.grid(s)
            before[s] = (box, ol, dims, ctx.neighbors(s, -1.0))
        ctx.step(1)
        ctx.sync()
        for s in picks:
            pop = pops[s]
            o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
            box, ol, dims, pairs = before[s]
            obox, ool, odims = o.grid()
            assert np.array_equal(ol, ool) and np.array_equal(dims, odims) and np.array_equal(box, obox), s
            assert np.array_equal(pairs, o.neighbors(-1.0)), s
            F0, nnz0, smag = o.forces()
            F, nnz, st, ov = ctx.forces(s, overlaps=True)
            err = rel_err(F, F0, smag)
            report(f"batched_sweep_256 sim {s} ({pop.n} agents)", err)
            assert err.max() <= TOL32, s
            assert np.array_equal(ov, overlap_counts(pop.n, pairs)), s
            check_nnz(nnz, nnz0, np.arange(pop.n), pop.xyz, pop.diameter, pairs, pop.params.k, pop.params.gamma)
            o.step(1)
            x_o, _, _ = o.get()
            x_g, _ = ctx.get_agents(s)
            fn = np.linalg.norm(F0, axis=1)
            flip = np.abs(fn - pop.params.adherence) <= 4 * TOL32 * np.maximum(smag, 1e-300)
            dx = np.abs(x_g - x_o).max(axis=1)
            bound = pop.params.dt * (4 * TOL32 * smag) + 4 * np.spacing(np.abs(x_o).max(axis=1))
            assert not ((dx > bound) & ~flip).any(), s
    finally:
        ctx.close()


def test_growth_division_65536_full_size(orc):
    """65,536 agents on the 32 x 32 x 64 lattice growing to the capacity of
    2,097,152: the agent count of every iteration and every diameter are
    exact.  Growth is synchronised and independent of position, so a
    2 x 2 x 2 oracle lattice with the same capacity factor gives the count
    (times 8,192) and the common diameter of each iteration.  Under the
    literal rates the division rounds fall at iterations 14, 26, 39, 51 and
    64 (counted from 0), so the capacity holds from the 65th iteration on."""
    import oracle
    pop = workloads.growth_division()
    small = workloads.growth_division(shape=(2, 2, 2))
    o = oracle.Sim(small.xyz, small.diameter, small.params)
    ctx = make_ctx([pop], force_variant=2, sort_interval=-1, sort_curve=0)
    try:
        rounds = []
        for t in range(66):
            n0 = o.n
            ctx.step(1)
            o.step(1)
            assert ctx.count(0) == 8192 * o.n, t
            if o.n != n0:
                rounds.append(t)
            if t % 8 == 7 or t in (14, 26, 39, 51, 64):
                _, d_o, _ = o.get()
                assert np.all(d_o == d_o[0])
                x_g, d_g = ctx.get_agents(0)
                assert np.all(d_g == d_o[0]), t
                assert np.isfinite(x_g).all(), t
        assert rounds == [14, 26, 39, 51, 64]
        assert ctx.count(0) == 2_097_152
    finally:
        ctx.close()
