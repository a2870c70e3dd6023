"""Parity of the sm_103a library (through the C ABI) with the CPU oracle.

Bit-exact: box indices, grid origin/length/dims, neighbor pair sets, the
per-agent overlap count (pairs with delta > 0) in both paths, nnz in the
FP64 path (in the FP32 path too, except at the force crossover).  Forces:
|F_gpu - F_oracle| / s_i <= 1e-12 (FP64 path) or 1e-5 (FP32-force path) with
s_i = sum_j (k delta + gamma sqrt(r delta)), the magnitude sum of agent i's
pair forces.
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads
from tests.pair_counts import check_nnz, overlap_counts

VARIANTS = range(7)

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


def ctx_for(pop_or_list, max_total=None, **kw):
    from paper_2503_10796_gb300 import binding
    pops = pop_or_list if isinstance(pop_or_list, list) else [pop_or_list]
    params = [binding.make_params(p.params, **kw) for p in pops]
    total = max_total or sum(max(p.n, p.params.capacity) for p in pops) + 16
    ctx = binding.Context(params, total)
    for s, p in enumerate(pops):
        ctx.set_agents(s, p.xyz, p.diameter)
    return ctx


def orc_for(pop, **kw):
    import oracle
    return oracle.Sim(pop.xyz, pop.diameter, pop.params, **kw)


def small_pops():
    return [
        workloads.plain_fp64(),                                                  # 4096, full size
        workloads.Population(*workloads.uniform_cube(1025, 90.0, seed=3)),       # ragged tail
        workloads.clustered(n_clusters=5, per_cluster=700, side=600.0, sigma=25.0, seed=2),
        workloads.Population(*workloads.uniform_cube(3, 12.0, seed=1)),
    ]


@pytest.mark.parametrize("k", range(4))
def test_grid_bit_exact(orc, k):
    pop = small_pops()[k]
    ctx = ctx_for(pop)
    box, ol, dims = ctx.grid(0)
    obox, ool, odims = orc_for(pop).grid()
    assert np.array_equal(ol, ool)
    assert np.array_equal(dims, odims)
    assert np.array_equal(box, obox)


def test_grid_boundary_cases(orc):
    """Centers exactly on box boundaries, and one ulp on either side."""
    L = 10.0
    base = np.array([[0.0, 0, 0], [40.0, 40, 40]])
    pts = [base]
    for c in (10.0, 20.0, 30.0):
        for v in (c, np.nextafter(c, 0), np.nextafter(c, 100)):
            pts.append(np.array([[v, 5.0, 5.0], [5.0, v, 5.0], [5.0, 5.0, v]]))
    xyz = np.concatenate(pts)
    pop = workloads.Population(xyz, np.full(len(xyz), 1.0), workloads.SimParams(box_length=L))
    ctx = ctx_for(pop)
    box, ol, dims = ctx.grid(0)
    obox, ool, odims = orc_for(pop).grid()
    assert np.array_equal(box, obox) and np.array_equal(dims, odims)


def boundary_values(rng, origin, L, span, n_edges):
    """Coordinates on box boundaries origin + k L, one to three ulps either
    side of them, and uniform ones, none below the origin."""
    k = np.sort(rng.choice(span, min(span, n_edges), replace=False)).astype(np.float64)
    edge = origin + k * L
    pts = [edge]
    for u in (1, 2, 3):
        lo = edge.copy()
        hi = edge.copy()
        for _ in range(u):
            lo = np.nextafter(lo, -np.inf)
            hi = np.nextafter(hi, np.inf)
        pts += [lo, hi]
    v = np.concatenate(pts + [origin + rng.uniform(0, span * L, 3 * n_edges)])
    v = np.clip(v, origin, None)
    v[0] = origin  # the grid origin is the smallest coordinate
    return v


def boundary_population(origin, L, span, const_x=None):
    """Boundary coordinates along a wide axis (x, or y when x is held at
    const_x) and along narrow ones (20 boxes), so that the dense box table
    stays small."""
    rng = np.random.default_rng(1)
    wide = boundary_values(rng, origin, L, span, 600)
    m = wide.size
    narrow = [rng.choice(boundary_values(rng, origin, L, 20, 20), m) for _ in range(2)]
    for v in narrow:
        v[0] = origin
    if const_x is None:
        xyz = np.stack([wide, narrow[0], narrow[1]], axis=1)
    else:
        xyz = np.stack([np.full(m, const_x), wide, narrow[0]], axis=1)
    # a clamp of one box length keeps the table's allowance for movement small
    return workloads.Population(xyz, np.full(m, 0.5 * L), workloads.SimParams(box_length=L, max_displacement=L))


@pytest.mark.parametrize("origin,L,span,const_x", [(-123456.789, 10.3, 3000, None), (9.87654321e8, 0.7, 5000, None),
                                                   (-2.5e-3, 1e-3, 40000, None), (0.0, 10.0, 3000, 1e28)])
def test_grid_boundaries_far_from_zero(orc, origin, L, span, const_x):
    """Box indices on and next to box boundaries with the origin far from
    zero and grids thousands of boxes wide; with x at 1e28 (box length 10)
    the coordinates are too large for the integer grid frame and the FP64
    route computes every index."""
    pop = boundary_population(origin, L, span, const_x)
    ctx = ctx_for(pop)
    box, ol, dims = ctx.grid(0)
    obox, ool, odims = orc_for(pop).grid()
    assert np.array_equal(ol, ool) and np.array_equal(dims, odims)
    assert np.array_equal(box, obox)


@pytest.mark.parametrize("shift", [1.0e6, -3.0e7])
def test_forces_far_from_zero(orc, shift):
    """Clusters a million and thirty million length units from zero: the
    box-relative FP32 records keep the force within the FP32 tolerance."""
    base = small_pops()[2]
    pop = workloads.Population(base.xyz + shift, base.diameter, workloads.SimParams(precision=1))
    check_forces(pop, 1)


@pytest.mark.parametrize("k", range(3))
@pytest.mark.parametrize("radius", [-1.0, 6.0, 25.0])
def test_neighbor_pairs_bit_exact(orc, k, radius):
    pop = small_pops()[k]
    ctx = ctx_for(pop)
    got = ctx.neighbors(0, radius)
    want = orc_for(pop).neighbors(radius)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def check_counts(pop, ov, nnz, o, nnz0, ids=None):
    """Overlap counts exact; nnz exact except at the force crossover."""
    pairs = o.neighbors(-1.0)
    want = overlap_counts(pop.n, pairs)
    ids = np.arange(pop.n) if ids is None else ids
    assert np.array_equal(ov, want[ids]), np.flatnonzero(ov != want[ids])[:10]
    check_nnz(nnz, nnz0, ids, pop.xyz, pop.diameter, pairs, pop.params.k, pop.params.gamma)


def check_forces(pop, precision, orc_sim=None, variant=None):
    ctx = ctx_for(pop, precision=precision)
    if variant is not None:
        ctx.set_tuning(force_variant=variant)
    o = orc_sim or orc_for(pop)
    F0, nnz0, smag = o.forces()
    ctx.step(1)
    ctx.sync()
    F, nnz, st, ov = ctx.forces(0, overlaps=True)
    assert not st.any()
    scale = np.maximum(smag, 1e-300)
    err = np.linalg.norm(F - F0, axis=1) / scale
    err[smag == 0] = np.linalg.norm(F[smag == 0], axis=1)
    assert err.max() <= TOL[precision], (err.max(), np.argmax(err))
    if precision == 0:
        assert np.array_equal(nnz, nnz0)
    check_counts(pop, ov, nnz, o, nnz0)
    return ctx, o, err


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("k", range(4))
def test_one_step_forces_and_positions(orc, precision, k):
    pop = small_pops()[k]
    ctx, o, err = check_forces(pop, precision)
    o.step(1)
    x_o, _, _ = o.get()
    x_g, d_g = ctx.get_agents(0)
    assert np.array_equal(d_g, pop.diameter)
    F0, D0, _, _, _ = o.last()
    # agents whose |F| sits within the tolerance of the adherence threshold
    # may take the other side of the decision
    _, _, smag = orc_for(pop).forces()
    fn = np.linalg.norm(F0, axis=1)
    flip = np.abs(fn - pop.params.adherence) <= 4 * TOL[precision] * np.maximum(smag, 1e-300)
    dx = np.abs(x_g - x_o).max(axis=1)
    bound = pop.params.dt * (4 * TOL[precision] * smag) + 4 * np.spacing(np.abs(x_o).max(axis=1))
    bad = (dx > bound) & ~flip
    assert not bad.any(), (dx[bad][:5], bound[bad][:5])


@pytest.mark.parametrize("precision", [0, 1])
def test_multi_step_trajectory(orc, precision):
    """10 iterations of the plain workload: position error against the oracle."""
    pop = workloads.plain_fp64()
    ctx = ctx_for(pop, precision=precision)
    o = orc_for(pop)
    ctx.step(10)
    o.step(10)
    x_g, _ = ctx.get_agents(0)
    x_o, _, _ = o.get()
    err = np.abs(x_g - x_o).max()
    L = pop.diameter.max()
    if precision == 0:
        assert err <= 1e-9 * L, err
    else:
        assert err <= 1e-4 * L, err


def test_fp32_error_growth_is_bounded(orc):
    """FP32-force path over 40 iterations of the plain workload: the position
    error against the oracle at every fifth iteration, reported, and bounded
    well below a box length (agents whose force sits at the adherence
    threshold may take the other branch, a jump of up to dt * |F|)."""
    pop = workloads.plain_fp64()
    ctx = ctx_for(pop, precision=1)
    o = orc_for(pop)
    L = pop.diameter.max()
    errs = []
    for t in range(8):
        ctx.step(5)
        o.step(5)
        x_g, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        e = np.abs(x_g - x_o).max(axis=1)
        errs.append((5 * (t + 1), e.max() / L, np.quantile(e, 0.999) / L))
    print("GROWTH " + " ".join(f"t={t}: max {a:.2e} p99.9 {b:.2e}" for t, a, b in errs))
    assert errs[1][1] <= 1e-4
    assert all(a <= 1e-2 for _, a, _ in errs)


@pytest.mark.parametrize("precision,variant", [(0, 0), (1, 1), (1, 5), (1, 6)])
def test_cluster_statistics_match_oracle(orc, precision, variant):
    """20 iterations of five dense clusters with static detection on: per
    cluster the radius of gyration, and over all agents the mean contact
    count and the static fraction, within 1% of the oracle's."""
    base = small_pops()[2]
    p = workloads.SimParams(precision=precision, detect_static=1)
    pop = workloads.Population(base.xyz, base.diameter, p, "clusters_static")
    ctx = ctx_for(pop)
    ctx.set_tuning(force_variant=variant)
    o = orc_for(pop)
    ctx.step(20)
    o.step(20)
    x_g, _ = ctx.get_agents(0)
    x_o, _, _ = o.get()
    _, nnz_g, st_g = ctx.forces(0)
    _, _, nnz_o, st_o, _ = o.last()
    for c in range(5):
        sl = slice(700 * c, 700 * (c + 1))
        rg = [np.sqrt(((x[sl] - x[sl].mean(axis=0)) ** 2).sum(axis=1).mean()) for x in (x_g, x_o)]
        assert abs(rg[0] - rg[1]) <= 0.01 * rg[1], (c, rg)
    assert abs(nnz_g.mean() - nnz_o.mean()) <= 0.01 * nnz_o.mean()
    assert abs(st_g.mean() - st_o.astype(bool).mean()) <= 0.01
    print(f"CLUSTERS precision {precision}: contacts {nnz_g.mean():.4f} / {nnz_o.mean():.4f}, "
          f"static {st_g.mean():.4f} / {st_o.astype(bool).mean():.4f}")


def test_two_sphere_closed_form_on_gpu(orc):
    for precision in (0, 1):
        pop = workloads.Population(np.array([[0.0, 0, 0], [8.0, 0, 0]]), np.array([10.0, 10.0]))
        ctx = ctx_for(pop, precision=precision)
        ctx.step(1)
        F, nnz, _ = ctx.forces(0)
        want = 4.0 - np.sqrt(5.0)
        assert F[0, 0] == pytest.approx(-want, rel=TOL[precision])
        assert nnz.tolist() == [1, 1]


def test_tiny_overlaps_keep_relative_accuracy(orc):
    """Pairs whose overlap is 1e-3 .. 1e-9 of the radius: the FP32 path must
    still meet its relative tolerance (the sqrt(r delta) term dominates)."""
    rng = np.random.default_rng(0)
    rows, diam = [], []
    for k, depth in enumerate(10.0 ** -rng.uniform(1, 9, 200)):
        c = np.array([k * 40.0, 0.0, 0.0])
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        d1, d2 = rng.uniform(8, 12, 2)
        rows += [c, c + u * ((d1 + d2) / 2 - depth)]
        diam += [d1, d2]
    pop = workloads.Population(np.array(rows), np.array(diam))
    check_forces(pop, 1)
    check_forces(pop, 0)


def test_empty_and_single(orc):
    from paper_2503_10796_gb300 import binding
    ctx = binding.Context([binding.make_params(), binding.make_params()], 8)
    ctx.set_agents(0, np.zeros((0, 3)), np.zeros(0))
    ctx.set_agents(1, np.array([[1.0, 2.0, 3.0]]), np.array([10.0]))
    ctx.step(3)
    ctx.sync()
    x, d = ctx.get_agents(0)
    assert x.shape == (0, 3)
    x, d = ctx.get_agents(1)
    assert x.tolist() == [[1.0, 2.0, 3.0]]
    assert ctx.neighbors(1, -1.0).shape == (0, 2)


def test_invalid_input_is_rejected(orc):
    from paper_2503_10796_gb300 import binding
    ctx = binding.Context(binding.make_params(), 8)
    with pytest.raises(binding.BdmError) as e:
        ctx.set_agents(0, np.array([[np.nan, 0, 0]]), np.array([1.0]))
    assert e.value.code == -1
    with pytest.raises(binding.BdmError) as e:
        ctx.set_agents(0, np.array([[0.0, 0, 0]]), np.array([-1.0]))
    assert e.value.code == -1
    with pytest.raises(binding.BdmError) as e:
        ctx.set_agents(0, np.zeros((9, 3)), np.ones(9))
    assert e.value.code == -4
    with pytest.raises(binding.BdmError) as e:
        ctx.step(1)  # nothing set yet
    assert e.value.code == -7
    # rejected calls reserved nothing: the full capacity is still free
    xyz = np.arange(24, dtype=np.float64).reshape(8, 3) * 10.0
    ctx.set_agents(0, xyz, np.ones(8))
    got, d = ctx.get_agents(0)
    assert np.array_equal(got, xyz) and np.array_equal(d, np.ones(8))
    xo = np.zeros((8, 3)); do = np.zeros(8)
    assert ctx.get_agents(0, out=(xo, do))[0] is xo
    assert np.array_equal(xo, xyz)


def test_batched_simulations_match_single_ones(orc):
    pops = workloads.batched_sweep(n_sims=6, lo=50, hi=3000, seed=4)
    ctx = ctx_for(pops)
    ctx.step(5)
    for s, p in enumerate(pops):
        single = ctx_for(p)
        single.step(5)
        a, _ = ctx.get_agents(s)
        b, _ = single.get_agents(0)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-4)
        o = orc_for(p)
        o.step(5)
        x_o, _, _ = o.get()
        np.testing.assert_allclose(a, x_o, rtol=0, atol=1e-3)


@pytest.mark.parametrize("precision,variant", [(0, 0), (1, 1), (1, 5), (1, 6)])
def test_static_skip_matches_no_skip(orc, precision, variant):
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    pop = workloads.Population(xyz, d, workloads.SimParams(dt=0.05, precision=precision))
    on = ctx_for(pop, detect_static=1)
    off = ctx_for(pop, detect_static=0)
    on.set_tuning(force_variant=variant)
    off.set_tuning(force_variant=variant)
    o = orc_for(pop, detect_static=1)
    n_static = 0
    for _ in range(15):
        on.step(1); off.step(1); o.step(1)
        _, _, st = on.forces(0)
        n_static += int(st.sum())
    a, _ = on.get_agents(0)
    b, _ = off.get_agents(0)
    c, _, _ = o.get()
    if precision == 0:
        # FP64 path: on, off and the oracle bit for bit
        assert np.array_equal(a, b) and np.array_equal(a, c)
    else:
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-3)
        np.testing.assert_allclose(a, c, rtol=0, atol=1e-3)
    assert n_static > 0
    assert on.stats(0)["static_agents"] >= 0


def morton_codes(box, dims):
    import oracle
    nx, ny = int(dims[0]), int(dims[1])
    return np.array([oracle.interleave(3, [b % nx, (b // nx) % ny, b // (nx * ny)]) for b in box], np.uint64)


@pytest.mark.parametrize("n_sims", [1, 3])
def test_morton_sort_orders_storage(orc, n_sims):
    """With no movement (huge adherence) the grid after the step equals the
    grid the re-sort used: storage must then be in Morton order of boxes,
    ties in any order, and hold every agent once."""
    pops = [workloads.clustered(n_clusters=3, per_cluster=900 + 37 * s, side=500.0, sigma=30.0, seed=s)
            for s in range(n_sims)]
    ctx = ctx_for(pops, adherence=1e9, sort_interval=1)
    ctx.step(1)
    for s, p in enumerate(pops):
        order = ctx.storage_order(s)
        assert np.array_equal(np.sort(order), np.arange(p.n))
        box, ol, dims = ctx.grid(s)
        codes = morton_codes(box, dims)
        seq = codes[order]
        assert np.all(seq[1:] >= seq[:-1])
        o = orc_for(p)
        want = codes[o.morton_agent_order()]
        assert np.array_equal(seq, want)
        x, _ = ctx.get_agents(s)
        assert np.array_equal(x, p.xyz)


def test_later_resorts_keep_morton_order(orc):
    """Re-sorts after the first permute the storage into the cell order; with
    no movement the storage stays in Morton order of boxes, every agent once,
    and the results stay the same."""
    pop = workloads.clustered(n_clusters=3, per_cluster=1200, side=500.0, sigma=30.0, seed=6)
    ctx = ctx_for(pop, adherence=1e9, sort_interval=1)
    ctx.step(4)
    order = ctx.storage_order(0)
    assert np.array_equal(np.sort(order), np.arange(pop.n))
    box, _, dims = ctx.grid(0)
    codes = morton_codes(box, dims)
    seq = codes[order]
    assert np.array_equal(seq, codes[orc_for(pop).morton_agent_order()])
    x, _ = ctx.get_agents(0)
    assert np.array_equal(x, pop.xyz)


@pytest.mark.parametrize("precision", [0, 1])
def test_sorting_does_not_change_results(orc, precision):
    pop = workloads.plain_fp64()
    a = ctx_for(pop, precision=precision, sort_interval=3)
    b = ctx_for(pop, precision=precision, sort_interval=0)
    a.step(7)
    b.step(7)
    xa, _ = a.get_agents(0)
    xb, _ = b.get_agents(0)
    tol = 1e-9 if precision == 0 else 1e-4
    np.testing.assert_allclose(xa, xb, rtol=0, atol=tol * pop.diameter.max())
    assert not np.array_equal(a.storage_order(0), np.arange(pop.n))


@pytest.mark.parametrize("precision", [0, 1])
def test_growth_division_matches_oracle(orc, precision):
    """Synchronised growth and division on a small lattice: the agent count
    of every iteration, the diameters and volumes are exact; positions stay
    within the trajectory tolerance."""
    pop = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=precision)
    ctx = ctx_for(pop)
    o = orc_for(pop)
    for t in range(45):
        ctx.step(1)
        o.step(1)
        assert ctx.count(0) == o.n, t
    x_g, d_g = ctx.get_agents(0)
    x_o, d_o, _ = o.get()
    assert np.array_equal(d_g, d_o)
    tol = 1e-9 if precision == 0 else 1e-3
    np.testing.assert_allclose(x_g, x_o, rtol=0, atol=tol * d_o.max())
    st = ctx.stats(0)
    assert st["iterations"] == 45 and st["agents"] == o.n


def test_division_stops_at_capacity(orc):
    pop = workloads.growth_division(shape=(3, 3, 3), cap_factor=1)
    pop.params.capacity = 40  # 27 agents; only 13 may divide
    ctx = ctx_for(pop)
    o = orc_for(pop)
    ctx.step(16)
    o.step(16)
    assert ctx.count(0) == o.n == 40
    x_g, d_g = ctx.get_agents(0)
    x_o, d_o, _ = o.get()
    assert np.array_equal(d_g, d_o)
    np.testing.assert_allclose(x_g, x_o, rtol=0, atol=1e-3)


def dense_clump(n=300, side=20.0, seed=11):
    """Heavily overlapping agents: each has far more than 16 partners, so the
    queues of the deferred and symmetric walks overflow and their second,
    evaluating walks take over."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, side, (n, 3))
    d = rng.uniform(8.0, 12.0, n)
    return workloads.Population(xyz, d, workloads.SimParams(precision=1), "dense_clump")


def test_deferred_walk_equals_direct_loop(orc):
    """The deferred walk (queue and overflow path), the symmetric half-stencil
    walk (queue and overflow path) and the direct loop find the same
    interacting pairs (nnz equal) and agree to FP32 rounding.  Bitwise
    equality is not expected: agents of one box are placed in the order their
    atomic count arrived, and the symmetric walk adds pair forces by atomics,
    which both set the order of the FP32 sum."""
    for pop in (workloads.clustered(n_clusters=4, per_cluster=2000, side=500.0, sigma=30.0, seed=2),
                dense_clump()):
        _, _, smag = orc_for(pop).forces()
        out = []
        for variant in (1, 0, 2, 3, 4, 5, 6):
            ctx = ctx_for(pop, precision=1, sort_interval=1)
            ctx.set_tuning(force_variant=variant)
            ctx.step(1)
            ctx.sync()
            F, nnz, _, ov = ctx.forces(0, overlaps=True)
            out.append((F, nnz, ov))
        F0, nnz0, ov0 = out[0]
        for F, nnz, ov in out[1:]:
            assert np.array_equal(nnz, nnz0)
            assert np.array_equal(ov, ov0)
            err = np.linalg.norm(F - F0, axis=1) / np.maximum(smag, 1e-30)
            assert err.max() <= 1e-5, err.max()


def crowded_boxes(n=6000, seed=12):
    """Many agents per box (about 30, like the late growth workload) and a
    ragged tail: lanes of the stream kernel with long segments."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, 60.0, (n, 3))
    d = rng.uniform(8.0, 12.0, n)
    return workloads.Population(xyz, d, workloads.SimParams(precision=1), "crowded")


@pytest.mark.parametrize("variant", VARIANTS)
def test_force_variants_match_oracle(orc, variant):
    """Every force-kernel variant of the FP32 path meets the tolerance, with
    exact overlap counts."""
    for pop in (workloads.plain_fp64(seed=5),
                workloads.clustered(n_clusters=4, per_cluster=2000, side=500.0, sigma=30.0, seed=1),
                dense_clump(), crowded_boxes(),
                workloads.Population(*workloads.uniform_cube(33, 40.0, seed=2)),
                workloads.Population(*workloads.uniform_cube(1, 10.0, seed=2))):
        ctx = ctx_for(pop, precision=1, sort_interval=1)
        ctx.set_tuning(force_variant=variant)
        o = orc_for(pop)
        F0, nnz0, smag = o.forces()
        ctx.step(1)
        ctx.sync()
        F, nnz, _, ov = ctx.forces(0, overlaps=True)
        err = np.linalg.norm(F - F0, axis=1) / np.maximum(smag, 1e-300)
        err[smag == 0] = np.linalg.norm(F[smag == 0], axis=1)
        assert err.max() <= TOL[1], (variant, err.max())
        check_counts(pop, ov, nnz, o, nnz0)


def test_autotune_restores_state(orc):
    pop = workloads.clustered(n_clusters=4, per_cluster=3000, side=600.0, sigma=30.0, seed=3)
    a = ctx_for(pop, sort_interval=10)
    b = ctx_for(pop, sort_interval=10)
    a.step(3)
    b.step(3)
    x_before, _ = a.get_agents(0)
    chosen = a.autotune(3)
    assert chosen["force_variant"] in VARIANTS
    assert chosen["sort_interval"] in (-1, 0, 5, 10, 25) and chosen["iter_batch"] in (1, 4, 10)
    x_after, _ = a.get_agents(0)
    assert np.array_equal(x_before, x_after)
    assert a.stats(0)["iterations"] == 3
    a.step(4)
    b.step(4)
    xa, _ = a.get_agents(0)
    xb, _ = b.get_agents(0)
    np.testing.assert_allclose(xa, xb, rtol=0, atol=1e-3)


def test_row_major_curve_orders_storage(orc):
    pop = workloads.clustered(n_clusters=3, per_cluster=1500, side=500.0, sigma=30.0, seed=8)
    ctx = ctx_for(pop, adherence=1e9, sort_interval=1)
    ctx.set_tuning(force_variant=0, sort_interval=1, sort_curve=1)
    ctx.step(1)
    order = ctx.storage_order(0)
    box, _, _ = ctx.grid(0)
    seq = box[order]
    assert np.all(seq[1:] >= seq[:-1])
    assert np.array_equal(np.sort(order), np.arange(pop.n))


def test_box_overflow_is_reported(orc):
    """More agents in one box than a table word counts: the step reports
    BDM_E_CAPACITY instead of silently dropping agents."""
    from paper_2503_10796_gb300 import binding
    rng = np.random.default_rng(0)
    xyz = rng.uniform(0.0, 50.0, (1100, 3))
    pop = workloads.Population(xyz, np.full(1100, 1.0), workloads.SimParams(box_length=60.0))
    ctx = ctx_for(pop)
    ctx.step(1)
    with pytest.raises(binding.BdmError) as e:
        ctx.sync()
    assert e.value.code == -4


def test_update_agents_keeps_the_simulation(orc):
    """bdm_update_agents moves agents by ID without resetting the simulation:
    the forces of the next step equal those of a fresh context set to the
    same positions, IDs are kept, and n must match the agent count."""
    from paper_2503_10796_gb300 import binding
    pop = workloads.clustered(n_clusters=3, per_cluster=3000, side=500.0, sigma=30.0, seed=4)
    a = ctx_for(pop, sort_interval=1)
    a.step(3)
    x, d = a.get_agents(0)
    rng = np.random.default_rng(1)
    x2 = x + rng.uniform(-0.5, 0.5, x.shape)
    a.update_agents(0, x2)                       # positions only: diameters kept
    assert a.stats(0)["iterations"] == 3
    got, gd = a.get_agents(0)
    assert np.array_equal(got, x2) and np.array_equal(gd, d)
    b = ctx_for(workloads.Population(x2, d, pop.params, "moved"), sort_interval=1)
    a.step(1)
    b.step(1)
    a.sync()
    b.sync()
    Fa, na, _ = a.forces(0)
    Fb, nb, _ = b.forces(0)
    _, _, smag = orc_for(workloads.Population(x2, d, pop.params, "moved")).forces()
    assert np.array_equal(na, nb)
    err = np.linalg.norm(Fa - Fb, axis=1) / np.maximum(smag, 1e-30)
    assert err.max() <= 2e-5
    with pytest.raises(binding.BdmError) as e:
        a.update_agents(0, x2[:-1])
    assert e.value.code == -1
    bad = x2.copy()
    bad[7, 1] = np.inf
    with pytest.raises(binding.BdmError) as e:
        a.update_agents(0, bad)
    assert e.value.code == -1


def test_update_agents_with_static_detection_and_diameters(orc):
    """Agents moved by bdm_update_agents count as changed: with static
    detection on, the trajectory equals the one without it (the oracle's
    static rules are exact), and new diameters change the grid's box length."""
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    pop = workloads.Population(xyz, d, workloads.SimParams(dt=0.05, precision=0))
    on = ctx_for(pop, detect_static=1)
    off = ctx_for(pop, detect_static=0)
    for _ in range(6):
        on.step(1)
        off.step(1)
    x, dd = on.get_agents(0)
    x2 = x.copy()
    x2[:5] += 0.25                      # disturb a few agents between steps
    on.update_agents(0, x2)
    off.update_agents(0, x2)
    for _ in range(6):
        on.step(1)
        off.step(1)
    a, _ = on.get_agents(0)
    b, _ = off.get_agents(0)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-10)
    # larger diameters: the next grid's box length is the new largest one
    d2 = dd * 1.1
    on.update_agents(0, a, d2)
    on.step(1)
    on.sync()
    st = on.stats(0)
    assert st["origin_len"][3] == d2.max()
    _, gd = on.get_agents(0)
    assert np.array_equal(gd, d2)


# ---- FP64 path: bit-exact trajectories -------------------------------------
# The FP64 path evaluates every definition with IEEE operations in the
# oracle's order and adds each agent's pair forces in ascending partner ID,
# so positions, static flags and nnz equal the oracle's bit for bit at every
# iteration, whatever the storage order.

def fp64_scenes():
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    base = small_pops()[2]
    return [
        ("plain_4096", workloads.plain_fp64()),
        ("perturbed", workloads.Population(xyz, d, workloads.SimParams(dt=0.05, precision=0))),
        ("clusters", workloads.Population(base.xyz, base.diameter, workloads.SimParams(precision=0))),
        ("dense_clump", workloads.Population(dense_clump().xyz, dense_clump().diameter,
                                             workloads.SimParams(precision=0))),
    ]


@pytest.mark.parametrize("static", [0, 1])
@pytest.mark.parametrize("sort_interval", [0, 3])
@pytest.mark.parametrize("scene", range(4))
def test_fp64_trajectory_bit_exact(orc, static, sort_interval, scene):
    name, pop = fp64_scenes()[scene]
    ctx = ctx_for(pop, precision=0, detect_static=static, sort_interval=sort_interval)
    o = orc_for(pop, detect_static=static)
    n_static = 0
    for t in range(16):
        ctx.step(1)
        o.step(1)
        x_g, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        assert np.array_equal(x_g, x_o), (name, t, np.abs(x_g - x_o).max())
        F_g, nnz_g, st_g = ctx.forces(0)
        F_o, _, nnz_o, st_o, _ = o.last()
        assert np.array_equal(st_g, st_o), (name, t)
        assert np.array_equal(nnz_g, np.minimum(nnz_o, 255)), (name, t)  # stored saturated at 255
        assert np.array_equal(F_g, F_o), (name, t)
        n_static += int(st_g.sum())
    if static and name in ("perturbed", "clusters"):
        assert n_static > 0
    print(f"FP64 BITWISE {name} static={static} sort={sort_interval}: 16 iterations, {n_static} static agent-steps")


def test_fp64_growth_division_bit_exact(orc):
    pop = workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)
    ctx = ctx_for(pop)
    o = orc_for(pop)
    for t in range(45):
        ctx.step(1)
        o.step(1)
        x_g, d_g = ctx.get_agents(0)
        x_o, d_o, _ = o.get()
        assert np.array_equal(d_g, d_o) and np.array_equal(x_g, x_o), t


def test_fp64_crowd_beyond_the_sort_capacity(orc):
    """760 agents of diameter 9.5-10.5 in a cube of side 5: every pair
    overlaps (the cube's diagonal is 8.7), so each agent has 759 partners,
    more than the FP64 overflow kernel sorts in shared memory (704), and its
    selection of the next partner ID takes over; the forces are still added
    in ascending partner ID, bit for bit the oracle's."""
    rng = np.random.default_rng(21)
    xyz = 100.0 + rng.uniform(0.0, 5.0, (760, 3))
    d = rng.uniform(9.5, 10.5, 760)
    pop = workloads.Population(xyz, d, workloads.SimParams(precision=0, dt=0.01))
    ctx = ctx_for(pop)
    o = orc_for(pop)
    for t in range(3):
        ctx.step(1)
        o.step(1)
        x_g, _ = ctx.get_agents(0)
        x_o, _, _ = o.get()
        assert np.array_equal(x_g, x_o), t
        F_g, nnz_g, _, ov = ctx.forces(0, overlaps=True)
        F_o, _, nnz_o, _, _ = o.last()
        assert np.array_equal(F_g, F_o) and np.array_equal(nnz_g, np.minimum(nnz_o, 255)), t
        if t == 0:
            assert (ov == 759).all()


def test_fp64_batched_simulations_bit_exact(orc):
    pops = workloads.batched_sweep(n_sims=5, lo=50, hi=3000, seed=9, precision=0)
    ctx = ctx_for(pops)
    ctx.step(8)
    for s, p in enumerate(pops):
        o = orc_for(p)
        o.step(8)
        x_o, _, _ = o.get()
        x_g, _ = ctx.get_agents(s)
        assert np.array_equal(x_g, x_o), s
