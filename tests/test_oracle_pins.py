"""Pins of the CPU oracle against values the thesis prints, closed forms,
invariants and brute force.  CPU only."""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def brute_pairs(xyz, d, radius):
    """All pairs i < j by exhaustive O(N^2) search (no grid)."""
    n = xyz.shape[0]
    i, j = np.triu_indices(n, 1)
    dx = xyz[i, 0] - xyz[j, 0]
    dy = xyz[i, 1] - xyz[j, 1]
    dz = xyz[i, 2] - xyz[j, 2]
    s = (dx * dx + dy * dy) + dz * dz
    if radius >= 0:
        hit = s < radius * radius
    else:
        hit = ((0.5 * d[i] + 0.5 * d[j]) - np.sqrt(s)) > 0
    return np.stack([i[hit], j[hit]], axis=1).astype(np.int64)


# ---------------------------------------------------------------- grid ----
def test_tutorial_neighbors(orc):
    g = golden("tutorial_neighbors.json")
    xyz = np.array(g["positions"], float)
    s = orc.Sim(xyz, np.full(3, float(g["diameter"])))
    pairs = s.neighbors(math.sqrt(g["squared_radius"]))
    got = {str(a): [] for a in range(3)}
    for a, b in pairs.tolist():
        got[str(a)].append(b)
        got[str(b)].append(a)
    assert {k: sorted(v) for k, v in got.items()} == g["neighbors"]
    for a, b in pairs.tolist():
        assert np.linalg.norm(xyz[a] - xyz[b]) == g["distance"]
    # box ids by hand: origin (10,0,0), L = 11 -> x boxes floor(0/11), floor(10/11), floor(20/11)
    box, ol, dims = s.grid()
    assert box.tolist() == [0, 0, 1]
    assert ol.tolist() == [10.0, 0.0, 0.0, 11.0]
    assert dims.tolist() == [2, 1, 1]


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("radius", [-1.0, 5.0, 13.5, 30.0])
def test_grid_neighbors_equal_brute_force(orc, seed, radius):
    xyz, d = workloads.uniform_cube(1500, 120.0, seed=seed)
    s = orc.Sim(xyz, d)
    got = s.neighbors(radius)
    want = brute_pairs(xyz, d, radius)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


def test_full_plain_workload_neighbors_equal_brute_force(orc):
    pop = workloads.plain_fp64()
    s = orc.Sim(pop.xyz, pop.diameter, pop.params)
    assert np.array_equal(s.neighbors(-1.0), brute_pairs(pop.xyz, pop.diameter, -1.0))


def test_interaction_pairs_lie_in_adjacent_boxes(orc):
    xyz, d = workloads.uniform_cube(3000, 130.0, seed=5)
    s = orc.Sim(xyz, d)
    box, ol, dims = s.grid()
    nx, ny = dims[0], dims[1]
    c = np.stack([box % nx, (box // nx) % ny, box // (nx * ny)], axis=1)
    pairs = s.neighbors(-1.0)
    assert len(pairs) > 1000
    assert np.all(np.abs(c[pairs[:, 0]] - c[pairs[:, 1]]) <= 1)
    assert ol[3] == d.max()
    assert np.all(c >= 0) and np.all(c < dims)


# --------------------------------------------------------------- force ----
def two(dist, d=(10.0, 10.0), **kw):
    import oracle
    return oracle.Sim(np.array([[0.0, 0, 0], [dist, 0, 0]]), np.array(d, float), **kw)


@pytest.mark.parametrize("case", golden("two_sphere_forces.json")["cases"], ids=lambda c: c["name"])
def test_two_sphere_closed_form(orc, case):
    s = two(case["distance"], case["d"])
    F, nnz, sm = s.forces()
    # the sphere at the origin is pushed towards -x by a positive F_N
    assert F[0, 0] == pytest.approx(-case["F_N"], rel=1e-15, abs=1e-16)
    assert F[1, 0] == -F[0, 0]
    assert F[0, 1] == 0 and F[0, 2] == 0
    assert nnz.tolist() == ([1, 1] if case["F_N"] != 0 else [0, 0])


def test_two_sphere_displacement_and_adherence(orc):
    s = two(8.0)
    s.step(1)
    xyz, _, _ = s.get()
    assert xyz[0, 0] == pytest.approx(-0.017639320225002102, rel=1e-14)
    assert xyz[1, 0] == pytest.approx(8.0 + 0.017639320225002102, rel=1e-14)
    # adhesive regime: |F| = 0.118 < adherence 0.4 -> no movement
    s = two(9.5)
    s.step(1)
    xyz, _, _ = s.get()
    assert xyz[:, 0].tolist() == [0.0, 9.5]
    _, D, nnz, _, _ = s.last()
    assert np.all(D == 0) and nnz.tolist() == [1, 1]


def test_clamp_limits_displacement_norm(orc):
    s = two(0.5, dt=1.0)
    F, _, _ = s.forces()
    assert abs(F[0, 0]) == pytest.approx(19.0 - math.sqrt(23.75), rel=1e-15)
    s.step(1)
    _, D, _, _, _ = s.last()
    assert np.linalg.norm(D[0]) == pytest.approx(3.0, rel=1e-15)
    assert np.linalg.norm(D[1]) == pytest.approx(3.0, rel=1e-15)


def test_three_spheres(orc):
    import oracle
    s = oracle.Sim(np.array([[0.0, 0, 0], [8.0, 0, 0], [16.0, 0, 0]]), np.full(3, 10.0))
    F, nnz, _ = s.forces()
    fn = 4.0 - math.sqrt(5.0)
    assert F[1].tolist() == [0.0, 0.0, 0.0]
    assert nnz.tolist() == [1, 2, 1]
    assert F[0, 0] == pytest.approx(-fn, rel=1e-15) and F[2, 0] == pytest.approx(fn, rel=1e-15)
    h = 8.0 * math.sqrt(3.0) / 2.0
    s = oracle.Sim(np.array([[0.0, 0, 0], [8.0, 0, 0], [4.0, h, 0]]), np.full(3, 10.0))
    F, nnz, _ = s.forces()
    assert nnz.tolist() == [2, 2, 2]
    for i in range(3):
        assert np.linalg.norm(F[i]) == pytest.approx(math.sqrt(3.0) * fn, rel=1e-12)


def test_pair_forces_are_antisymmetric_bitwise(orc):
    rng = np.random.default_rng(3)
    import oracle
    for _ in range(200):
        a = rng.uniform(-50, 50, 3)
        b = a + rng.uniform(-8, 8, 3)
        d = rng.uniform(8, 12, 2)
        F, _, _ = oracle.Sim(np.stack([a, b]), d).forces()
        assert np.array_equal(F[0], -F[1])


def test_momentum_balance(orc):
    xyz, d = workloads.uniform_cube(4000, 140.0, seed=11)
    s = orc.Sim(xyz, d)
    F, nnz, sm = s.forces()
    assert nnz.sum() > 4000
    total = F.sum(axis=0)
    assert np.all(np.abs(total) <= 64 * np.finfo(float).eps * sm.sum())


def test_forces_sampled_ids_match_full(orc):
    xyz, d = workloads.uniform_cube(2000, 120.0, seed=4)
    s = orc.Sim(xyz, d)
    F, nnz, sm = s.forces()
    ids = np.array([5, 1999, 0, 77, 5])
    F2, nnz2, sm2 = s.forces(ids)
    assert np.array_equal(F2, F[ids]) and np.array_equal(nnz2, nnz[ids])


# ---------------------------------------------------------- multi-step ----
def test_two_cells_reach_adhesive_equilibrium(orc):
    """Force tutorial scenario (two cells of diameter 20, centers 10 apart)
    with dt/mass = 0.1: the cells separate monotonically and stop where
    |F_N| <= adherence, near the zero of Eq 4.1 (delta = gamma^2 r / k^2)."""
    import oracle
    s = oracle.Sim(np.array([[0.0, 0, 0], [10.0, 0, 0]]), np.full(2, 20.0), dt=0.1,
                   max_displacement=50.0)
    s.step(1)
    xyz, _, _ = s.get()
    assert xyz[0, 0] == pytest.approx(-0.1 * (20.0 - math.sqrt(50.0)), rel=1e-14)
    last = 10.0 + 2 * 0.1 * (20.0 - math.sqrt(50.0))
    for _ in range(200):
        s.step(1)
        xyz, _, _ = s.get()
        sep = xyz[1, 0] - xyz[0, 0]
        assert sep >= last - 1e-12
        last = sep
    delta = 20.0 - last
    fn = 2.0 * delta - math.sqrt(5.0 * delta)
    assert abs(fn) <= 0.4
    assert abs(delta - 1.25) < 0.5


def perturbed_scene(seed=0):
    """Sparse agents (mostly isolated, static after one iteration) plus
    a few dense clusters that keep moving."""
    rng = np.random.default_rng(seed)
    xyz = [rng.uniform(0, 400, (400, 3))]
    for c in rng.uniform(50, 350, (4, 3)):
        xyz.append(c + rng.normal(0, 6, (30, 3)))
    xyz = np.concatenate(xyz)
    d = rng.uniform(8, 12, xyz.shape[0])
    return xyz, d


def arrival_scene():
    """A lone agent (index 2, force 0, static-eligible) is reached in one
    step by an agent (index 4) that starts outside its 27-box stencil and is
    pulled across by adhesion (dt = 60, clamp 30).  Two anchors fix the grid
    so that it stays the same between iterations."""
    xyz = np.array([[0.0, -100, -100], [200.0, 100, 100],   # anchors
                    [9.0, 0, 0],                              # lone agent
                    [25.2, 0, 0], [35.0, 0, 0],               # attractor k, mover j
                    [20.3, 8.4870, 0], [20.3, -8.4870, 0]])   # balance k's pull
    return xyz, np.full(len(xyz), 10.0), dict(dt=60.0, max_displacement=30.0, adherence=0.05)


@pytest.mark.parametrize("scene", ["perturbed", "arrival"])
def test_static_skip_is_exact(orc, scene):
    import oracle
    if scene == "perturbed":
        xyz, d = perturbed_scene()
        kw = dict(dt=0.05)
    else:
        xyz, d, kw = arrival_scene()
    on = oracle.Sim(xyz, d, detect_static=1, **kw)
    off = oracle.Sim(xyz, d, detect_static=0, **kw)
    n_static = 0
    for _ in range(25):
        on.step(1)
        off.step(1)
        a, _, _ = on.get()
        b, _, _ = off.get()
        assert np.array_equal(a, b)
        _, Da, nnza, sta, _ = on.last()
        _, Db, nnzb, stb, _ = off.last()
        assert np.array_equal(Da, Db)
        assert not stb.any()
        n_static += int(sta.sum())
    assert n_static > 0
    if scene == "arrival":
        # the lone agent was moved by the arriving one after the first step
        assert a[2, 0] != 9.0


def test_permutation_invariance(orc):
    import oracle
    xyz, d = workloads.uniform_cube(800, 90.0, seed=7)
    perm = np.random.default_rng(1).permutation(800)
    a = oracle.Sim(xyz, d)
    b = oracle.Sim(xyz[perm], d[perm])
    a.step(5)
    b.step(5)
    xa, _, _ = a.get()
    xb, _, _ = b.get()
    np.testing.assert_allclose(xb, xa[perm], rtol=0, atol=1e-11)
    ba, _, _ = a.grid()
    bb, _, _ = b.grid()
    assert np.array_equal(bb, ba[perm])


# ---------------------------------------------------- growth/division ----
def test_growth_division_population_step_function(orc):
    import oracle
    pop = workloads.growth_division(shape=(4, 4, 4), cap_factor=8)
    p = pop.params
    s = oracle.Sim(pop.xyz, pop.diameter, p)
    # Scalar recurrence of the synchronised population.
    v = math.pi * 729.0 / 6.0
    n, cap, vdiv, dv = 64, 512, p.divide_volume, p.growth_rate * p.dt
    division_rounds = []
    for t in range(60):
        if v < vdiv:
            v += dv
        elif n < cap:
            n, v = 2 * n, v / 2
            division_rounds.append(t)
        s.step(1)
        assert s.n == n, t
    assert len(division_rounds) == 3 and division_rounds[0] == 14
    _, dd, vv = s.get()
    assert np.all(vv >= vdiv / 2) and s.n == cap


def test_division_conserves_volume_and_places_daughters(orc):
    import oracle
    pop = workloads.growth_division(shape=(3, 3, 3), cap_factor=2)
    s = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    s.step(14)
    assert s.n == 27
    x0, d0, v0 = s.get()
    s.step(1)
    assert s.n == 54
    x1, d1, v1 = s.get()
    _, D, _, _, _ = s.last()
    for i in range(27):
        j = 27 + i  # ascending parent ID
        assert v1[i] + v1[j] == v0[i]
        assert d1[i] == d1[j] == oracle.diameter_of_volume(v0[i] / 2)
        mid = 0.5 * (x1[i] + x1[j])
        np.testing.assert_allclose(mid, x0[i] + D[i], rtol=0, atol=1e-12)
        assert np.linalg.norm(x1[j] - x1[i]) == pytest.approx(d1[i] / 2, rel=1e-13)


def test_cbrt_correctly_rounded(orc):
    import oracle
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(1, 2000, 300), np.exp(rng.uniform(-200, 200, 300)),
                         [1.0, 8.0, 27.0, 1728.0, 2.0, 3.0]])
    for x in xs:
        y = oracle.cbrt_rn(float(x))
        lo = Fraction(np.nextafter(y, 0.0)) / 2 + Fraction(y) / 2
        hi = Fraction(np.nextafter(y, np.inf)) / 2 + Fraction(y) / 2
        fx = Fraction(float(x))
        assert lo ** 3 < fx < hi ** 3 or Fraction(y) ** 3 == fx
    assert oracle.cbrt_rn(27.0) == 3.0 and oracle.cbrt_rn(1728.0) == 12.0


def test_philox_matches_numpy(orc):
    """numpy's Philox (4x64, 10 rounds) increments its 256-bit counter
    before producing each block, so it is started one below ours."""
    import oracle
    key = [0x0123456789ABCDEF, 0xFEDCBA9876543210]
    for ctr in ([0, 0, 0, 0], [5, 7, 11, 13], [2**64 - 2, 3, 0, 0], [0, 9, 1, 2]):
        c = sum(v << (64 * k) for k, v in enumerate(ctr))
        c = (c - 1) % 2**256
        prev = [(c >> (64 * k)) & (2**64 - 1) for k in range(4)]
        ref = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
        assert oracle.philox4x64_10(ctr, key) == [int(v) for v in ref.random_raw(4)]


def test_division_axis_is_unit_and_reproducible(orc):
    import oracle
    us = np.array([oracle.division_axis(9, i, 3) for i in range(2000)])
    np.testing.assert_allclose(np.linalg.norm(us, axis=1), 1.0, atol=1e-15)
    assert np.all(np.abs(us.mean(axis=0)) < 0.06)
    assert np.array_equal(us[17], oracle.division_axis(9, 17, 3))
    assert not np.array_equal(us[17], oracle.division_axis(9, 17, 4))


# --------------------------------------------------------------- Morton ----
def test_fig5_4_gap_offsets_and_order(orc):
    import oracle
    g = golden("fig5_4_morton.json")
    assert [list(e) for e in oracle.morton_gaps(2, g["dims"])] == g["gap_offsets"]
    assert oracle.morton_sequence(2, g["dims"]).tolist() == g["morton_order"]


def test_fig5_4_agent_order_prefix(orc):
    """Place agents in a 3x3 grid with the printed per-box counts; the
    oracle's Morton agent order must reproduce the printed prefix sums."""
    import oracle
    g = golden("fig5_4_morton.json")
    # de-interleave the 2D codes (x at bit 0) into box coordinates
    boxes = []
    for code in g["morton_order"]:
        x = sum(((code >> (2 * b)) & 1) << b for b in range(4))
        y = sum(((code >> (2 * b + 1)) & 1) << b for b in range(4))
        boxes.append((x, y))
    xyz = []
    for (bx, by), cnt in zip(boxes, g["agents_per_box_in_morton_order"]):
        for k in range(cnt):
            xyz.append([bx * 10.0 + 5.0 + 0.1 * k, by * 10.0 + 5.0, 0.0])
    xyz = np.array(xyz)
    s = oracle.Sim(xyz, np.full(len(xyz), 1.0), box_length=10.0)
    box, ol, dims = s.grid()
    assert dims.tolist() == [3, 3, 1]
    order = s.morton_agent_order()
    seq = [(int(box[i] % 3), int(box[i] // 3)) for i in order]
    counts = [seq.count(b) for b in boxes]
    assert counts == g["agents_per_box_in_morton_order"]
    assert np.cumsum(counts).tolist() == g["prefix_sum"]
    assert [b for b in boxes if b in seq] == list(dict.fromkeys(seq))


@pytest.mark.parametrize("dim,dims", [(2, [3, 3]), (2, [5, 2]), (3, [3, 3, 3]), (3, [7, 2, 5]),
                                      (3, [1, 1, 9]), (3, [16, 16, 16]), (2, [1, 1])])
def test_gap_algorithm_equals_sorted_interleave(orc, dim, dims):
    import itertools
    import oracle
    codes = sorted(oracle.interleave(dim, list(c)) for c in itertools.product(*[range(n) for n in dims]))
    assert oracle.morton_sequence(dim, dims).tolist() == codes
