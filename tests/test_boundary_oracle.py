"""Pins of the oracle's space boundary conditions (§4.4.11: open, closed,
toroidal) and agent removal (§5.3.2, Fig 5.1), on the CPU.

Each pin is fixed by something other than the oracle itself: closed forms
of Eq 4.1 / Eq 4.2 for spheres across a wall or a seam, a brute-force
minimum-image pair search, invariance of a torus under translation, the
index swaps of the removal algorithm worked by hand, and the equality of a
simulation after a removal with one started from the survivors.
"""
import numpy as np
import pytest


def sim(xyz, d, **kw):
    import oracle
    return oracle.Sim(np.asarray(xyz, np.float64), np.asarray(d, np.float64), **kw)


def test_closed_wall_stops_the_pushed_agent(orc):
    """Two spheres of diameter 10, centres 8 apart, the right one 1 from the
    wall at 100: each is pushed with F_N = 4 - sqrt(5) (Eq 4.1, delta = 2,
    r = 2.5); with dt = 1 the right one would cross the wall and stays on it,
    the left one moves freely."""
    fn = 4.0 - np.sqrt(5.0)
    s = sim([[91.0, 50.0, 50.0], [99.0, 50.0, 50.0]], [10.0, 10.0], dt=1.0, boundary=1,
            bound_min=0.0, bound_max=100.0)
    s.step(1)
    x, _, _ = s.get()
    assert x[1, 0] == 100.0
    assert x[0, 0] == 91.0 - fn
    assert np.all(x[:, 1:] == 50.0)
    _, D, _, _, changed = s.last()
    assert changed.all() and D[1, 0] == fn  # pushed: changed, although the wall stopped it


def test_toroidal_seam_pair_closed_form(orc):
    """Spheres of diameter 10 at x = 1 and x = 97 in the torus [0, 100):
    the minimum-image distance is 4, delta = 6, r = 2.5, so F_N = 12 -
    sqrt(15), pushing the first to +x across the seam; with dt = 1 the
    displacement is clamped to 3."""
    p = dict(dt=1.0, boundary=2, bound_min=0.0, bound_max=100.0)
    s = sim([[1.0, 50.0, 50.0], [97.0, 50.0, 50.0]], [10.0, 10.0], **p)
    F, nnz, smag = s.forces()
    fn = 12.0 - np.sqrt(15.0)
    assert F[0, 0] == fn and F[1, 0] == -fn and np.all(F[:, 1:] == 0.0)
    assert nnz.tolist() == [1, 1]
    s.step(1)
    x, _, _ = s.get()
    assert x[0, 0] == 4.0 and x[1, 0] == 94.0


def test_toroidal_wrap_crosses_the_face(orc):
    """A sphere 0.5 below the upper face pushed +x by 4 - sqrt(5) re-enters
    at the lower face: (99.5 + D) - 100."""
    fn = 4.0 - np.sqrt(5.0)
    s = sim([[91.5, 5.0, 5.0], [99.5, 5.0, 5.0]], [10.0, 10.0], dt=1.0, boundary=2, bound_min=0.0,
            bound_max=100.0)
    s.step(1)
    x, _, _ = s.get()
    assert x[1, 0] == (99.5 + fn) - 100.0
    assert 0.0 <= x[1, 0] < 100.0


def brute_torus_pairs(xyz, d, size, radius):
    n = len(xyz)
    out = []
    for i in range(n):
        dd = xyz[i] - xyz[i + 1:]
        dd = np.where(dd > size / 2, dd - size, dd)
        dd = np.where(dd < -size / 2, dd + size, dd)
        s = (dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1]) + dd[:, 2] * dd[:, 2]
        if radius < 0:
            hit = (0.5 * d[i] + 0.5 * d[i + 1:]) - np.sqrt(s) > 0.0
        else:
            hit = s < radius * radius
        out += [(i, i + 1 + j) for j in np.flatnonzero(hit)]
    return np.array(out, np.int64).reshape(-1, 2)


@pytest.mark.parametrize("radius", [-1.0, 7.5, 20.0])
@pytest.mark.parametrize("seed", [0, 1])
def test_toroidal_pairs_equal_brute_force(orc, seed, radius):
    rng = np.random.default_rng(seed)
    size = 90.0
    xyz = rng.uniform(0.0, size, (900, 3))
    d = rng.uniform(8.0, 12.0, 900)
    s = sim(xyz, d, boundary=2, bound_min=0.0, bound_max=size)
    assert np.array_equal(s.neighbors(radius), brute_torus_pairs(xyz, d, size, radius))


def test_toroidal_translation_invariance(orc):
    """Shifting every centre by the same vector on the torus leaves every
    pair's overlap, hence every force, the same (to rounding)."""
    rng = np.random.default_rng(4)
    size = 80.0
    xyz = rng.uniform(0.0, size, (700, 3))
    d = rng.uniform(8.0, 12.0, 700)
    p = dict(boundary=2, bound_min=0.0, bound_max=size)
    F0, nnz0, smag = sim(xyz, d, **p).forces()
    shifted = np.mod(xyz + np.array([31.25, 57.5, 72.75]), size)
    F1, nnz1, _ = sim(shifted, d, **p).forces()
    assert np.array_equal(nnz0, nnz1)
    assert (np.linalg.norm(F1 - F0, axis=1) <= 1e-12 * np.maximum(smag, 1.0)).all()


def test_toroidal_space_narrower_than_three_boxes(orc):
    s = sim([[1.0, 1.0, 1.0], [20.0, 20.0, 20.0]], [10.0, 10.0], boundary=2, bound_min=0.0, bound_max=25.0)
    with pytest.raises(RuntimeError):
        s.step(1)


def test_positions_outside_the_space_are_rejected(orc):
    for boundary, v in ((1, 100.5), (1, -0.5), (2, 100.0), (2, -1e-9)):
        with pytest.raises(ValueError):
            sim([[v, 5.0, 5.0]], [1.0], boundary=boundary, bound_min=0.0, bound_max=100.0)
    sim([[100.0, 5.0, 5.0]], [1.0], boundary=1, bound_min=0.0, bound_max=100.0)  # a closed wall is inside


def test_removal_swaps_of_fig_5_1(orc):
    """Seven agents (IDs 0-6), three removed (1, 4, 6): n' = 4; agent 1 is a
    hole below n', agents 4 and 6 lie at or above it; the one survivor at or
    above n' (5) moves into the hole: the new order is 0, 5, 2, 3."""
    xyz = np.arange(21, dtype=np.float64).reshape(7, 3) * 100.0
    d = np.arange(1, 8, dtype=np.float64)
    s = sim(xyz, d)
    s.remove([4, 1, 6])
    x, dd, _ = s.get()
    assert s.n == 4
    assert np.array_equal(x, xyz[[0, 5, 2, 3]]) and np.array_equal(dd, d[[0, 5, 2, 3]])
    with pytest.raises(ValueError):
        s.remove([2, 2])
    with pytest.raises(ValueError):
        s.remove([4])


def test_removal_equals_a_fresh_start(orc):
    """After a removal every survivor counts as changed, so the trajectory
    equals that of a simulation started from the survivors (in their new ID
    order), bit for bit, static detection included."""
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    a = sim(xyz, d, detect_static=1, dt=0.05)
    a.step(6)
    rng = np.random.default_rng(2)
    gone = rng.choice(a.n, a.n // 3, replace=False)
    a.remove(gone)
    x, dd, _ = a.get()
    b = sim(x, dd, detect_static=1, dt=0.05)
    for _ in range(10):
        a.step(1)
        b.step(1)
        xa, _, _ = a.get()
        xb, _, _ = b.get()
        assert np.array_equal(xa, xb)
        _, _, _, sa, _ = a.last()
        _, _, _, sb, _ = b.last()
        assert np.array_equal(sa, sb)
    assert sa.any()
