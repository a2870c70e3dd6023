"""Pins of the oracle pieces the in-step substance composes (CPU): the
position setter that follows the mechanical step (an agent it moves counts
as changed, so neither it nor its neighbours are static next iteration,
while distant static agents stay static), and mass conservation of one
composed iteration (secretion adds n x quantity, Eq 4.3 without decay keeps
the mass while no substance reaches the grid's faces)."""
import numpy as np
import pytest


def settled_pair_scene():
    """Two isolated spheres far apart (nnz 0, no force): static from the
    second iteration on."""
    return np.array([[0.0, 0.0, 0.0], [500.0, 0.0, 0.0], [0.0, 500.0, 0.0]]), np.array([10.0, 10.0, 10.0])


def test_set_positions_marks_changed(orc):
    import oracle
    xyz, d = settled_pair_scene()
    s = oracle.Sim(xyz, d, detect_static=1)
    s.step(3)
    _, _, _, st, _ = s.last()
    assert st.all()
    moved = xyz.copy()
    moved[1, 0] += 0.5
    s.set_positions(moved)
    s.step(1)
    _, _, _, st, changed = s.last()
    assert not st[1] and st[0] and st[2]  # only the moved agent lost its static state
    with pytest.raises(ValueError):
        s.set_positions(moved[:2])


def test_composed_iteration_conserves_mass(orc):
    import oracle
    rng = np.random.default_rng(4)
    xyz = 200.0 + rng.uniform(-20.0, 20.0, (300, 3))
    d = rng.uniform(8.0, 12.0, 300)
    s = oracle.Sim(xyz, d, dt=0.01)
    u = np.zeros((40, 40, 40))
    lo, h = np.array([0.0, 0.0, 0.0]), np.array([10.0, 10.0, 10.0])
    q = 2.0
    for t in range(3):
        s.step(1)
        x, _, _ = s.get()
        before = u.sum()
        oracle.secrete(u, lo, h, x, q)
        assert u.sum() == pytest.approx(before + q * x.shape[0], rel=1e-15)
        m = u.sum()
        oracle.diffuse(u, h, nu=1.0, mu=0.0, dt=0.01, steps=1)
        assert u.sum() == pytest.approx(m, rel=1e-12)
        s.set_positions(oracle.chemotaxis(u, lo, h, x, 0.5))
    assert not np.array_equal(s.get()[0], xyz)
