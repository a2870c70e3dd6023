"""Pins of the oracle's in-place execution context (§5.2), on the CPU.

The in-place context makes an agent's new position visible to the agents
processed after it in the same iteration, in the order: boxes by colour
(box-coordinate parities; a third colour for the last box of an odd
toroidal axis), boxes of a colour in ascending index, agents of a box in
ascending ID.  The pins are fixed by something other than the oracle:

- two spheres in one box, in closed form (Eq 4.1): the first moves by the
  copy-context force, the second then sees the larger distance and stays;
- two spheres in neighbouring boxes where the higher ID has the lower
  colour: that one moves first;
- the seam pair of a torus with an odd number of boxes per axis: the box
  at 0 (colour 0) comes before the last box (colour 2), in closed form;
- a Gauss-Seidel sweep written out in this test over all pairs (brute
  force, no grid) in the same agent order, bit for bit, on 400 agents whose
  moves are too small to reach a pair outside the start grid's stencils.
"""
import math

import numpy as np
import pytest


def sim(xyz, d, **kw):
    import oracle
    return oracle.Sim(np.asarray(xyz, np.float64), np.asarray(d, np.float64), execution_context=1, **kw)


FN8 = 4.0 - math.sqrt(5.0)  # d = 10, distance 8: delta = 2, r = 2.5


def test_two_spheres_in_one_box(orc):
    s = sim([[50.0, 50.0, 50.0], [58.0, 50.0, 50.0]], [10.0, 10.0], dt=1.0)
    s.step(1)
    x, _, _ = s.get()
    assert x[0, 0] == 50.0 - FN8  # moved by the full copy-context force
    # agent 1 then sees distance 8 + FN8: delta = 2 - FN8, F_N < 0 with
    # |F_N| = |2 delta - sqrt(2.5 delta)| < 0.4 (adherence): it stays
    delta = 2.0 - FN8
    assert abs(2.0 * delta - math.sqrt(2.5 * delta)) < 0.4
    assert x[1, 0] == 58.0
    # the copy context moves both
    import oracle
    c = oracle.Sim(np.array([[50.0, 50.0, 50.0], [58.0, 50.0, 50.0]]), np.array([10.0, 10.0]), dt=1.0)
    c.step(1)
    xc, _, _ = c.get()
    assert xc[0, 0] == 50.0 - FN8 and xc[1, 0] == 58.0 + FN8


def test_colour_order_before_id_order(orc):
    """A third, isolated agent puts the origin at x = 45, so agent 1 (x =
    50) lies in box 0 (colour 0) and agent 0 (x = 58) in box 1 (colour 1):
    agent 1 moves first although its ID is higher."""
    s = sim([[58.0, 50.0, 50.0], [50.0, 50.0, 50.0], [45.0, 500.0, 500.0]], [10.0, 10.0, 10.0], dt=1.0)
    s.step(1)
    x, _, _ = s.get()
    assert x[1, 0] == 50.0 - FN8
    assert x[0, 0] == 58.0
    assert np.array_equal(x[2], [45.0, 500.0, 500.0])
    box, _, dims = s.grid()
    assert box[1] % dims[0] == 0 and box[0] % dims[0] == 1


def test_odd_torus_seam_colour(orc):
    """Torus [0, 90): 9 boxes of 10 per axis.  Agent 0 at x = 88 lies in box
    8, the last box of an odd axis (colour 2); agent 1 at x = 2 in box 0
    (colour 0) goes first.  Minimum-image distance 4: agent 1 moves by
    dt * (12 - sqrt(15)); agent 0 then sees the new distance."""
    p = dict(dt=0.1, max_displacement=100.0, boundary=2, bound_min=0.0, bound_max=90.0)
    s = sim([[88.0, 45.0, 45.0], [2.0, 45.0, 45.0]], [10.0, 10.0], **p)
    s.step(1)
    x, _, _ = s.get()
    fn1 = 12.0 - math.sqrt(15.0)
    x1 = 2.0 + 0.1 * fn1
    assert x[1, 0] == x1
    dist = (x1 + 90.0) - 88.0
    delta = 10.0 - dist
    fn0 = 2.0 * delta - math.sqrt(2.5 * delta)
    assert x[0, 0] == pytest.approx(88.0 - 0.1 * fn0, abs=1e-12)
    assert not x[0, 0] == pytest.approx(88.0 - 0.1 * fn1, abs=1e-6)  # the copy context's answer


def colour_order(box, dims, ids):
    """Agent order of the in-place sweep: colour (parities, 2 per axis on an
    open grid), box index, ID."""
    c = np.stack([box % dims[0], (box // dims[0]) % dims[1], box // (dims[0] * dims[1])], axis=1)
    col = (c[:, 0] % 2) + 2 * ((c[:, 1] % 2) + 2 * (c[:, 2] % 2))
    return sorted(ids, key=lambda i: (col[i], box[i], i))


def brute_sweep(xyz, d, order, k, gamma, adherence, dt, m):
    x = xyz.copy()
    n = len(d)
    for i in order:
        F = [0.0, 0.0, 0.0]
        for j in range(n):
            if j == i:
                continue
            dx, dy, dz = x[i, 0] - x[j, 0], x[i, 1] - x[j, 1], x[i, 2] - x[j, 2]
            dist = math.sqrt((dx * dx + dy * dy) + dz * dz)
            delta = (0.5 * d[i] + 0.5 * d[j]) - dist
            if not delta > 0.0:
                continue
            ri, rj = 0.5 * d[i], 0.5 * d[j]
            r = (ri * rj) / (ri + rj)
            fn = k * delta - gamma * math.sqrt(r * delta)
            if dist > 0.0:
                F[0] += fn * (dx / dist)
                F[1] += fn * (dy / dist)
                F[2] += fn * (dz / dist)
        fnorm = math.sqrt((F[0] * F[0] + F[1] * F[1]) + F[2] * F[2])
        if not fnorm > adherence:
            continue
        D = [dt * F[0], dt * F[1], dt * F[2]]
        dn = math.sqrt((D[0] * D[0] + D[1] * D[1]) + D[2] * D[2])
        if dn > m:
            s = m / dn
            D = [D[0] * s, D[1] * s, D[2] * s]
        x[i] = [x[i, 0] + D[0], x[i, 1] + D[1], x[i, 2] + D[2]]
    return x


def test_equals_brute_force_gauss_seidel(orc):
    rng = np.random.default_rng(3)
    n = 400
    xyz = rng.uniform(0.0, 60.0, (n, 3))
    d = rng.uniform(8.0, 12.0, n)
    p = dict(dt=0.0002, adherence=0.0, max_displacement=3.0)
    s = sim(xyz, d, **p)
    box, _, dims = s.grid()
    # every pair within r_i + r_j + 0.05 lies in neighbouring start boxes, so
    # moves below 0.025 per agent cannot bring in a pair the grid misses
    c = np.stack([box % dims[0], (box // dims[0]) % dims[1], box // (dims[0] * dims[1])], axis=1)
    for i in range(n):
        dist = np.linalg.norm(xyz - xyz[i], axis=1)
        near = np.flatnonzero(dist < 0.5 * d + 0.5 * d[i] + 0.05)
        assert (np.abs(c[near] - c[i]).max(axis=1) <= 1).all()
    order = colour_order(box, dims, range(n))
    want = brute_sweep(xyz, d, order, 2.0, 1.0, p["adherence"], p["dt"], p["max_displacement"])
    s.step(1)
    x, _, _ = s.get()
    assert np.abs(x - xyz).max() < 0.025
    assert np.array_equal(x, want)
    # and it differs from the copy context (the order matters)
    import oracle
    cpy = oracle.Sim(xyz, d, **p)
    cpy.step(1)
    assert not np.array_equal(cpy.get()[0], x)


def test_static_detection_is_refused(orc):
    with pytest.raises(Exception):
        sim([[0.0, 0.0, 0.0]], [1.0], detect_static=1)
