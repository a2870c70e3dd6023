"""Pins of the diffusion oracle (§4.5.2 Eq 4.3, Algorithms 6 and 7): values
fixed by hand for small cases, conservation and decay laws, the maximum
principle, the outflow at the boundary, and the convergence towards the
analytical solution of an instantaneous point source (the test of Fig 4.9,
measured at sqrt(1000) from the source)."""
import math

import numpy as np
import pytest


def test_point_source_one_step_by_hand(orc):
    import oracle
    # nu = 1, dt = 0.01, h = (1, 2, 0.5), mu = 0.5: cx = 0.01, cy = 0.0025,
    # cz = 0.04, 1 - mu dt = 0.995; the source keeps 0.995 - 2 (0.0525) = 0.89
    u = np.zeros((5, 5, 5))
    u[2, 2, 2] = 1.0
    oracle.diffuse(u, [1.0, 2.0, 0.5], 1.0, 0.5, 0.01, 1)
    assert u[2, 2, 2] == pytest.approx(0.89, abs=1e-15)
    assert u[2, 2, 3] == pytest.approx(0.01, abs=1e-16) and u[2, 2, 1] == pytest.approx(0.01, abs=1e-16)
    assert u[2, 3, 2] == pytest.approx(0.0025, abs=1e-16) and u[2, 1, 2] == pytest.approx(0.0025, abs=1e-16)
    assert u[3, 2, 2] == pytest.approx(0.04, abs=1e-16) and u[1, 2, 2] == pytest.approx(0.04, abs=1e-16)
    assert np.count_nonzero(u) == 7
    # a second step reaches the diagonal neighbours: cx cy each way
    oracle.diffuse(u, [1.0, 2.0, 0.5], 1.0, 0.5, 0.01, 1)
    assert u[2, 3, 3] == pytest.approx(2 * 0.01 * 0.0025, rel=1e-12)


def test_mass_is_conserved_and_decays_geometrically(orc):
    import oracle
    rng = np.random.default_rng(3)
    u = np.zeros((30, 30, 30))
    u[12:18, 12:18, 12:18] = rng.uniform(0.0, 1.0, (6, 6, 6))
    m0 = u.sum()
    oracle.diffuse(u, [1.0, 1.0, 1.0], 0.8, 0.0, 0.1, 10)  # support grows by 10 < 12 cells
    assert u.sum() == pytest.approx(m0, rel=1e-13)
    mu, dt = 0.3, 0.1
    v = np.zeros((30, 30, 30))
    v[12:18, 12:18, 12:18] = rng.uniform(0.0, 1.0, (6, 6, 6))
    m1 = v.sum()
    oracle.diffuse(v, [1.0, 1.0, 1.0], 0.8, mu, dt, 10)
    assert v.sum() == pytest.approx(m1 * (1.0 - mu * dt) ** 10, rel=1e-13)


def test_outflow_through_the_boundary(orc):
    import oracle
    # a source on the x = 0 face loses the share of its missing neighbour:
    # total after one step = 1 - mu dt - cx
    u = np.zeros((5, 5, 5))
    u[2, 2, 0] = 1.0
    oracle.diffuse(u, [1.0, 1.0, 1.0], 1.0, 0.2, 0.05, 1)
    assert u.sum() == pytest.approx(1.0 - 0.2 * 0.05 - 0.05, rel=1e-14)


def test_maximum_principle_when_stable(orc):
    import oracle
    rng = np.random.default_rng(7)
    u = rng.uniform(0.0, 1.0, (12, 10, 8))
    top = u.max()
    # nu dt (1/hx^2 + 1/hy^2 + 1/hz^2) = 0.4 <= 1/2: no new extrema
    oracle.diffuse(u, [1.0, 1.0, 1.0], 1.0, 0.1, 0.4 / 3.0, 20)
    assert u.min() >= 0.0 and u.max() <= top


def test_convergence_to_the_point_source_solution(orc):
    """Instantaneous point source of mass M at the origin in free space:
    c(r, t) = M / (4 pi nu t)^(3/2) exp(-r^2 / (4 nu t)) exp(-mu t).  The
    error at r = sqrt(1000) = |(30, 10, 0)| falls as the grid is refined."""
    import oracle
    nu, mu, M, half = 1.0, 0.001, 1.0, 100.0
    r2 = 30.0 ** 2 + 10.0 ** 2
    errs = []
    for h in (10.0, 5.0, 2.5):
        n = int(round(2 * half / h)) + 1
        i0 = int(round(half / h))
        u = np.zeros((n, n, n))
        u[i0, i0, i0] = M / h ** 3  # the source as a concentration
        dt = h * h / 8.0
        steps = int(round(200.0 / dt))
        rel = []
        done = 0
        for t_probe in (100.0, 150.0, 200.0):
            k = int(round(t_probe / dt)) - done
            oracle.diffuse(u, [h, h, h], nu, mu, dt, k)
            done += k
            t = done * dt
            exact = M / (4.0 * math.pi * nu * t) ** 1.5 * math.exp(-r2 / (4.0 * nu * t)) * math.exp(-mu * t)
            got = u[i0, i0 + int(round(10.0 / h)), i0 + int(round(30.0 / h))]
            rel.append(abs(got - exact) / exact)
        assert done == steps
        errs.append(max(rel))
    # second order in h: each halving divides the error by about four
    assert errs[0] / errs[1] > 3.0 and errs[1] / errs[2] > 3.0
    assert errs[2] < 0.015


def test_secretion_by_hand(orc):
    import oracle
    u = np.zeros((3, 4, 5))  # n = (5, 4, 3)
    xyz = np.array([[2.5, 0.5, 1.0],   # box (2, 0, 1)
                    [3.0, 3.99, 2.5],  # on a box boundary in x: box (3, 3, 2)
                    [-0.1, 1.0, 1.0],  # outside: nothing
                    [2.7, 0.2, 1.9]])  # box (2, 0, 1) again
    oracle.secrete(u, [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], xyz, 0.25)
    assert u[1, 0, 2] == 0.5 and u[2, 3, 3] == 0.25 and u.sum() == 0.75


def test_gradient_of_a_linear_field_and_at_the_boundary(orc):
    import oracle
    h = 2.0
    n = 8
    x = (np.arange(n) + 0.5) * h
    u = np.broadcast_to(3.0 * x, (4, 5, n)).copy()  # u = 3 x, rising along x
    pts = np.array([[x[3], 3.0, 3.0], [x[n - 1], 3.0, 3.0], [x[0], 1.0, 1.0]])
    g = oracle.gradient(u, [0.0, 0.0, 0.0], [h, h, h], pts)
    assert g[0].tolist() == [1.0, 0.0, 0.0]
    # last box: the outside neighbour is zero, so the slope turns negative
    assert g[1].tolist() == [-1.0, 0.0, 0.0]
    # first box, first rows in y and z: the y and z neighbours outside are
    # zero too, so the gradient leans towards the interior in y and z
    assert g[2][0] > 0 and g[2][1] > 0 and g[2][2] > 0
    assert np.linalg.norm(g[2]) == pytest.approx(1.0, rel=1e-15)


def test_chemotaxis_follows_a_radial_field(orc):
    import oracle
    h = 1.0
    n = 40
    c = np.array([20.0, 20.0, 20.0])
    centers = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(centers, centers, centers, indexing="ij")
    u = np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / 200.0)
    rng = np.random.default_rng(5)
    pts = c + rng.uniform(-12.0, 12.0, (200, 3))
    moved = oracle.chemotaxis(u, [0.0, 0.0, 0.0], [h, h, h], pts, 0.5)
    step = moved - pts
    norms = np.linalg.norm(step, axis=1)
    assert np.allclose(norms, 0.5, rtol=1e-12)
    # every step points up the field, towards the centre
    assert (np.einsum("ij,ij->i", step, c - pts) > 0).all()
    # a uniform interior field has no gradient: nobody moves
    flat = np.ones((10, 10, 10))
    p = np.array([[5.2, 5.5, 4.9]])
    assert np.array_equal(oracle.chemotaxis(flat, [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], p, 0.5), p)
