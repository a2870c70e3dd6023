"""Pins of the epidemiology oracle (§4.6.3, Algorithms 3-5): infection
inside the radius by hand, the copy execution context along a chain, the
recovery rule and its rate, movement by exactly the speed on the torus, and
agreement with the SIR model the thesis compares against (measles
parameters of Table 4.3, Fig 4.17A)."""
import numpy as np

S, I, R = 0, 1, 2


def test_infection_inside_the_radius_by_hand(orc):
    import oracle
    c = np.array([50.0, 50.0, 50.0])
    xyz = np.array([c, c + [1.0, 0, 0], c + [0, 3.2, 0], c + [0, 0, 3.3], c + [2.0, 2.0, 2.0]])
    st = [I, S, S, S, S]  # radius 3.24179: 1.0 and 3.2 inside, 3.3 and sqrt(12) outside
    _, got = oracle.sir_step(xyz, st, 3.24179, 1.0, 0.0, 0.0, 100.0)
    assert got.tolist() == [I, I, I, S, S]


def test_copy_context_along_a_chain(orc):
    import oracle
    xyz = np.array([[10.0, 10.0, 10.0], [12.0, 10.0, 10.0], [14.5, 10.0, 10.0]])
    x, st = oracle.sir_step(xyz, [I, S, S], 3.0, 1.0, 0.0, 0.0, 100.0)
    assert st.tolist() == [I, I, S]  # C reads B's state at the start of the step
    x, st = oracle.sir_step(x, st, 3.0, 1.0, 0.0, 0.0, 100.0, t0=1)
    assert st.tolist() == [I, I, I]


def test_recovery_rule_and_rate(orc):
    import oracle
    rng = np.random.default_rng(0)
    xyz = rng.uniform(0.0, 100.0, (30, 3))
    st = np.array([S] * 10 + [I] * 10 + [R] * 10, np.uint8)
    _, got = oracle.sir_step(xyz, st, 5.0, 0.0, 1.0, 1.0, 100.0)
    assert got.tolist() == [S] * 10 + [R] * 20
    n = 20000
    _, got = oracle.sir_step(rng.uniform(0.0, 100.0, (n, 3)), np.full(n, I, np.uint8), 0.0, 0.0, 0.3, 1.0, 100.0,
                             seed=3)
    k = int((got == R).sum())
    assert abs(k - 0.3 * n) < 5 * np.sqrt(n * 0.3 * 0.7)


def test_movement_by_the_speed_on_the_torus(orc):
    import oracle
    rng = np.random.default_rng(1)
    L, speed = 100.0, 2.5
    xyz = rng.uniform(0.0, L, (500, 3))
    xyz[:10, 0] = L - 0.5  # near the upper x face: several wrap
    xyz[10:20, 1] = 0.25   # near the lower y face
    moved, _ = oracle.sir_step(xyz, np.zeros(500, np.uint8), 0.0, 0.0, 0.0, speed, L, seed=9)
    assert moved.min() >= 0.0 and moved.max() < L
    d = moved - xyz
    d -= L * np.round(d / L)  # nearest image
    assert np.allclose(np.linalg.norm(d, axis=1), speed, rtol=1e-12)
    assert (np.abs(moved[:10, 0] - xyz[:10, 0]) > L / 2).any()  # someone crossed the face


def test_measles_follows_the_sir_model(orc):
    """2,000 susceptible and 20 infected persons in a 100 m cube, infection
    radius 3.24179 m, infection probability 0.28510, recovery probability
    0.00521, movement 5.78594 m per 1 h step (Table 4.3).  The thesis
    compares the mean of agent-based runs with dS/dt = -beta S I / N,
    dI/dt = beta S I / N - gamma I, dR/dt = gamma I (beta = 0.06719,
    gamma = 0.00521 per hour): the mean of three runs stays within 2% of N
    of the model's I and R every 100 hours up to 1,000 (measured: 0.6%)."""
    import oracle
    N0, I0, L = 2000, 20, 100.0
    n = N0 + I0
    runs = []
    for seed in range(3):
        rng = np.random.default_rng(100 + seed)
        x = rng.uniform(0.0, L, (n, 3))
        st = np.array([I] * I0 + [S] * N0, np.uint8)
        series = []
        for k in range(10):
            x, st = oracle.sir_step(x, st, 3.24179, 0.28510, 0.00521, 5.78594, L, seed=seed, t0=100 * k, steps=100)
            series.append(((st == I).sum(), (st == R).sum()))
        runs.append(series)
    abm = np.mean(np.array(runs, dtype=np.float64), axis=0)
    beta, gamma = 0.06719, 0.00521

    def f(y):
        s, i, _ = y
        return np.array([-beta * s * i / n, beta * s * i / n - gamma * i, gamma * i])

    y = np.array([float(N0), float(I0), 0.0])
    h = 0.1
    ode = []
    for step in range(1, 10001):
        k1 = f(y)
        k2 = f(y + h / 2 * k1)
        k3 = f(y + h / 2 * k2)
        k4 = f(y + h * k3)
        y = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if step % 1000 == 0:
            ode.append((y[1], y[2]))
    ode = np.array(ode)
    assert np.abs(abm - ode).max() <= 0.02 * n, np.c_[abm, ode]
    # and the epidemic happened: most of the population recovered by 1,000 h
    assert abm[-1, 1] > 0.9 * n
