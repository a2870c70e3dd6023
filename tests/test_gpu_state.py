"""Checkpoint state: bdm_get_state / bdm_set_state.

A simulation saved after N iterations and restored (into the same context,
a new one, or another simulation of a context) continues exactly as the
saved one would have: in the FP64 path, whose trajectories equal the
oracle's bit for bit, every position, diameter, static flag and nnz of the
next iterations is the same bit for bit, and equal to the oracle after N + M
iterations.  This covers static detection (its history: changed flags, nnz,
the last grid and the boxes of the last iteration), growth and division (the
iteration counter is the counter of the division axes' random numbers) and
re-sorting (storage order is not part of the state).
"""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu


def scenes():
    from tests.test_oracle_pins import perturbed_scene
    xyz, d = perturbed_scene()
    base = workloads.clustered(n_clusters=5, per_cluster=700, side=600.0, sigma=25.0, seed=2)
    return [
        ("perturbed_static", workloads.Population(xyz, d, workloads.SimParams(dt=0.05, precision=0, detect_static=1))),
        ("clusters_static_sorted", workloads.Population(base.xyz, base.diameter,
                                                        workloads.SimParams(precision=0, detect_static=1,
                                                                            sort_interval=4))),
        ("growth", workloads.growth_division(shape=(4, 4, 4), cap_factor=8, precision=0)),
    ]


def make(pops, **kw):
    from paper_2503_10796_gb300 import binding
    pops = pops if isinstance(pops, list) else [pops]
    ctx = binding.Context([binding.make_params(p.params, **kw) for p in pops],
                          sum(max(p.n, p.params.capacity) for p in pops) + 16)
    for s, p in enumerate(pops):
        ctx.set_agents(s, p.xyz, p.diameter)
    return ctx


def snapshot(ctx, sim=0):
    x, d = ctx.get_agents(sim)
    F, nnz, st = ctx.forces(sim)
    return x, d, nnz, st


@pytest.mark.parametrize("k", range(3))
def test_resume_is_bit_identical(orc, k):
    import oracle
    name, pop = scenes()[k]
    N, M = 17, 12
    a = make(pop)
    a.step(N)
    state = a.get_state(0)
    traj = []
    for _ in range(M):
        a.step(1)
        traj.append(snapshot(a))
    # a new context whose simulation never had agents set
    from paper_2503_10796_gb300 import binding
    b = binding.Context([binding.make_params(pop.params)], max(pop.n, pop.params.capacity) + 16)
    b.set_state(0, state)
    assert b.stats(0)["iterations"] == N
    for t in range(M):
        b.step(1)
        got = snapshot(b)
        for u, v in zip(got, traj[t]):
            assert np.array_equal(u, v), (name, t)
    # the same context, rewound
    a.set_state(0, state)
    a.step(M)
    for u, v in zip(snapshot(a), traj[-1]):
        assert np.array_equal(u, v), name
    # and the oracle over N + M iterations
    o = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    o.step(N + M)
    x_o, d_o, _ = o.get()
    assert np.array_equal(traj[-1][0], x_o) and np.array_equal(traj[-1][1], d_o), name
    _, _, nnz_o, st_o, _ = o.last()
    assert np.array_equal(traj[-1][3], st_o) and np.array_equal(traj[-1][2], np.minimum(nnz_o, 255)), name


def test_state_moves_between_simulations(orc):
    """A state saved from simulation 1 of one context continues in
    simulation 0 of another that also holds other simulations."""
    pops = workloads.batched_sweep(n_sims=3, lo=200, hi=2000, seed=5, precision=0)
    a = make(pops)
    a.step(6)
    state = a.get_state(1)
    a.step(5)
    want, _ = a.get_agents(1)
    b = make([pops[1], pops[2]])
    b.set_state(0, state)
    b.step(5)
    got, _ = b.get_agents(0)
    assert np.array_equal(got, want)


def test_fp32_resume_within_tolerance(orc):
    pop = workloads.clustered(n_clusters=4, per_cluster=2000, side=500.0, sigma=30.0, seed=1)
    a = make(pop)
    a.step(5)
    state = a.get_state(0)
    a.step(5)
    want, _ = a.get_agents(0)
    b = make(pop)
    b.set_state(0, state)
    b.step(5)
    got, _ = b.get_agents(0)
    # FP32 forces are summed by atomics: the same to rounding, not bitwise
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-4 * pop.diameter.max())


def test_invalid_states_are_rejected(orc):
    from paper_2503_10796_gb300 import binding
    pop = workloads.plain_fp64(n=200, precision=0)
    a = make(pop)
    a.step(2)
    state = a.get_state(0)
    assert len(state) == 144 + 200 * 50
    b = make(pop)
    x_before, _ = b.get_agents(0)
    for bad in (state[:-8], b"NOTSTATE" + state[8:], state[:144]):
        with pytest.raises(binding.BdmError) as e:
            b.set_state(0, bad)
        assert e.value.code == -1
    # a NaN position inside an otherwise valid state
    arr = bytearray(state)
    arr[144 + 8 * 7: 144 + 8 * 8] = np.array([np.nan]).tobytes()
    with pytest.raises(binding.BdmError) as e:
        b.set_state(0, bytes(arr))
    assert e.value.code == -1
    # nothing changed by the rejected calls
    x_after, _ = b.get_agents(0)
    assert np.array_equal(x_before, x_after)
    # a capacity too small for the state's agents
    small = make(workloads.plain_fp64(n=50, precision=0))
    with pytest.raises(binding.BdmError) as e:
        small.set_state(0, state)
    assert e.value.code == -4
