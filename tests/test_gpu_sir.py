"""Parity of the epidemiology step on the GPU (through the C ABI) with the
oracle (§4.6.3, Algorithms 3-5): states and positions bit for bit, the
same counter-based draws on both sides."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

S, I, R = 0, 1, 2
MEASLES = dict(radius=3.24179, p_infect=0.28510, p_recover=0.00521, speed=5.78594, length=100.0)


def persons_ctx(xyz):
    from paper_2503_10796_gb300 import binding
    n = xyz.shape[0]
    ctx = binding.Context([binding.make_params()], n + 16)
    ctx.set_agents(0, xyz, np.full(n, 1.0))
    return ctx


@pytest.mark.parametrize("steps", [1, 40])
def test_measles_steps_bit_exact(orc, steps):
    import oracle
    rng = np.random.default_rng(11)
    n = 2020
    xyz = rng.uniform(0.0, 100.0, (n, 3))
    st = np.array([I] * 20 + [S] * 2000, np.uint8)
    want_x, want_s = oracle.sir_step(xyz, st, seed=5, t0=3, steps=steps, **MEASLES)
    ctx = persons_ctx(xyz)
    got_s = st.copy()
    ctx.sir_step(0, got_s, seed=5, t0=3, steps=steps, **MEASLES)
    got_x, _ = ctx.get_agents(0)
    assert np.array_equal(got_s, want_s)
    assert np.array_equal(got_x, want_x)
    assert (got_s != st).any()


def test_chain_and_rules(orc):
    import oracle
    xyz = np.array([[10.0, 10.0, 10.0], [12.0, 10.0, 10.0], [14.5, 10.0, 10.0], [50.0, 50.0, 50.0]])
    st = np.array([I, S, S, R], np.uint8)
    prm = dict(radius=3.0, p_infect=1.0, p_recover=0.0, speed=0.0, length=100.0)
    ctx = persons_ctx(xyz)
    ctx.sir_step(0, st, **prm)
    assert st.tolist() == [I, I, S, R]
    ctx.sir_step(0, st, t0=1, **prm)
    assert st.tolist() == [I, I, I, R]
    want_x, want_s = oracle.sir_step(xyz, [I, S, S, R], steps=2, **prm)
    got_x, _ = ctx.get_agents(0)
    assert np.array_equal(got_x, want_x) and st.tolist() == want_s.tolist()


def test_device_states_and_bad_arguments(orc):
    import torch

    import oracle
    from paper_2503_10796_gb300 import binding
    rng = np.random.default_rng(2)
    xyz = rng.uniform(0.0, 100.0, (500, 3))
    st = np.array([I] * 10 + [S] * 490, np.uint8)
    want_x, want_s = oracle.sir_step(xyz, st, seed=1, steps=5, **MEASLES)
    ctx = persons_ctx(xyz)
    t = torch.from_numpy(st.copy()).cuda()
    torch.cuda.synchronize()
    ctx.sir_step(0, t, seed=1, steps=5, **MEASLES)
    assert np.array_equal(t.cpu().numpy(), want_s)
    with pytest.raises(binding.BdmError):
        ctx.sir_step(0, st.copy(), **dict(MEASLES, p_infect=1.5))
    with pytest.raises(binding.BdmError):
        ctx.sir_step(0, np.full(500, 3, np.uint8), **MEASLES)
