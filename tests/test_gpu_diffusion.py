"""Parity of the soma-clustering slice on the GPU (through the C ABI) with
the diffusion oracle: Eq 4.3 steps, secretion (Algorithm 6) and chemotaxis
(Algorithm 7) bit for bit.  The GPU evaluates every FP64 operation in the
order of the definition; secretion adds equal quantities, whose sum does not
depend on the order of the atomics."""
import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu


def ctx_with(pop):
    from paper_2503_10796_gb300 import binding
    ctx = binding.Context([binding.make_params(pop.params)], pop.n + 16)
    ctx.set_agents(0, pop.xyz, pop.diameter)
    return ctx


def empty_ctx():
    from paper_2503_10796_gb300 import binding
    return binding.Context([binding.make_params()], 16)


@pytest.mark.parametrize("shape,h,nu,mu,dt,steps", [
    ((23, 29, 37), (1.0, 2.0, 0.5), 1.0, 0.5, 0.01, 5),    # ragged, anisotropic
    ((1, 1, 1), (1.0, 1.0, 1.0), 2.0, 0.1, 0.05, 3),       # one point: every neighbour outside
    ((1, 40, 1), (1.0, 0.7, 1.0), 0.3, 0.0, 0.2, 4),       # a line along y
    ((8, 8, 8), (1.0, 1.0, 1.0), 1.0, 0.0, 0.1, 0),        # no step
])
def test_diffusion_bit_exact(orc, shape, h, nu, mu, dt, steps):
    import oracle
    rng = np.random.default_rng(1)
    u = rng.uniform(0.0, 1.0, shape)
    want = oracle.diffuse(u.copy(), h, nu, mu, dt, steps)
    ctx = empty_ctx()
    got = ctx.diffuse(u.copy(), (0.0, 0.0, 0.0), h, nu, mu, dt, steps)
    assert np.array_equal(got, want)


def test_diffusion_device_pointers_and_full_size(orc):
    """A 378^3 grid (54M points, the diffusion volume count of the thesis's
    cell-clustering benchmark), two steps on device memory."""
    import torch

    import oracle
    n = 378
    rng = np.random.default_rng(2)
    u = np.zeros((n, n, n))
    u[150:230, 150:230, 150:230] = rng.uniform(0.0, 1.0, (80, 80, 80))
    want = oracle.diffuse(u.copy(), (1.0, 1.0, 1.0), 0.4, 0.01, 0.2, 2)
    ctx = empty_ctx()
    t = torch.from_numpy(u).cuda()
    torch.cuda.synchronize()  # the library works on its own stream
    ctx.diffuse(t, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 0.4, 0.01, 0.2, 2)
    assert np.array_equal(t.cpu().numpy(), want)


def test_secretion_bit_exact(orc):
    import oracle
    pop = workloads.clustered(n_clusters=5, per_cluster=700, side=600.0, sigma=25.0, seed=2)
    lo, h = (-10.0, 20.0, 5.0), (7.0, 6.5, 8.0)
    shape = (80, 90, 85)  # part of the agents lie outside
    u = np.random.default_rng(3).uniform(0.0, 1.0, shape)
    want = oracle.secrete(u.copy(), lo, h, pop.xyz, 0.37)
    ctx = ctx_with(pop)
    got = ctx.secrete(0, u.copy(), lo, h, 0.37)
    assert np.array_equal(got, want)
    assert not np.array_equal(got, u)


def test_chemotaxis_bit_exact_and_marks_agents_changed(orc):
    import oracle
    pop = workloads.clustered(n_clusters=5, per_cluster=700, side=600.0, sigma=25.0, seed=2)
    lo, h = (0.0, 0.0, 0.0), (5.0, 5.0, 5.0)
    n = 120
    c = (np.arange(n) + 0.5) * 5.0
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    u = np.exp(-((X - 300.0) ** 2 + (Y - 250.0) ** 2 + (Z - 320.0) ** 2) / 5.0e4)
    want = oracle.chemotaxis(u, lo, h, pop.xyz, 0.8)
    ctx = ctx_with(pop)
    ctx.chemotaxis(0, u, lo, h, 0.8)
    got, _ = ctx.get_agents(0)
    assert np.array_equal(got, want)
    # the moved agents take part in the next mechanics step as changed ones
    ctx.step(1)
    ctx.sync()


def test_diffusion_rejects_bad_arguments(orc):
    from paper_2503_10796_gb300 import binding
    ctx = empty_ctx()
    u = np.zeros((4, 4, 4))
    with pytest.raises(binding.BdmError):
        ctx.diffuse(u, (0.0, 0.0, 0.0), (1.0, 0.0, 1.0), 1.0, 0.0, 0.1, 1)
    with pytest.raises(binding.BdmError):
        ctx.diffuse(u, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), -1.0, 0.0, 0.1, 1)
    with pytest.raises(binding.BdmError):
        ctx.diffuse(u, (0.0, np.nan, 0.0), (1.0, 1.0, 1.0), 1.0, 0.0, 0.1, 1)
    with pytest.raises(binding.BdmError):  # no agents set
        ctx.secrete(0, u, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1.0)
