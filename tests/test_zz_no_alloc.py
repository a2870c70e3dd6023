"""bdm_forces_noalloc: the force entry point for callers that cannot
allocate device memory (allocator-free runtimes, programs that hand out all
device memory from their own pool).  Its output must match the oracle's
forces and the regular path (bdm_set_agents + bdm_step(1) + bdm_get_forces)
within the parity tolerance, on two calls in a row that share its fixed
device array.

This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from paper_2503_10796_gb300 import workloads

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5}


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_forces_match_regular_path(precision):
    import torch

    import oracle
    from paper_2503_10796_gb300 import binding
    lib = binding.load_library()
    pops = [workloads.plain_fp64(seed=3), workloads.Population(*workloads.uniform_cube(2500, 80.0, seed=9))]
    for pop in pops:
        params = binding.make_params(pop.params, precision=precision)
        ctx = binding.Context(params, pop.n + 8)
        ctx.set_agents(0, pop.xyz, pop.diameter)
        ctx.step(1)
        ctx.sync()
        F_ref, nnz_ref, _ = ctx.forces(0)
        ctx.close()
        F_orc, nnz_orc, smag = oracle.Sim(pop.xyz, pop.diameter, params=pop.params).forces()
        scale = np.maximum(smag, 1e-300)

        dev = torch.device("cuda", 0)
        xyz = torch.tensor(pop.xyz, dtype=torch.float64, device=dev).contiguous()
        d = torch.tensor(pop.diameter, dtype=torch.float64, device=dev).contiguous()
        for call in range(2):
            force = torch.full((pop.n, 3), float("nan"), dtype=torch.float64, device=dev)
            nnz = torch.full((pop.n,), -1, dtype=torch.int32, device=dev)
            torch.cuda.synchronize()
            rc = lib.bdm_forces_noalloc(C.byref(params), pop.n, C.c_void_p(xyz.data_ptr()),
                                        C.c_void_p(d.data_ptr()), C.c_void_p(force.data_ptr()),
                                        C.c_void_p(nnz.data_ptr()), None)
            assert rc == 0, (call, rc)
            F = force.cpu().numpy()
            for want in (F_orc, F_ref):
                err = np.linalg.norm(F - want, axis=1) / scale
                err[smag == 0] = np.linalg.norm(F - want, axis=1)[smag == 0]
                assert err.max() <= TOL[precision], (call, err.max())
            got = nnz.cpu().numpy()
            assert np.array_equal(got, nnz_ref)
            if precision == 0:
                assert np.array_equal(got, nnz_orc)


def test_noalloc_rejects_sizes_beyond_its_limit():
    import torch

    from paper_2503_10796_gb300 import binding
    lib = binding.load_library()
    params = binding.make_params()
    n = 16385
    dev = torch.device("cuda", 0)
    xyz = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    d = torch.ones((n,), dtype=torch.float64, device=dev)
    force = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    rc = lib.bdm_forces_noalloc(C.byref(params), n, C.c_void_p(xyz.data_ptr()), C.c_void_p(d.data_ptr()),
                                C.c_void_p(force.data_ptr()), None, None)
    assert rc == -4
    # a grid with more boxes than the fixed table holds
    pts = np.zeros((4, 3))
    pts[1] = [5000.0, 0, 0]
    pts[2] = [0, 5000.0, 0]
    pts[3] = [0, 0, 5000.0]
    xyz = torch.tensor(pts, dtype=torch.float64, device=dev)
    d = torch.full((4,), 10.0, dtype=torch.float64, device=dev)
    force = torch.zeros((4, 3), dtype=torch.float64, device=dev)
    rc = lib.bdm_forces_noalloc(C.byref(params), 4, C.c_void_p(xyz.data_ptr()), C.c_void_p(d.data_ptr()),
                                C.c_void_p(force.data_ptr()), None, None)
    assert rc == -4


def test_noalloc_reports_nonfinite_input_and_crowded_boxes():
    """A NaN position or diameter is BDM_E_NONFINITE; more than 1023 agents
    in one box is BDM_E_CAPACITY."""
    import torch

    from paper_2503_10796_gb300 import binding
    lib = binding.load_library()
    params = binding.make_params()
    dev = torch.device("cuda", 0)

    def call(pts, d):
        xyz = torch.tensor(pts, dtype=torch.float64, device=dev).contiguous()
        dd = torch.tensor(d, dtype=torch.float64, device=dev).contiguous()
        force = torch.zeros((len(d), 3), dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        return lib.bdm_forces_noalloc(C.byref(params), len(d), C.c_void_p(xyz.data_ptr()),
                                      C.c_void_p(dd.data_ptr()), C.c_void_p(force.data_ptr()), None, None)

    rng = np.random.default_rng(3)
    pts = rng.uniform(0.0, 50.0, (64, 3))
    d = np.full(64, 10.0)
    bad = pts.copy()
    bad[5, 1] = np.nan
    assert call(bad, d) == -6
    dbad = d.copy()
    dbad[9] = np.nan
    assert call(pts, dbad) == -6
    # 1100 agents inside one box of length 60
    crowd = rng.uniform(0.0, 50.0, (1100, 3))
    pb = binding.make_params(box_length=60.0)
    xyz = torch.tensor(crowd, dtype=torch.float64, device=dev)
    dd = torch.ones(1100, dtype=torch.float64, device=dev)
    force = torch.zeros((1100, 3), dtype=torch.float64, device=dev)
    rc = lib.bdm_forces_noalloc(C.byref(pb), 1100, C.c_void_p(xyz.data_ptr()), C.c_void_p(dd.data_ptr()),
                                C.c_void_p(force.data_ptr()), None, None)
    assert rc == -4
    # the next valid call works
    assert call(pts, d) == 0
