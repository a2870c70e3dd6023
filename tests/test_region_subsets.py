"""The sub-population argument of the full-size parity tests, checked on the
oracle alone: a region's agents plus the agents that fix the grid give the
full population's box indices, and the agents at least one largest diameter
inside the region keep their overlap pairs, forces and one-step positions
bit for bit (the oracle sums in ascending ID order, which ascending subset
IDs preserve)."""
import numpy as np

from paper_2503_10796_gb300 import workloads
from test_gpu_full_size import region_subset


def test_region_subset_reproduces_full_population(orc):
    import oracle
    pop = workloads.clustered(n_clusters=2, per_cluster=65536, side=3000.0, seed=4)
    full = oracle.Sim(pop.xyz, pop.diameter, pop.params)
    fbox, fol, fdims = full.grid()
    fpairs = full.neighbors(-1.0)
    c = pop.xyz[:65536].mean(axis=0)
    for off in (0.0, 250.0):
        lo = c + np.array([off, -off, 0.0]) - 90.0
        ids, core = region_subset(pop.xyz, pop.diameter, lo, lo + 180.0)
        assert core.sum() >= 200
        sub = oracle.Sim(pop.xyz[ids], pop.diameter[ids], pop.params)
        sbox, sol, sdims = sub.grid()
        assert np.array_equal(sol, fol) and np.array_equal(sdims, fdims)
        assert np.array_equal(sbox, fbox[ids])
        in_core = np.zeros(pop.n, bool)
        in_core[ids[core]] = True
        want = fpairs[in_core[fpairs[:, 0]] | in_core[fpairs[:, 1]]]
        got = ids[sub.neighbors(-1.0)]
        got = got[in_core[got[:, 0]] | in_core[got[:, 1]]]
        assert len(want) > 0 and np.array_equal(got, want)
        loc = np.flatnonzero(core)
        F1, n1, s1 = sub.forces(loc)
        F2, n2, s2 = full.forces(ids[loc])
        assert np.array_equal(F1, F2) and np.array_equal(n1, n2) and np.array_equal(s1, s2)
    # one step of the last region against one step of the whole population
    sub.step(1)
    full.step(1)
    xs, _, _ = sub.get()
    xf, _, _ = full.get()
    assert np.array_equal(xs[loc], xf[ids[loc]])
