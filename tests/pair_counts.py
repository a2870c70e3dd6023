"""Per-agent pair counts for the parity tests.

The overlap count of an agent (pairs with delta > 0, Eq 4.1) is fixed by the
pair set, which both paths decide exactly, so the GPU's count must equal the
count of the oracle's overlap pairs.  The non-zero-force count (nnz) can
differ only for a pair whose force F_N = k delta - gamma sqrt(r delta) lies
within FP32 rounding of zero (the crossover delta = gamma^2 r / k^2): such a
disagreement is allowed and reported, any other is a failure.
"""
import numpy as np


def overlap_counts(n, pairs):
    """Overlapping pairs per agent from an (m, 2) array of pairs."""
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    return np.bincount(pairs.ravel(), minlength=n).astype(np.int64)[:n]


def pair_force_scale(xyz, d, pairs, k, gamma):
    """|F_N| and k delta + gamma sqrt(r delta) of every pair (FP64)."""
    i, j = pairs[:, 0], pairs[:, 1]
    dist = np.sqrt(((xyz[i] - xyz[j]) ** 2).sum(axis=1))
    ri, rj = 0.5 * d[i], 0.5 * d[j]
    delta = (ri + rj) - dist
    r = ri * rj / (ri + rj)
    rep, adh = k * delta, gamma * np.sqrt(np.maximum(r * delta, 0.0))
    return np.abs(rep - adh), rep + adh


def check_nnz(nnz_gpu, nnz_orc, ids, xyz, d, pairs, k, gamma, rel=1e-5):
    """nnz of the agents `ids` (GPU and oracle values given for them) equal,
    except agents with a pair at the force crossover; returns the number of
    those excepted disagreements."""
    nnz_gpu = np.asarray(nnz_gpu)
    nnz_orc = np.asarray(nnz_orc)
    bad = np.flatnonzero(nnz_gpu != nnz_orc)
    if bad.size == 0:
        return 0
    pairs = np.asarray(pairs, np.int64).reshape(-1, 2)
    fn, scale = pair_force_scale(xyz, d, pairs, k, gamma)
    near = fn <= rel * scale
    near_agents = set(pairs[near].ravel().tolist())
    unexplained = [int(ids[b]) for b in bad if int(ids[b]) not in near_agents]
    assert not unexplained, ("nnz differs away from the force crossover", unexplained[:10])
    print(f"NNZ: {bad.size} agents differ at the force crossover (|F_N| within FP32 rounding of 0)")
    return bad.size
