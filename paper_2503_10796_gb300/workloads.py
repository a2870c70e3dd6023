"""Seeded synthetic agent populations shaped like the thesis's benchmark models.

This module only draws inputs (positions, diameters, per-simulation
parameters).  It holds none of the mechanics: no grid, no force, no
displacement.  Both the CUDA path (through the C ABI) and the CPU oracle
consume what it returns, so it is the one piece of code they share.

Every generator uses ``numpy.random.default_rng(seed)`` and draws positions
before diameters.  Shapes follow the thesis's synthetic workloads (§4.4.1,
Fig 4.10 population generators; Table 5.1 benchmark simulations; the
cell-proliferation ``Grid3D`` initialisation of §4.7).

Mean sphere volume for d ~ U[8, 12]: E[d^3] = (12^4 - 8^4) / 16 = 1040, so
the mean volume is pi/6 * 1040 = 544.54; cube sides for a target volume
fraction phi are (n * 544.54 / phi)^(1/3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

MEAN_SPHERE_VOLUME = math.pi / 6.0 * 1040.0


@dataclass
class SimParams:
    """Per-simulation parameters (thesis ``Param`` / ``Cell`` attributes)."""
    k: float = 2.0                 # Eq 4.1 repulsion coefficient
    gamma: float = 1.0             # Eq 4.1 adhesion coefficient
    adherence: float = 0.4         # no movement while |F| <= adherence
    max_displacement: float = 3.0  # norm clamp of one step's displacement
    dt: float = 0.01               # simulation time step
    box_length: float = 0.0        # 0: largest diameter of each iteration
    growth_rate: float = 0.0       # volume per unit time (0: no growth)
    divide_volume: float = 0.0     # volume at which a cell divides
    precision: int = 1             # 0: FP64 force path, 1: FP32 force path
    detect_static: int = 0
    sort_interval: int = 0         # Morton re-sort every n iterations (0 never)
    seed: int = 0                  # counter-RNG key (division axes)
    capacity: int = 0              # per-simulation agent cap (0: initial n)
    boundary: int = 0              # 0 open, 1 closed, 2 toroidal space (§4.4.11)
    bound_min: float = 0.0         # the space [bound_min, bound_max] per axis
    bound_max: float = 0.0         #   (closed and toroidal boundaries)
    execution_context: int = 0     # 0 copy, 1 in-place (§5.2)

    def as_dict(self):
        return asdict(self)


@dataclass
class Population:
    xyz: np.ndarray                # (n, 3) float64, caller-ID order
    diameter: np.ndarray           # (n,) float64
    params: SimParams = field(default_factory=SimParams)
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])


def uniform_cube(n: int = 4096, side: float = 160.0, dmin: float = 8.0,
                 dmax: float = 12.0, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Centers uniform in [0, side)^3, diameters uniform [dmin, dmax]."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, side, size=(n, 3))
    d = rng.uniform(dmin, dmax, size=n)
    return xyz, d


def plain_fp64(n: int = 4096, side: float = 160.0, seed: int = 0,
               precision: int = 0) -> Population:
    """Plain mechanics: 4,096 spheres in a 160^3 cube, d ~ U[8, 12]."""
    xyz, d = uniform_cube(n, side, seed=seed)
    p = SimParams(precision=precision)
    return Population(xyz, d, p, f"plain_{n}")


def jittered_lattice(shape=(32, 32, 64), spacing: float = 10.0,
                     jitter: float = 1.0, d: float = 9.0, seed: int = 0):
    """Cubic lattice (x fastest, then y, then z) with U(-jitter, jitter)
    per-axis jitter; every sphere has diameter ``d``."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    base = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64) * spacing
    xyz = base + rng.uniform(-jitter, jitter, size=base.shape)
    diam = np.full(xyz.shape[0], d, dtype=np.float64)
    return xyz, diam


def growth_division(shape=(32, 32, 64), seed: int = 0, precision: int = 1,
                    cap_factor: int = 32, divide_diameter: float = 12.0) -> Population:
    """Cell growth + division: jittered lattice (spacing 10, jitter +-1,
    d = 9), volume growth 4000 per unit time at dt = 0.01, division at the
    volume of a sphere of diameter 12, capacity 32x the initial count."""
    xyz, d = jittered_lattice(shape, seed=seed)
    n = xyz.shape[0]
    vdiv = (math.pi * (divide_diameter * divide_diameter * divide_diameter)) / 6.0
    p = SimParams(growth_rate=4000.0, divide_volume=vdiv, precision=precision,
                  capacity=n * cap_factor, seed=seed)
    return Population(xyz, d, p, f"growth_{n}")


def clustered(n_clusters: int = 64, per_cluster: int = 131072, side: float = 1.0e4,
              sigma: float = 200.0, seed: int = 0, precision: int = 1,
              detect_static: int = 0, sort_interval: int = 10) -> Population:
    """Gaussian clusters: centers uniform in [0, side)^3, offsets N(0, sigma^2)
    per axis, d ~ U[8, 12].  Agents are listed cluster by cluster."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(0.0, side, size=(n_clusters, 3))
    offs = rng.normal(0.0, sigma, size=(n_clusters, per_cluster, 3))
    xyz = (centers[:, None, :] + offs).reshape(-1, 3)
    d = rng.uniform(8.0, 12.0, size=xyz.shape[0])
    p = SimParams(precision=precision, detect_static=detect_static,
                  sort_interval=sort_interval)
    return Population(xyz, d, p, f"clustered_{xyz.shape[0]}")


def cube_side_for_fraction(n: int, phi: float) -> float:
    return (n * MEAN_SPHERE_VOLUME / phi) ** (1.0 / 3.0)


def uniform_fraction(n: int, phi: float = 0.3, seed: int = 0, precision: int = 1,
                     sort_interval: int = 0) -> Population:
    """Large single domain: n spheres uniform in a cube at volume fraction phi."""
    side = cube_side_for_fraction(n, phi)
    xyz, d = uniform_cube(n, side, seed=seed)
    p = SimParams(precision=precision, sort_interval=sort_interval)
    return Population(xyz, d, p, f"uniform_{n}")


def batched_sweep(n_sims: int = 256, lo: float = 1.0e3, hi: float = 2.0e5,
                  phi: float = 0.3, seed: int = 0, precision: int = 1,
                  sort_interval: int = 0) -> list[Population]:
    """Independent simulations with log-uniform agent counts in [lo, hi],
    each in its own cube at volume fraction phi, with k ~ U[1, 4] and
    adherence ~ U[0.1, 1]; gamma = 1, dt = 0.01, max displacement 3."""
    rng = np.random.default_rng(seed)
    counts = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=n_sims))).astype(np.int64)
    ks = rng.uniform(1.0, 4.0, size=n_sims)
    adh = rng.uniform(0.1, 1.0, size=n_sims)
    pops = []
    for s in range(n_sims):
        n = int(counts[s])
        side = cube_side_for_fraction(n, phi)
        xyz = rng.uniform(0.0, side, size=(n, 3))
        d = rng.uniform(8.0, 12.0, size=n)
        p = SimParams(k=float(ks[s]), adherence=float(adh[s]), precision=precision,
                      sort_interval=sort_interval, seed=seed + s)
        pops.append(Population(xyz, d, p, f"sweep_{s}"))
    return pops


# Named workloads (sizes as in the thesis-shaped benchmark list).
WORKLOADS = {
    "plain_fp64_4096": lambda: plain_fp64(),
    "growth_division_65536": lambda: growth_division(),
    "clustered_8M": lambda: clustered(),
    "batched_sweep_256": lambda: batched_sweep(),
    "uniform_200M": lambda: uniform_fraction(200_000_000),
}
