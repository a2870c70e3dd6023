"""Python handle on the plain FP64 CPU oracle (``bdm_oracle.c``: the
mechanics step; ``diffusion_oracle.c``: diffusion, secretion, chemotaxis;
``sir_oracle.c``: the epidemiology use case).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check of
``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``.  The
library path never imports this package.

``build()`` compiles both C files with gcc (``-O2 -ffp-contract=off``, no
fused multiply-add) into ``oracle/_build/libbdm_oracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bdm_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "diffusion_oracle.c"), os.path.join(_HERE, "sir_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libbdm_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcParams(C.Structure):
    _fields_ = [
        ("k", C.c_double), ("gamma", C.c_double), ("adherence", C.c_double),
        ("max_displacement", C.c_double), ("dt", C.c_double), ("box_length", C.c_double),
        ("growth_rate", C.c_double), ("divide_volume", C.c_double),
        ("precision", C.c_int32), ("detect_static", C.c_int32),
        ("sort_interval", C.c_int32), ("boundary", C.c_int32),
        ("seed", C.c_uint64), ("capacity", C.c_int64),
        ("bound_min", C.c_double), ("bound_max", C.c_double),
        ("execution_context", C.c_int32), ("reserved", C.c_int32),
    ]


class SirParams(C.Structure):
    _fields_ = [("radius", C.c_double), ("p_infect", C.c_double), ("p_recover", C.c_double),
                ("speed", C.c_double), ("length", C.c_double), ("seed", C.c_uint64)]


def build(force: bool = False) -> str:
    """Compile the oracle if its library is missing or older than the source."""
    with _lock:
        if (not force and os.path.exists(_LIB_PATH)
                and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f) for f in _SRCS)):
            return _LIB_PATH
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-std=gnu11", "-Wall", "-o", tmp, *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
        return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = C.CDLL(path)
        P = C.POINTER
        dp, i64p, i32p, u8p = P(C.c_double), P(C.c_int64), P(C.c_int32), P(C.c_uint8)
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [P(OrcParams), C.c_int64, dp, dp]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_count.restype = C.c_int64
        L.orc_count.argtypes = [C.c_void_p]
        L.orc_iteration.restype = C.c_int64
        L.orc_iteration.argtypes = [C.c_void_p]
        L.orc_get.argtypes = [C.c_void_p, dp, dp, dp]
        L.orc_last.argtypes = [C.c_void_p, dp, dp, i32p, u8p, u8p]
        L.orc_grid.restype = C.c_int
        L.orc_grid.argtypes = [C.c_void_p, i64p, dp, i64p]
        L.orc_forces.restype = C.c_int
        L.orc_forces.argtypes = [C.c_void_p, i64p, C.c_int64, dp, i32p, dp]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_int32]
        L.orc_remove.restype = C.c_int
        L.orc_remove.argtypes = [C.c_void_p, C.c_int64, i64p]
        L.orc_set_positions.restype = C.c_int
        L.orc_set_positions.argtypes = [C.c_void_p, dp]
        L.orc_neighbors.restype = C.c_int64
        L.orc_neighbors.argtypes = [C.c_void_p, C.c_double, C.c_int64, i64p]
        L.orc_interleave.restype = C.c_uint64
        L.orc_interleave.argtypes = [C.c_int, i64p]
        L.orc_morton_gaps.restype = C.c_int64
        L.orc_morton_gaps.argtypes = [C.c_int, i64p, C.c_int64, i64p, i64p]
        L.orc_morton_sequence.restype = C.c_int64
        L.orc_morton_sequence.argtypes = [C.c_int, i64p, i64p]
        L.orc_morton_agent_order.restype = C.c_int
        L.orc_morton_agent_order.argtypes = [C.c_void_p, i64p]
        L.orc_philox4x64_10.argtypes = [P(C.c_uint64), P(C.c_uint64), P(C.c_uint64)]
        L.orc_division_axis.argtypes = [C.c_uint64, C.c_int64, C.c_int64, dp]
        L.orc_cbrt_rn.restype = C.c_double
        L.orc_cbrt_rn.argtypes = [C.c_double]
        L.orc_diameter_of_volume.restype = C.c_double
        L.orc_diameter_of_volume.argtypes = [C.c_double]
        L.orc_volume_of_diameter.restype = C.c_double
        L.orc_volume_of_diameter.argtypes = [C.c_double]
        L.orc_diffuse.restype = C.c_int
        L.orc_diffuse.argtypes = [i64p, dp, C.c_double, C.c_double, C.c_double, C.c_int32, dp]
        L.orc_secrete.restype = C.c_int
        L.orc_secrete.argtypes = [dp, dp, i64p, dp, C.c_int64, dp, C.c_double]
        L.orc_gradient.restype = C.c_int
        L.orc_gradient.argtypes = [dp, dp, i64p, dp, C.c_int64, dp, dp]
        L.orc_chemotaxis.restype = C.c_int
        L.orc_chemotaxis.argtypes = [dp, dp, i64p, dp, C.c_int64, dp, C.c_double]
        L.orc_sir_step.restype = C.c_int
        L.orc_sir_step.argtypes = [P(SirParams), C.c_int64, dp, u8p, C.c_int64, C.c_int32]
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def make_params(p=None, **kw) -> OrcParams:
    """OrcParams from a ``SimParams``-like object (or keyword overrides)."""
    d = dict(k=2.0, gamma=1.0, adherence=0.4, max_displacement=3.0, dt=0.01,
             box_length=0.0, growth_rate=0.0, divide_volume=0.0, precision=0,
             detect_static=0, sort_interval=0, seed=0, capacity=0, boundary=0,
             bound_min=0.0, bound_max=0.0, execution_context=0)
    if p is not None:
        src = p.as_dict() if hasattr(p, "as_dict") else dict(p)
        for k in d:
            if k in src:
                d[k] = src[k]
    d.update(kw)
    return OrcParams(d["k"], d["gamma"], d["adherence"], d["max_displacement"], d["dt"],
                     d["box_length"], d["growth_rate"], d["divide_volume"], int(d["precision"]),
                     int(d["detect_static"]), int(d["sort_interval"]), int(d["boundary"]), int(d["seed"]),
                     int(d["capacity"]), float(d["bound_min"]), float(d["bound_max"]),
                     int(d["execution_context"]), 0)


class Sim:
    """One oracle simulation (agents in caller-ID order)."""

    def __init__(self, xyz, diameter, params=None, **kw):
        self._L = lib()
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(diameter, dtype=np.float64).reshape(-1)
        self.params = make_params(params, **kw)
        h = self._L.orc_create(C.byref(self.params), xyz.shape[0], _ptr(xyz, C.c_double), _ptr(d, C.c_double))
        if not h:
            raise ValueError("oracle rejected the input (non-finite value or diameter <= 0)")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    @property
    def n(self) -> int:
        return int(self._L.orc_count(self._h))

    @property
    def iteration(self) -> int:
        return int(self._L.orc_iteration(self._h))

    def step(self, iterations: int = 1):
        rc = self._L.orc_step(self._h, int(iterations))
        if rc:
            raise RuntimeError(f"oracle step failed ({rc})")

    def remove(self, ids):
        """Remove the agents `ids` (the swaps of §5.3.2, see orc_remove)."""
        ids = np.ascontiguousarray(ids, dtype=np.int64).reshape(-1)
        rc = self._L.orc_remove(self._h, ids.shape[0], _ptr(ids, C.c_int64))
        if rc:
            raise ValueError("oracle rejected the removal (IDs out of range or repeated)")

    def set_positions(self, xyz):
        """New positions of the current agents by ID (orc_set_positions)."""
        x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        if x.shape[0] != self.n:
            raise ValueError("one position per agent")
        if self._L.orc_set_positions(self._h, _ptr(x, C.c_double)):
            raise ValueError("a position outside the space")

    def get(self):
        n = self.n
        xyz = np.empty((n, 3)); d = np.empty(n); v = np.empty(n)
        self._L.orc_get(self._h, _ptr(xyz, C.c_double), _ptr(d, C.c_double), _ptr(v, C.c_double))
        return xyz, d, v

    def last(self):
        """Force, displacement, nnz, static and changed flags of the last iteration."""
        n = self.n
        F = np.empty((n, 3)); D = np.empty((n, 3)); nnz = np.empty(n, np.int32)
        st = np.empty(n, np.uint8); ch = np.empty(n, np.uint8)
        self._L.orc_last(self._h, _ptr(F, C.c_double), _ptr(D, C.c_double), _ptr(nnz, C.c_int32),
                         _ptr(st, C.c_uint8), _ptr(ch, C.c_uint8))
        return F, D, nnz, st.astype(bool), ch.astype(bool)

    def grid(self):
        n = self.n
        box = np.empty(n, np.int64); ol = np.empty(4); dims = np.empty(3, np.int64)
        rc = self._L.orc_grid(self._h, _ptr(box, C.c_int64), _ptr(ol, C.c_double), _ptr(dims, C.c_int64))
        if rc:
            raise RuntimeError(f"oracle grid failed ({rc})")
        return box, ol, dims

    def forces(self, ids=None):
        """(F, nnz, magnitude sum) from the current snapshot, no static skip."""
        if ids is None:
            m = self.n
            idp = None
        else:
            ids = np.ascontiguousarray(ids, dtype=np.int64)
            m = ids.shape[0]
            idp = _ptr(ids, C.c_int64)
        F = np.empty((m, 3)); nnz = np.empty(m, np.int32); sm = np.empty(m)
        rc = self._L.orc_forces(self._h, idp, m, _ptr(F, C.c_double), _ptr(nnz, C.c_int32), _ptr(sm, C.c_double))
        if rc:
            raise RuntimeError(f"oracle forces failed ({rc})")
        return F, nnz, sm

    def neighbors(self, radius: float) -> np.ndarray:
        cnt = self._L.orc_neighbors(self._h, float(radius), 0, None)
        if cnt < 0:
            raise RuntimeError("oracle neighbor query failed")
        out = np.empty((max(cnt, 1), 2), np.int64)
        cnt2 = self._L.orc_neighbors(self._h, float(radius), cnt, _ptr(out, C.c_int64))
        assert cnt2 == cnt
        return out[:cnt]

    def morton_agent_order(self) -> np.ndarray:
        ids = np.empty(max(self.n, 1), np.int64)
        rc = self._L.orc_morton_agent_order(self._h, _ptr(ids, C.c_int64))
        if rc:
            raise RuntimeError("oracle morton order failed")
        return ids[: self.n]


def interleave(dim: int, c) -> int:
    c = np.ascontiguousarray(c, dtype=np.int64)
    return int(lib().orc_interleave(dim, _ptr(c, C.c_int64)))


def morton_gaps(dim: int, dims):
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    n = lib().orc_morton_gaps(dim, _ptr(dims, C.c_int64), 0, None, None)
    c = np.empty(max(n, 1), np.int64); o = np.empty(max(n, 1), np.int64)
    lib().orc_morton_gaps(dim, _ptr(dims, C.c_int64), n, _ptr(c, C.c_int64), _ptr(o, C.c_int64))
    return list(zip(c[:n].tolist(), o[:n].tolist()))


def morton_sequence(dim: int, dims) -> np.ndarray:
    dims = np.ascontiguousarray(dims, dtype=np.int64)
    nb = int(np.prod(dims))
    out = np.empty(max(nb, 1), np.int64)
    lib().orc_morton_sequence(dim, _ptr(dims, C.c_int64), _ptr(out, C.c_int64))
    return out[:nb]


def philox4x64_10(ctr, key):
    c = (C.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64_10(c, k, o)
    return [int(v) for v in o]


def division_axis(seed: int, agent_id: int, t: int) -> np.ndarray:
    u = np.empty(3)
    lib().orc_division_axis(int(seed), int(agent_id), int(t), _ptr(u, C.c_double))
    return u


def cbrt_rn(x: float) -> float:
    return float(lib().orc_cbrt_rn(float(x)))


def diameter_of_volume(v: float) -> float:
    return float(lib().orc_diameter_of_volume(float(v)))


def volume_of_diameter(d: float) -> float:
    return float(lib().orc_volume_of_diameter(float(d)))


# --------------------------------------------------- diffusion slice ----
# Grids are numpy arrays of shape (n_z, n_y, n_x), C order (x fastest), the
# layout of the C functions.  lo, h: 3-vectors (x, y, z).

def _grid_args(u, lo=None, h=None):
    if u.dtype != np.float64 or not u.flags.c_contiguous or u.ndim != 3:
        raise ValueError("u must be a C-contiguous float64 array of shape (nz, ny, nx)")
    n = np.array([u.shape[2], u.shape[1], u.shape[0]], dtype=np.int64)
    lo = np.ascontiguousarray(lo if lo is not None else np.zeros(3), dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    return n, lo, h


def diffuse(u, h, nu: float, mu: float, dt: float, steps: int = 1):
    """Eq 4.3 applied `steps` times to u in place (zero outside the grid)."""
    n, _, h = _grid_args(u, None, h)
    rc = lib().orc_diffuse(_ptr(n, C.c_int64), _ptr(h, C.c_double), float(nu), float(mu), float(dt),
                           int(steps), _ptr(u, C.c_double))
    if rc:
        raise RuntimeError(f"oracle diffusion failed ({rc})")
    return u


def secrete(u, lo, h, xyz, quantity: float):
    """Algorithm 6: each agent adds `quantity` to the box of its center."""
    n, lo, h = _grid_args(u, lo, h)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    lib().orc_secrete(_ptr(lo, C.c_double), _ptr(h, C.c_double), _ptr(n, C.c_int64), _ptr(u, C.c_double),
                      xyz.shape[0], _ptr(xyz, C.c_double), float(quantity))
    return u


def gradient(u, lo, h, xyz):
    """Normalized central-difference gradient of each position's box."""
    n, lo, h = _grid_args(u, lo, h)
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    g = np.empty_like(xyz)
    lib().orc_gradient(_ptr(lo, C.c_double), _ptr(h, C.c_double), _ptr(n, C.c_int64), _ptr(u, C.c_double),
                       xyz.shape[0], _ptr(xyz, C.c_double), _ptr(g, C.c_double))
    return g


def chemotaxis(u, lo, h, xyz, weight: float):
    """Algorithm 7: positions moved by weight x normalized gradient (a copy)."""
    n, lo, h = _grid_args(u, lo, h)
    x = np.array(xyz, dtype=np.float64).reshape(-1, 3)
    lib().orc_chemotaxis(_ptr(lo, C.c_double), _ptr(h, C.c_double), _ptr(n, C.c_int64), _ptr(u, C.c_double),
                         x.shape[0], _ptr(x, C.c_double), float(weight))
    return x


# ------------------------------------------------------- epidemiology ----
SUSCEPTIBLE, INFECTED, RECOVERED = 0, 1, 2


def sir_step(xyz, state, radius: float, p_infect: float, p_recover: float, speed: float, length: float,
             seed: int = 0, t0: int = 0, steps: int = 1):
    """Algorithms 3-5 for `steps` steps from step t0, on copies of xyz
    (n x 3) and state (n, uint8: 0 S, 1 I, 2 R); returns (xyz, state)."""
    x = np.array(xyz, dtype=np.float64).reshape(-1, 3)
    st = np.array(state, dtype=np.uint8).reshape(-1)
    prm = SirParams(float(radius), float(p_infect), float(p_recover), float(speed), float(length), int(seed))
    rc = lib().orc_sir_step(C.byref(prm), x.shape[0], _ptr(x, C.c_double), _ptr(st, C.c_uint8), int(t0),
                            int(steps))
    if rc:
        raise RuntimeError(f"oracle SIR step failed ({rc})")
    return x, st
