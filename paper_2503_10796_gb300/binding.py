"""Thin ctypes binding of the C ABI (``include/bdm.h``).

Argument marshalling only: every step of the mechanics runs in the CUDA
library.  There is no fallback: if ``_build/libbdm.so`` cannot be loaded the
import of the library fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

BDM_OK = 0
ERRORS = {-1: "BDM_E_INVAL", -2: "BDM_E_NOMEM", -3: "BDM_E_CUDA", -4: "BDM_E_CAPACITY",
          -5: "BDM_E_TIMEOUT", -6: "BDM_E_NONFINITE", -7: "BDM_E_STATE"}
PREC_FP64, PREC_FP32_FORCE = 0, 1
DEVICE_PTRS = 1
NUM_STAGES = 9

# Every symbol the header declares, with (restype, argtypes).
_P = C.POINTER
_vp, _i32, _i64, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double


class BdmParams(C.Structure):
    _fields_ = [
        ("k", C.c_double), ("gamma", C.c_double), ("adherence", C.c_double),
        ("max_displacement", C.c_double), ("dt", C.c_double), ("box_length", C.c_double),
        ("growth_rate", C.c_double), ("divide_volume", C.c_double),
        ("precision", C.c_int32), ("detect_static", C.c_int32), ("sort_interval", C.c_int32),
        ("boundary", C.c_int32), ("seed", C.c_uint64), ("capacity", C.c_int64),
        ("bound_min", C.c_double), ("bound_max", C.c_double),
        ("execution_context", C.c_int32), ("reserved", C.c_int32),
    ]


class BdmStats(C.Structure):
    _fields_ = [("agents", C.c_int64), ("iterations", C.c_int64), ("static_agents", C.c_int64),
                ("moved_agents", C.c_int64), ("origin_len", C.c_double * 4), ("dims", C.c_int64 * 3),
                ("agent_updates", C.c_int64), ("reserved", C.c_int64 * 3)]


class BdmTuning(C.Structure):
    _fields_ = [("force_variant", C.c_int32), ("sort_interval", C.c_int32), ("sort_curve", C.c_int32),
                ("box_scale_pct", C.c_int32), ("iter_batch", C.c_int32), ("test_flags", C.c_int32),
                ("grid_reuse", C.c_int32), ("reserved", C.c_int32)]


TUNING_FIELDS = ("force_variant", "sort_interval", "sort_curve", "box_scale_pct", "iter_batch", "test_flags",
                 "grid_reuse")
TUNE_FORCE, TUNE_CURVE, TUNE_INTERVAL, TUNE_BOX, TUNE_BATCH, TUNE_ALL = 1, 2, 4, 8, 16, 31


class BdmCounters(C.Structure):
    _fields_ = [("graph_launches", C.c_int64), ("kernels", C.c_int64), ("graph_iterations", C.c_int64),
                ("grid_builds", C.c_int64), ("reserved", C.c_int64 * 4)]


class BdmDiffusionGrid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("h", C.c_double * 3), ("n", C.c_int64 * 3)]


class BdmSirParams(C.Structure):
    _fields_ = [("radius", C.c_double), ("p_infect", C.c_double), ("p_recover", C.c_double),
                ("speed", C.c_double), ("length", C.c_double), ("seed", C.c_uint64)]


SIGNATURES = {
    "bdm_create": (C.c_int, [_P(BdmParams), _i32, _i64, _i32, _vp, _P(_vp)]),
    "bdm_set_agents": (C.c_int, [_vp, _i32, _i64, _vp, _vp, _i32]),
    "bdm_update_agents": (C.c_int, [_vp, _i32, _i64, _vp, _vp, _i32]),
    "bdm_step": (C.c_int, [_vp, _i32]),
    "bdm_get_state": (C.c_int, [_vp, _i32, _vp, _i64, _P(_i64)]),
    "bdm_remove_agents": (C.c_int, [_vp, _i32, _i64, _vp]),
    "bdm_set_ghosts": (C.c_int, [_vp, _i32, _i64, _vp]),
    "bdm_set_agent_kinds": (C.c_int, [_vp, _i32, _i64, _vp]),
    "bdm_set_substance": (C.c_int, [_vp, _i32, _i32, _vp, _vp, C.c_double, C.c_double, C.c_double, C.c_double,
                                    _i32]),
    "bdm_get_substance": (C.c_int, [_vp, _i32, _i32, _vp, _i64, _P(_i64), _i32]),
    "bdm_set_state": (C.c_int, [_vp, _i32, _vp, _i64]),
    "bdm_sync": (C.c_int, [_vp]),
    "bdm_get_agents": (C.c_int, [_vp, _i32, _i64, _vp, _vp, _P(_i64), _i32]),
    "bdm_neighbors": (C.c_int, [_vp, _i32, _dbl, _i64, _vp, _P(_i64)]),
    "bdm_get_grid": (C.c_int, [_vp, _i32, _i64, _vp, _P(_dbl), _P(_i64)]),
    "bdm_get_forces": (C.c_int, [_vp, _i32, _i64, _vp, _vp, _vp, _vp, _P(_i64)]),
    "bdm_get_storage_order": (C.c_int, [_vp, _i32, _i64, _vp, _P(_i64)]),
    "bdm_get_stats": (C.c_int, [_vp, _i32, _P(BdmStats)]),
    "bdm_profile": (C.c_int, [_vp, _i32]),
    "bdm_get_profile": (C.c_int, [_vp, _P(_i64), _P(_dbl), _P(C.c_char_p)]),
    "bdm_set_tuning": (C.c_int, [_vp, _P(BdmTuning)]),
    "bdm_get_tuning": (C.c_int, [_vp, _P(BdmTuning)]),
    "bdm_autotune": (C.c_int, [_vp, _i32, _i32, _P(BdmTuning)]),
    "bdm_get_counters": (C.c_int, [_vp, _P(BdmCounters)]),
    "bdm_forces_noalloc": (C.c_int, [_P(BdmParams), _i64, _vp, _vp, _vp, _vp, _vp]),
    "bdm_diffuse": (C.c_int, [_vp, _P(BdmDiffusionGrid), _vp, _dbl, _dbl, _dbl, _i32, _i32]),
    "bdm_secrete": (C.c_int, [_vp, _i32, _P(BdmDiffusionGrid), _vp, _dbl, _i32]),
    "bdm_chemotaxis": (C.c_int, [_vp, _i32, _P(BdmDiffusionGrid), _vp, _dbl, _i32]),
    "bdm_sir_step": (C.c_int, [_vp, _i32, _P(BdmSirParams), _vp, _i64, _i32, _i32]),
    "bdm_destroy": (None, [_vp]),
    "bdm_last_error": (C.c_char_p, [_vp]),
}

_lib = None


def load_library(path: str | None = None, build: bool = True):
    """Load (building first if needed) the sm_103a library."""
    global _lib
    if _lib is None:
        if path is None:
            path = _build.build() if build else _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"CUDA library not built: {path}")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


class BdmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def make_params(p=None, **kw) -> BdmParams:
    d = dict(k=2.0, gamma=1.0, adherence=0.4, max_displacement=3.0, dt=0.01, box_length=0.0,
             growth_rate=0.0, divide_volume=0.0, precision=PREC_FP32_FORCE, detect_static=0,
             sort_interval=0, seed=0, capacity=0, boundary=0, bound_min=0.0, bound_max=0.0,
             execution_context=0)
    if p is not None:
        src = p.as_dict() if hasattr(p, "as_dict") else dict(p)
        for k in d:
            if k in src:
                d[k] = src[k]
    d.update(kw)
    return BdmParams(d["k"], d["gamma"], d["adherence"], d["max_displacement"], d["dt"], d["box_length"],
                     d["growth_rate"], d["divide_volume"], int(d["precision"]), int(d["detect_static"]),
                     int(d["sort_interval"]), int(d["boundary"]), int(d["seed"]) & (2**64 - 1),
                     int(d["capacity"]), float(d["bound_min"]), float(d["bound_max"]),
                     int(d["execution_context"]), 0)


def _dptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


class Context:
    """A set of independent simulations on one GPU (``bdm_create``)."""

    def __init__(self, params, max_agents_total: int, device: int = 0, stream=None):
        self._lib = load_library()
        plist = params if isinstance(params, (list, tuple)) else [params]
        arr = (BdmParams * len(plist))(*[p if isinstance(p, BdmParams) else make_params(p) for p in plist])
        h = C.c_void_p()
        st = C.c_void_p(stream) if stream else None
        rc = self._lib.bdm_create(arr, len(plist), int(max_agents_total), int(device), st, C.byref(h))
        if rc != BDM_OK:
            raise BdmError(rc, self._lib.bdm_last_error(None).decode())
        self._h = h
        self.n_sims = len(plist)

    def _check_size_query(self, rc, n):
        # BDM_E_CAPACITY with a count is the answer to a size query (cap 0);
        # without one it is an error latched on the device
        if rc == BDM_OK or (rc == -4 and n.value > 0):
            return
        self._check(rc)

    def _check(self, rc):
        if rc != BDM_OK:
            raise BdmError(rc, self._lib.bdm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bdm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- agents ------------------------------------------------------------
    def set_agents(self, sim: int, xyz, diameter):
        """Host numpy arrays, or CUDA torch tensors (passed as device pointers)."""
        if hasattr(xyz, "data_ptr") and getattr(xyz, "is_cuda", False):
            n = int(xyz.shape[0])
            self._check(self._lib.bdm_set_agents(self._h, sim, n, C.c_void_p(xyz.data_ptr()),
                                                 C.c_void_p(diameter.data_ptr()), DEVICE_PTRS))
            return
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        d = np.ascontiguousarray(diameter, dtype=np.float64).reshape(-1)
        if d.shape[0] != xyz.shape[0]:
            raise ValueError("xyz and diameter differ in length")
        self._check(self._lib.bdm_set_agents(self._h, sim, xyz.shape[0], _dptr(xyz), _dptr(d), 0))

    def update_agents(self, sim: int, xyz, diameter=None):
        """New positions (n x 3, by ID) and optionally diameters of the current
        agents, keeping storage order, iteration counter and history."""
        xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        d = None
        if diameter is not None:
            d = np.ascontiguousarray(diameter, dtype=np.float64).reshape(-1)
            if d.shape[0] != xyz.shape[0]:
                raise ValueError("xyz and diameter differ in length")
        self._check(self._lib.bdm_update_agents(self._h, sim, xyz.shape[0], _dptr(xyz),
                                                _dptr(d) if d is not None else None, 0))

    def set_ghosts(self, sim: int, ghost):
        """Ghost flags by ID (bdm_set_ghosts): True marks a read-only
        neighbour, which bdm_step does not move, grow or divide."""
        m = np.ascontiguousarray(np.asarray(ghost).reshape(-1) != 0, dtype=np.uint8)
        self._check(self._lib.bdm_set_ghosts(self._h, sim, m.shape[0], _dptr(m)))

    def get_state(self, sim: int) -> bytes:
        """Checkpoint of simulation `sim` (bdm_get_state) as bytes."""
        n = C.c_int64()
        rc = self._lib.bdm_get_state(self._h, sim, None, 0, C.byref(n))
        self._check_size_query(rc, n)
        buf = C.create_string_buffer(n.value)
        self._check(self._lib.bdm_get_state(self._h, sim, buf, n.value, C.byref(n)))
        return buf.raw[: n.value]

    def set_state(self, sim: int, state: bytes):
        """Replace simulation `sim` by a checkpoint (bdm_set_state)."""
        buf = C.create_string_buffer(bytes(state), len(state))
        self._check(self._lib.bdm_set_state(self._h, sim, buf, len(state)))

    def remove_agents(self, sim: int, ids):
        """Remove the agents `ids` of `sim` (bdm_remove_agents: the swaps of
        the thesis's parallel removal renumber the survivors)."""
        ids = np.ascontiguousarray(ids, dtype=np.int64).reshape(-1)
        self._check(self._lib.bdm_remove_agents(self._h, sim, ids.shape[0], _dptr(ids) if ids.size else None))

    def step(self, iterations: int = 1):
        self._check(self._lib.bdm_step(self._h, int(iterations)))

    def sync(self):
        self._check(self._lib.bdm_sync(self._h))

    def count(self, sim: int) -> int:
        return self.stats(sim)["agents"]

    def get_agents(self, sim: int, out=None):
        """Positions (n x 3) and diameters (n) in ID order.  out: a pair of
        C-contiguous float64 host arrays with room for the agents (pinned
        memory makes the copy a direct DMA); views of their first n rows
        are returned."""
        n = C.c_int64()
        if out is None:
            rc = self._lib.bdm_get_agents(self._h, sim, 0, None, None, C.byref(n), 0)
            self._check_size_query(rc, n)
            xyz = np.empty((n.value, 3)); d = np.empty(n.value)
        else:
            xyz, d = out
            if xyz.dtype != np.float64 or not xyz.flags.c_contiguous or (d is not None and (
                    d.dtype != np.float64 or not d.flags.c_contiguous or xyz.shape[0] != d.shape[0])):
                raise ValueError("out must be C-contiguous float64 arrays (n x 3, n), d may be None")
        self._check(self._lib.bdm_get_agents(self._h, sim, xyz.shape[0], _dptr(xyz),
                                             _dptr(d) if d is not None else None, C.byref(n), 0))
        k = n.value
        if out is not None and k == xyz.shape[0]:
            return xyz, d
        return xyz[:k], (d[:k] if d is not None else None)

    def get_agents_device(self, sim: int, xyz_t, d_t):
        """Write into CUDA tensors (n x 3 and n float64) on the context stream."""
        n = C.c_int64()
        self._check(self._lib.bdm_get_agents(self._h, sim, int(xyz_t.shape[0]), C.c_void_p(xyz_t.data_ptr()),
                                             C.c_void_p(d_t.data_ptr()), C.byref(n), DEVICE_PTRS))
        return n.value

    # -- queries -----------------------------------------------------------
    def neighbors(self, sim: int, radius: float) -> np.ndarray:
        n = C.c_int64()
        rc = self._lib.bdm_neighbors(self._h, sim, float(radius), 0, None, C.byref(n))
        self._check_size_query(rc, n)
        out = np.empty((max(n.value, 1), 2), np.int64)
        self._check(self._lib.bdm_neighbors(self._h, sim, float(radius), n.value, _dptr(out), C.byref(n)))
        return out[: n.value]

    def grid(self, sim: int):
        st = self.stats(sim)
        n = max(st["agents"], 1)
        box = np.empty(n, np.int64); ol = (C.c_double * 4)(); dims = (C.c_int64 * 3)()
        self._check(self._lib.bdm_get_grid(self._h, sim, n, _dptr(box), ol, dims))
        return box[: st["agents"]], np.array(list(ol)), np.array(list(dims), np.int64)

    def forces(self, sim: int, overlaps: bool = False):
        """Force (n x 3), non-zero pair count and static flag per agent ID of
        the last iteration; with overlaps=True also the overlapping-pair
        count (delta > 0; -1 for static agents)."""
        n = C.c_int64()
        rc = self._lib.bdm_get_forces(self._h, sim, 0, None, None, None, None, C.byref(n))
        self._check_size_query(rc, n)
        m = max(n.value, 1)
        F = np.empty((m, 3)); nnz = np.empty(m, np.int32); st = np.empty(m, np.uint8)
        ov = np.empty(m, np.int32)
        self._check(self._lib.bdm_get_forces(self._h, sim, m, _dptr(F), _dptr(nnz), _dptr(st), _dptr(ov),
                                             C.byref(n)))
        k = n.value
        if overlaps:
            return F[:k], nnz[:k], st[:k].astype(bool), ov[:k]
        return F[:k], nnz[:k], st[:k].astype(bool)

    def storage_order(self, sim: int) -> np.ndarray:
        n = C.c_int64()
        rc = self._lib.bdm_get_storage_order(self._h, sim, 0, None, C.byref(n))
        self._check_size_query(rc, n)
        out = np.empty(max(n.value, 1), np.int64)
        self._check(self._lib.bdm_get_storage_order(self._h, sim, n.value, _dptr(out), C.byref(n)))
        return out[: n.value]

    def stats(self, sim: int) -> dict:
        s = BdmStats()
        self._check(self._lib.bdm_get_stats(self._h, sim, C.byref(s)))
        return dict(agents=s.agents, iterations=s.iterations, static_agents=s.static_agents,
                    moved_agents=s.moved_agents, origin_len=list(s.origin_len), dims=list(s.dims),
                    agent_updates=s.agent_updates)

    # -- diffusion slice (§4.5.2, Algorithms 6 and 7) ------------------------
    @staticmethod
    def _diffusion_grid(u, lo, h):
        """Grid descriptor for a concentration array of shape (nz, ny, nx)
        (numpy float64, C order, or a CUDA torch tensor); flags for it."""
        if hasattr(u, "data_ptr") and getattr(u, "is_cuda", False):
            if u.dim() != 3 or not u.is_contiguous() or str(u.dtype) != "torch.float64":
                raise ValueError("u must be a contiguous float64 CUDA tensor of shape (nz, ny, nx)")
            shape, ptr, flags = tuple(u.shape), C.c_void_p(u.data_ptr()), DEVICE_PTRS
        else:
            if not isinstance(u, np.ndarray) or u.dtype != np.float64 or not u.flags.c_contiguous or u.ndim != 3:
                raise ValueError("u must be a C-contiguous float64 array of shape (nz, ny, nx)")
            shape, ptr, flags = u.shape, _dptr(u), 0
        g = BdmDiffusionGrid((C.c_double * 3)(*[float(v) for v in lo]), (C.c_double * 3)(*[float(v) for v in h]),
                             (C.c_int64 * 3)(shape[2], shape[1], shape[0]))
        return g, ptr, flags

    def diffuse(self, u, lo, h, nu: float, mu: float, dt: float, steps: int = 1):
        """Eq 4.3, `steps` explicit steps of u in place."""
        g, ptr, flags = self._diffusion_grid(u, lo, h)
        self._check(self._lib.bdm_diffuse(self._h, C.byref(g), ptr, float(nu), float(mu), float(dt), int(steps),
                                          flags))
        return u

    def secrete(self, sim: int, u, lo, h, quantity: float):
        """Algorithm 6 for the agents of `sim`, into u in place."""
        g, ptr, flags = self._diffusion_grid(u, lo, h)
        self._check(self._lib.bdm_secrete(self._h, sim, C.byref(g), ptr, float(quantity), flags))
        return u

    def chemotaxis(self, sim: int, u, lo, h, weight: float):
        """Algorithm 7: moves the agents of `sim` up the gradient of u."""
        g, ptr, flags = self._diffusion_grid(u, lo, h)
        self._check(self._lib.bdm_chemotaxis(self._h, sim, C.byref(g), ptr, float(weight), flags))

    def set_agent_kinds(self, sim: int, kinds):
        """Agent kinds (0..3) by ID (bdm_set_agent_kinds)."""
        k = np.ascontiguousarray(kinds, dtype=np.uint8).reshape(-1)
        self._check(self._lib.bdm_set_agent_kinds(self._h, sim, k.shape[0], _dptr(k)))

    def set_substance(self, sim: int, u, lo, h, nu: float, mu: float, quantity: float, weight: float,
                      kind: int = 0):
        """A substance that the agents of `kind` secrete into, diffuse and
        follow in every iteration of bdm_step (bdm_set_substance); u is
        copied."""
        g, ptr, flags = self._diffusion_grid(u, lo, h)
        self._substance_shape = getattr(self, "_substance_shape", {})
        self._substance_shape[(sim, kind)] = tuple(u.shape)
        self._check(self._lib.bdm_set_substance(self._h, sim, int(kind), C.byref(g), ptr, float(nu), float(mu),
                                                float(quantity), float(weight), flags))

    def clear_substance(self, sim: int, kind: int = 0):
        self._check(self._lib.bdm_set_substance(self._h, sim, int(kind), None, None, 0.0, 0.0, 0.0, 0.0, 0))

    def get_substance(self, sim: int, kind: int = 0) -> np.ndarray:
        """The substance's concentrations, shape (nz, ny, nx) as set."""
        n = C.c_int64()
        rc = self._lib.bdm_get_substance(self._h, sim, int(kind), None, 0, C.byref(n), 0)
        self._check_size_query(rc, n)
        out = np.empty(getattr(self, "_substance_shape", {}).get((sim, kind), (n.value,)), np.float64)
        self._check(self._lib.bdm_get_substance(self._h, sim, int(kind), _dptr(out), out.size, C.byref(n), 0))
        return out

    # -- epidemiology (§4.6.3, Algorithms 3-5) -------------------------------
    def sir_step(self, sim: int, state, radius: float, p_infect: float, p_recover: float, speed: float,
                 length: float, seed: int = 0, t0: int = 0, steps: int = 1):
        """`steps` steps of the persons of `sim` from step t0; state (uint8
        by agent ID: 0 S, 1 I, 2 R; numpy, or a CUDA torch tensor) is
        updated in place."""
        prm = BdmSirParams(float(radius), float(p_infect), float(p_recover), float(speed), float(length), int(seed))
        if hasattr(state, "data_ptr") and getattr(state, "is_cuda", False):
            ptr, flags = C.c_void_p(state.data_ptr()), DEVICE_PTRS
        else:
            if not isinstance(state, np.ndarray) or state.dtype != np.uint8 or not state.flags.c_contiguous:
                raise ValueError("state must be a C-contiguous uint8 array")
            ptr, flags = _dptr(state), 0
        self._check(self._lib.bdm_sir_step(self._h, sim, C.byref(prm), ptr, int(t0), int(steps), flags))
        return state

    # -- tuning ------------------------------------------------------------
    def set_tuning(self, force_variant: int = 0, sort_interval: int = -1, sort_curve: int = 0,
                   box_scale_pct: int = 100, iter_batch: int = 1, test_flags: int = 0, grid_reuse: int = 0):
        t = BdmTuning(int(force_variant), int(sort_interval), int(sort_curve), int(box_scale_pct),
                      int(iter_batch), int(test_flags), int(grid_reuse))
        self._check(self._lib.bdm_set_tuning(self._h, C.byref(t)))

    def get_tuning(self) -> dict:
        t = BdmTuning()
        self._check(self._lib.bdm_get_tuning(self._h, C.byref(t)))
        return {k: getattr(t, k) for k in TUNING_FIELDS}

    def autotune(self, iterations: int = 5, knobs: int = TUNE_ALL) -> dict:
        """Time the candidates of the knobs selected in `knobs` (TUNE_* bits)
        and keep the fastest setting (bdm_autotune)."""
        t = BdmTuning()
        self._check(self._lib.bdm_autotune(self._h, int(iterations), int(knobs), C.byref(t)))
        return {k: getattr(t, k) for k in TUNING_FIELDS}

    def counters(self) -> dict:
        c = BdmCounters()
        self._check(self._lib.bdm_get_counters(self._h, C.byref(c)))
        return dict(graph_launches=c.graph_launches, kernels=c.kernels, graph_iterations=c.graph_iterations,
                    grid_builds=c.grid_builds)

    # -- profiling ---------------------------------------------------------
    def profile(self, enable: bool = True):
        self._check(self._lib.bdm_profile(self._h, 1 if enable else 0))

    def get_profile(self) -> dict:
        launches = (C.c_int64 * NUM_STAGES)(); ms = (C.c_double * NUM_STAGES)()
        names = (C.c_char_p * NUM_STAGES)()
        self._check(self._lib.bdm_get_profile(self._h, launches, ms, names))
        return {names[k].decode(): dict(launches=launches[k], ms=ms[k]) for k in range(NUM_STAGES)}
