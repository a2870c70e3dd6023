"""GB300 (sm_103a) mechanical-interaction step for spherical agents, after
the BioDynaMo thesis (arXiv 2503.10796): uniform-grid neighbor search,
Eq 4.1/4.2 sphere-sphere force, displacement with adherence threshold and
clamp, Morton re-sort, static-agent skip, growth and division.

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/bdm.h``); ``binding`` is its ctypes binding and ``workloads`` the
seeded input generators.  Submodules load lazily so that importing the
input generators needs no GPU.
"""

__all__ = ["binding", "workloads", "build"]


def __getattr__(name):
    import importlib
    if name in ("binding", "workloads", "build"):
        return importlib.import_module(f"{__name__}.{name}")
    if name in ("Context", "BdmError", "load_library", "make_params"):
        return getattr(importlib.import_module(f"{__name__}.binding"), name)
    raise AttributeError(name)
