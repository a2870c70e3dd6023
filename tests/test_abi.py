"""The C-ABI library builds, loads and exports every symbol that
include/bdm.h declares (no compute calls: CPU only)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    with open(os.path.join(ROOT, "include", "bdm.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bdm_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["bdm_create", "bdm_set_agents", "bdm_step", "bdm_get_agents", "bdm_neighbors",
                     "bdm_sync", "bdm_get_grid", "bdm_destroy", "bdm_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_2503_10796_gb300 import binding
    lib = binding.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in binding.SIGNATURES, name
    # the binding declares nothing that the header lacks
    assert set(binding.SIGNATURES) == set(declared_functions())
    assert isinstance(lib, ctypes.CDLL)


def test_params_struct_layouts_agree():
    """bdm_params (library) and the oracle's parameter struct are declared
    separately; both must keep the field order of the workload parameters."""
    from paper_2503_10796_gb300 import binding, workloads
    import oracle
    names_b = [f[0] for f in binding.BdmParams._fields_]
    names_o = [f[0] for f in oracle.OrcParams._fields_]
    assert names_b == names_o
    assert set(workloads.SimParams().as_dict()) <= set(names_b)
    import ctypes
    assert ctypes.sizeof(binding.BdmParams) == 8 * 8 + 4 * 4 + 8 + 8 + 2 * 8 + 2 * 4


def test_create_without_gpu_fails_loudly():
    """No CPU fallback: without a usable GPU, bdm_create reports an error."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2503_10796_gb300 import binding
    with pytest.raises(binding.BdmError):
        binding.Context(binding.make_params(), 16)
