"""CPU checks of the C ABI: the library builds, loads and exports every symbol
the header declares; calls without a GPU fail with a clean status."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sllbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sllbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_binding_symbols():
    from paper_2412_09051_gb300 import capi
    assert _declared() == capi.EXPORTED


def test_library_exports_every_declared_symbol(built_lib):
    for name in _declared():
        assert hasattr(built_lib, name), name


def test_struct_sizes_match_header():
    """The ctypes mirrors have the C layout (checked against offsets by hand)."""
    from paper_2412_09051_gb300 import capi
    assert ctypes.sizeof(capi.Bc) == 48
    assert capi.MeshDesc.bc.offset % 8 == 0
    assert ctypes.sizeof(capi.Params) == 6 * 8 + 5 * 4 + 4 + 8


def test_create_without_gpu_reports_arch(built_lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2412_09051_gb300.sim import Sim
    from paper_2412_09051_gb300.capi import SllbmError
    from workloads import get_config
    with pytest.raises(SllbmError) as e:
        Sim(get_config("tgv2d", cells=4))
    assert e.value.code == -3


def test_release_build_flags_and_null_context_arguments(built_lib):
    """sllbm_build_flags needs no context or GPU: 0 for the release build.
    Calls that take a context reject NULL with SLLBM_ERR_ARG before touching
    a device."""
    assert built_lib.sllbm_build_flags() == 0
    assert built_lib.sllbm_debug_wait_limit(None, 0) == -1
    code = ctypes.c_int32(7)
    assert built_lib.sllbm_device_status(None, ctypes.byref(code)) == -1
    assert built_lib.sllbm_mlp_path(None, 0) == -1
