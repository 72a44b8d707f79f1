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


def _custom_cfg(xi, w):
    from workloads import get_config
    cfg = get_config("tgv2d", cells=4)
    cfg["velset"] = "CUSTOM"
    cfg["velset_xi"] = xi
    cfg["velset_w"] = w
    return cfg


def test_custom_velocity_sets_are_checked_before_any_device_work(built_lib):
    """sllbm_create_desc copies and checks a caller's set (Sec. 3.2) before it
    queries a device: a set that is not symmetric, does not reproduce the
    weight function's moments to second order, has a non-positive weight or
    too many velocities fails with SLLBM_ERR_ARG and a message naming the
    check; a valid set passes them (and then, without a GPU, stops at the
    device query with SLLBM_ERR_ARCH)."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2412_09051_gb300.capi import SllbmError
    from paper_2412_09051_gb300.sim import Sim
    from oracle.velocity_sets import velocity_set
    xi, w, _ = velocity_set("D2Q9")
    cases = [
        (xi[:8], w[:8] / w[:8].sum(), "symmetric"),                          # drops (s, -s): no opposite left
        (xi * 1.1, w, "moments"),                                             # second moment 1.21
        (xi, np.where(np.arange(9) == 0, -w, w), "positive"),
        (np.zeros((129, 2)), np.full(129, 1 / 129), "Q <= 128"),
    ]
    for bad_xi, bad_w, word in cases:
        with pytest.raises(SllbmError) as e:
            Sim(_custom_cfg(bad_xi, bad_w))
        assert e.value.code == -1, (word, e.value)
        assert word in str(e.value), (word, str(e.value))
    with pytest.raises(SllbmError) as e:
        Sim(_custom_cfg(xi, w))
    assert e.value.code == -3


def test_custom_kind_needs_the_descriptor(built_lib):
    """sllbm_create with the custom kind (no arrays to read) is an argument error."""
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import mesh_desc, params
    from workloads import get_config
    cfg = get_config("tgv2d", cells=4)
    h = ctypes.c_void_p()
    d, p = mesh_desc(cfg), params(cfg)
    assert built_lib.sllbm_create(ctypes.byref(d), capi.VELSET["CUSTOM"], ctypes.byref(p), ctypes.byref(h)) == -1
    assert b"sllbm_create_desc" in built_lib.sllbm_last_error(None)


def test_set_allocator_arguments(built_lib):
    """sllbm_set_allocator needs both functions or neither (no device work)."""
    from paper_2412_09051_gb300 import capi
    alloc = capi.TorchAllocator()
    assert built_lib.sllbm_set_allocator(alloc._alloc, capi.FREE_FN(), None) == -1
    assert b"both functions" in built_lib.sllbm_last_error(None)
    assert built_lib.sllbm_set_allocator(capi.ALLOC_FN(), alloc._free, None) == -1
    assert built_lib.sllbm_set_allocator(capi.ALLOC_FN(), capi.FREE_FN(), None) == 0


def test_explicit_mesh_descriptors_are_checked_before_device_work(built_lib):
    """SLLBM_MESH_EXPLICIT: vertex arrays that are missing, not strictly
    increasing, or (on a periodic dimension) not starting at 0, and a y axis
    periodic at one end only, fail with SLLBM_ERR_ARG before the device query;
    a valid descriptor reaches it (SLLBM_ERR_ARCH without a GPU)."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2412_09051_gb300.capi import SllbmError
    from paper_2412_09051_gb300.sim import Sim
    from workloads import get_config

    def cfg(vx, vy, vz, bc_kinds=(3, 3)):
        c = get_config("channel", cells=(4, 3, 2))
        c = dict(c, mesh=dict(c["mesh"], kind=4, vertices=[vx, vy, vz]))
        c["bcs"] = [dict(c["bcs"][b], kind=bc_kinds[b]) for b in range(2)]
        return c

    vx, vy, vz = np.linspace(0, 4, 5), np.array([0.0, 0.2, 1.0, 2.0]), np.linspace(0, 1, 3)
    bad = [
        (cfg(vx, vy[::-1], vz), "strictly increasing"),
        (cfg(vx + 1.0, vy, vz), "starts at 0"),
        (cfg(vx, vy, vz, bc_kinds=(0, 3)), "at both ends"),
    ]
    for c, word in bad:
        with pytest.raises(SllbmError) as e:
            Sim(c)
        assert e.value.code == -1 and word in str(e.value), (word, str(e.value))
    with pytest.raises(SllbmError) as e:
        Sim(cfg(vx, vy, vz))
    assert e.value.code == -3
