"""Bounded waits of the tensor-core and bulk-copy kernels.

A test limit (sllbm_debug_wait_limit: 2 SM cycles instead of about 2^31) makes
the mbarrier waits run out without any fault.  The kernels must record their
timeout bit in the status word, finish their own operations in flight (the
products of the tensor cores, the bulk copies) and return.  Once the default
limit is back, the context must step exactly as a fresh context does.
"""
import numpy as np
import pytest

from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _learned_cfg():
    cfg = get_config("learned", cells=8)
    cfg["init"] = dict(kind="isentropic_vortex", mach=0.6, seed=3)
    return cfg


def _tc_sim(cfg):
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    from tests.test_gpu_learned import _random_install
    s = Sim(cfg)
    _random_install(s, s.Q, seed=11, sigma=3e-2)
    s.mlp_path(capi.MLP_TENSOR)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    return s


def test_tensor_core_wait_timeout_is_reported_and_recoverable(built_lib):
    from paper_2412_09051_gb300 import capi
    cfg = _learned_cfg()
    s = _tc_sim(cfg)
    s.debug_wait_limit(1)
    s.step(1)
    assert s.step_kernel() == "k_step_tiled_smem_tc"
    assert s.device_status() & capi.DEV_TC_TIMEOUT
    s.debug_wait_limit(0)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    s.step(2)
    assert s.device_status() == 0
    ref = _tc_sim(cfg)
    ref.step(2)
    assert ref.device_status() == 0
    assert np.array_equal(s.get_state_raw(), ref.get_state_raw())
    s.close()
    ref.close()


@pytest.mark.parametrize("name,cells", [("channel", (16, 4, 3)), ("learned", 16)])   # 32-node rows
def test_bulk_copy_wait_timeout_is_reported_and_recoverable(built_lib, name, cells):
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config(name, cells=cells)
    s = Sim(cfg, stream_mode=capi.STREAM_ROW_COPY)
    X = s.node_coords()
    s.init_state(*initial_fields(cfg, X))
    s.debug_wait_limit(1)
    s.step(1)
    assert s.step_kernel() == "k_step_row_copy"
    assert s.device_status() & capi.DEV_COPY_TIMEOUT
    s.debug_wait_limit(0)
    s.init_state(*initial_fields(cfg, X))
    s.step(2)
    assert s.device_status() == 0
    ref = Sim(cfg, stream_mode=capi.STREAM_ROW_COPY)
    ref.init_state(*initial_fields(cfg, X))
    ref.step(2)
    assert np.array_equal(s.get_state_raw(), ref.get_state_raw())
    s.close()
    ref.close()


@pytest.mark.parametrize("name,cells,mode,kernel", [("channel", (32, 3, 3), 7, "k_step_rows_tmem"),
                                                    ("learned", 16, 7, "k_step_rows_tmem"),
                                                    ("channel", (32, 3, 2), 10, "k_step_rows_pairs"),
                                                    ("learned", 32, 10, "k_step_rows_pairs")])
def test_row_tile_wait_timeout_is_reported_and_recoverable(built_lib, name, cells, mode, kernel):
    """The tensor-memory row-tile kernels (SLLBM_STREAM_ROWS_TMEM and
    SLLBM_STREAM_ROWS_PAIRS): under the test limit their consumers also wait on a barrier that nothing completes,
    record the timeout, stop waiting and storing; the producers wait (with
    the default limit) for the copies they issued; the CTA frees its tensor
    memory and exits."""
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config(name, cells=cells)
    s = Sim(cfg, stream_mode=mode)
    assert s.info.stream_mode == mode
    X = s.node_coords()
    s.init_state(*initial_fields(cfg, X))
    s.debug_wait_limit(1)
    s.step(1)
    assert s.step_kernel() == kernel
    assert s.device_status() & capi.DEV_COPY_TIMEOUT
    s.debug_wait_limit(0)
    s.init_state(*initial_fields(cfg, X))
    s.step(2)
    assert s.device_status() == 0
    ref = Sim(cfg, stream_mode=mode)
    ref.init_state(*initial_fields(cfg, X))
    ref.step(2)
    assert np.array_equal(s.get_state_raw(), ref.get_state_raw())
    s.close()
    ref.close()


def test_wait_limit_arguments(built_lib):
    from paper_2412_09051_gb300.capi import SllbmError
    from paper_2412_09051_gb300.sim import Sim
    s = Sim(get_config("learned", cells=4))
    for bad in (-1, 32):
        with pytest.raises(SllbmError) as e:
            s.debug_wait_limit(bad)
        assert e.value.code == -1
    s.close()
