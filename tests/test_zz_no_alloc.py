"""GPU test of the allocation-free conservation entry point.

sllbm_conservation_static is for callers that must not allocate device memory
when they check conservation (their memory budget belongs to another
framework's pool, or a cudaFree would stall their time loop).  It must give
the same sums as sllbm_conservation, call after call, leave the device's free
memory unchanged, report an unstable state the same way, and refuse a mesh
beyond its fixed limit.  This file sorts last so that a stop-at-first-failure
run has executed every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu

ERR_ARG, ERR_UNSTABLE = -1, -6


def _static_call(sim):
    from paper_2412_09051_gb300 import capi
    out = np.zeros(sim.D + 2)
    rc = capi.lib().sllbm_conservation_static(sim.h, out.ctypes.data_as(C.c_void_p))
    return out, rc


def _static_sums(sim):
    from paper_2412_09051_gb300 import capi
    out, rc = _static_call(sim)
    capi.check(rc, sim.h)
    return out


@pytest.mark.parametrize("name,over,prec", [("tgv2d", dict(cells=16), "fp32"),
                                            ("channel", dict(cells=(8, 12, 6)), "fp32"),
                                            ("tgv2d", dict(cells=8), "fp64")])
def test_static_conservation_matches_context_scratch(built_lib, name, over, prec):
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config(name, **over)
    sim = Sim(cfg, precision=prec)
    rho, u, T = initial_fields(cfg, sim.node_coords())
    sim.init_state(rho, u, T)
    for call in range(2):                      # two calls in a row, the state changing between them
        ref, rc = sim.conservation()
        got = _static_sums(sim)
        assert rc == 0
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), (call, got, ref)
        sim.step(3)
    sim.close()


def test_static_conservation_allocates_nothing(built_lib):
    """After one warm-up call (which loads the kernels), further calls leave
    the device's free memory exactly where it was."""
    import torch
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=(8, 12, 6))
    sim = Sim(cfg)
    rho, u, T = initial_fields(cfg, sim.node_coords())
    sim.init_state(rho, u, T)
    _static_sums(sim)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(3):
        _static_sums(sim)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0, (free0, free1)
    sim.close()


def test_static_conservation_reports_unstable_state(built_lib):
    """A node with negative density: both entry points return
    SLLBM_ERR_UNSTABLE and still fill the same sums."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("tgv2d", cells=8)
    sim = Sim(cfg, precision="fp64")
    rho, u, T = initial_fields(cfg, sim.node_coords())
    sim.init_state(rho, u, T)
    f, g = sim.get_state()
    f[:, 5] *= -1.0                            # rho < 0 at node 5
    sim.set_state(f, g)
    ref, rc_ref = sim.conservation(check=False)
    got, rc = _static_call(sim)
    assert rc_ref == ERR_UNSTABLE and rc == ERR_UNSTABLE
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # a clean state afterwards: the flag is cleared at the start of each call
    sim.init_state(rho, u, T)
    _, rc = _static_call(sim)
    assert rc == 0
    sim.close()


def test_static_conservation_rejects_mesh_beyond_limit(built_lib):
    """2D limit: 8,387,584 nodes (one partial per 256 nodes in 1 MiB); a
    2898 x 2898-node box is refused with SLLBM_ERR_ARG and the limit named."""
    from paper_2412_09051_gb300 import capi
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("learned", cells=1449)      # time step scaled with the cell size
    sim = Sim(cfg, precision="fp32")
    assert sim.N == 2898 * 2898 > 8387584
    rho, u, T = initial_fields(cfg, sim.node_coords())
    sim.init_state(rho, u, T)
    _, rc = _static_call(sim)
    assert rc == ERR_ARG
    msg = capi.lib().sllbm_last_error(sim.h).decode()
    assert "8387584" in msg, msg
    sim.close()
