"""GPU test of the allocation-free conservation entry point.

sllbm_conservation_static is for callers that must not allocate device memory
when they check conservation (their memory budget belongs to another
framework's pool, or a cudaFree would stall their time loop).  It must give
the same sums as sllbm_conservation, call after call.  This file sorts last so
that a stop-at-first-failure run has executed every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _static_sums(sim):
    from paper_2412_09051_gb300 import capi
    out = np.zeros(sim.D + 2)
    capi.check(capi.lib().sllbm_conservation_static(sim.h, out.ctypes.data_as(C.c_void_p)), sim.h)
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
