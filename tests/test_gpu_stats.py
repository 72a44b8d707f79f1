"""GPU tests of the flow statistics (plane Reynolds / Favre averages, Reynolds
stresses, mixing-layer thicknesses, pressure coefficient) against the oracle's
definitions (oracle/stats.py): on the GPU's own moments the two must agree to
FP64 rounding; against the oracle's independent initial fields to the FP32
storage of the state."""
import numpy as np
import pytest

from oracle import stats
from oracle.mesh import Mesh
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _mesh(cfg):
    m = cfg["mesh"]
    return Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0),
                m.get("thickness", 0.12))


def _naca_small():
    cfg = get_config("naca", cells=(16, 6))
    cfg["mesh"] = dict(cfg["mesh"], stretch=1.3)
    cfg["dt"] = 2e-3
    return cfg


def _close(a, b, rel):
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= rel * max(1.0, np.abs(np.asarray(b)).max())


@pytest.mark.parametrize("name,cells", [("mixing", (3, 8, 2)), ("channel", (4, 6, 3)), ("mixing", None)])
def test_plane_profiles_match_oracle(built_lib, name, cells):
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config(name, cells=cells) if cells else get_config(name)
    mesh = _mesh(cfg)
    s = Sim(cfg)
    rho, u, T = initial_fields(cfg, s.node_coords())
    s.init_state(rho, u, T)
    for steps in (0, 3):
        s.step(steps)
        g = s.plane_profiles()
        ref = stats.plane_profiles(mesh, *s.moments())          # same moments: FP64 rounding
        for k in ("y", "rho", "u", "u_favre", "T", "p", "R"):
            assert _close(g[k], ref[k], 1e-12), (k, steps)
        if steps == 0:                                          # the oracle's own fields: FP32 storage
            ref0 = stats.plane_profiles(mesh, rho, u, T)
            for k in ("rho", "u", "u_favre", "T", "p"):
                assert _close(g[k], ref0[k], 2e-6), k
            assert np.abs(g["R"] - ref0["R"]).max() < 2e-6
    if name == "mixing":
        du = cfg["init"]["du"]
        th, om = s.mixing_thickness(du, 1.0)
        th_ref, om_ref = stats.mixing_thickness(mesh, stats.plane_profiles(mesh, *s.moments()), du, 1.0)
        # 1e-10: away from the layer the integrand (du/2 - u~)(du/2 + u~)
        # cancels, amplifying the plane means' summation-order differences
        assert abs(th - th_ref) < 1e-10 * th_ref and abs(om - om_ref) < 1e-12 * om_ref
    s.close()


def test_time_averaged_profiles_match_oracle(built_lib):
    """Running sums over three states of the channel (every second step):
    the time-and-plane averages against the oracle over the same states."""
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=(4, 6, 3))
    mesh = _mesh(cfg)
    s = Sim(cfg)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    s.stats_reset()
    states = []
    for k in range(3):
        s.stats_accumulate()
        states.append(s.moments())
        s.step(2)
    g = s.plane_profiles_mean()
    assert g["samples"] == 3
    ref = stats.plane_profiles_over_states(mesh, states)
    for k in ("y", "rho", "u", "u_favre", "T", "p", "R"):
        assert _close(g[k], ref[k], 1e-12), k
    s.stats_reset()
    from paper_2412_09051_gb300.capi import SllbmError
    with pytest.raises(SllbmError):
        s.plane_profiles_mean()
    s.close()


@pytest.mark.parametrize("side", [0, 1])
def test_pressure_coefficient_matches_oracle(built_lib, side):
    from paper_2412_09051_gb300.sim import Sim
    cfg = _naca_small()
    mesh = _mesh(cfg)
    s = Sim(cfg)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    s.step(2)
    U = cfg["init"]["U"]
    mach = U / np.sqrt(cfg["gamma"] * 1.0)
    x, cp = s.plane_cp(side, 1.0, mach)
    n = stats.plane_nodes(mesh, side)
    assert np.abs(x - mesh.X[n]).max() < 1e-13 * np.abs(mesh.X).max()
    r, _, T = s.moments()
    ref = stats.pressure_coefficient(r[n], T[n], 1.0, mach, cfg["gamma"])
    assert _close(cp, ref, 1e-13)
    s.close()


def test_plane_statistics_need_an_axis_aligned_mesh(built_lib):
    from paper_2412_09051_gb300.capi import SllbmError
    from paper_2412_09051_gb300.sim import Sim
    cfg = _naca_small()
    s = Sim(cfg)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    with pytest.raises(SllbmError):
        s.plane_profiles()
    with pytest.raises(SllbmError):
        s.mixing_thickness(1.0)
    s.close()
