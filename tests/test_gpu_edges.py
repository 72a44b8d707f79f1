"""GPU edge cases: no-op steps, the degenerate states the method has (rest,
uniform flow), the smallest meshes against the oracle, and the documented
error codes for invalid inputs."""
import numpy as np
import pytest

from oracle import step as ost
from tests.oracle_cases import box_cfg, oracle_case

pytestmark = pytest.mark.gpu


def _sim(cfg, prec="fp32", mode=0):
    from paper_2412_09051_gb300.sim import Sim
    return Sim(cfg, precision=prec, stream_mode=mode)


def _fields(sim, rho, u, T):
    N, D = sim.N, sim.D
    return np.full(N, rho), np.tile(np.asarray(u[:D], dtype=float), (N, 1)), np.full(N, T)


def test_step_zero_is_a_no_op(built_lib):
    from workloads import get_config, initial_fields
    cfg = get_config("channel", cells=(4, 6, 3))
    s = _sim(cfg)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    a = s.get_state_raw()
    s.step(0)
    assert np.array_equal(s.get_state_raw(), a)
    s.close()


@pytest.mark.parametrize("velset,cells", [("D2Q19", (8, 8)), ("D3Q45", (4, 4, 4))])
@pytest.mark.parametrize("mode", [0, 1, 3, 4, 5])
def test_rest_state_stays_exactly_at_rest(built_lib, velset, cells, mode):
    """rho = 1, u = 0, T = 1 in a periodic box: every stored deviation is 0 and
    every step keeps it exactly 0 (streaming of zeros, zero moments, zero
    equilibrium deviation, zero relaxation increment), in every streaming mode."""
    cfg = box_cfg(cells=cells, p=2, L=(1.0,) * len(cells), dt=0.01, velset=velset)
    s = _sim(cfg, "fp32", mode)
    s.init_state(*_fields(s, 1.0, (0.0, 0.0, 0.0), 1.0))
    assert not np.any(s.get_state_raw())
    s.step(5)
    assert not np.any(s.get_state_raw())
    s.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("fp32", 2e-6)])
def test_uniform_flow_is_invariant(built_lib, prec, tol):
    """A uniform state in a periodic box is an equilibrium that streaming
    reproduces (the Lagrange weights sum to one): it stays uniform."""
    cfg = box_cfg(cells=(6, 5), p=2, L=(1.0, 0.8), dt=0.004, mu=0.01, Pr=0.71, mu_exp=0.7)
    s = _sim(cfg, prec)
    rho0, u0, T0 = 1.1, (0.3, -0.2, 0.0), 0.9
    s.init_state(*_fields(s, rho0, u0, T0))
    s.step(10)
    r, u, T = s.moments()
    assert np.abs(r - rho0).max() < tol and np.abs(T - T0).max() < tol
    assert np.abs(u - np.asarray(u0[:2])).max() < tol
    s.close()


@pytest.mark.parametrize("velset,cells", [("D2Q19", (1, 1)), ("D2Q19", (2, 1)), ("D3Q45", (1, 1, 1))])
def test_smallest_meshes_match_oracle(built_lib, velset, cells):
    """One cell per dimension (p = 2: two nodes per periodic dimension, so the
    departure points wrap onto the same cell): three FP64 steps against the
    oracle to 1e-12."""
    from workloads import initial_fields
    cfg = box_cfg(cells=cells, p=2, L=(1.0,) * len(cells), dt=0.01, velset=velset)
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    s = _sim(cfg, "fp64")
    rho, u, T = initial_fields(cfg, mesh.X)
    s.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    for _ in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par)
    s.step(3)
    fg, gg = s.get_state()
    sc = np.maximum(np.abs(f).max(axis=1, keepdims=True), w[:, None])
    assert (np.abs(fg - f) / sc).max() < 1e-12 and (np.abs(gg - g) / sc).max() < 1e-12
    s.close()


def test_invalid_state_and_parameters_are_reported(built_lib):
    from paper_2412_09051_gb300.capi import SllbmError
    cfg = box_cfg(cells=(4, 4), p=2)
    s = _sim(cfg)
    rho, u, T = _fields(s, 1.0, (0.1, 0.0, 0.0), 1.0)
    rho[3] = -0.5                                  # negative density (exactly 0 is not representable:
                                                   # rho = 1 + sum of FP32 deviations)
    s.init_state(rho, u, T)
    _, rc = s.conservation(check=False)
    assert rc == -6                                # SLLBM_ERR_UNSTABLE
    rho[3] = 1.0
    T[5] = np.nan                                  # non-finite state
    s.init_state(rho, u, T)
    _, rc = s.conservation(check=False)
    assert rc == -6
    s.close()
    bad = dict(cfg, mu_ref=0.0)                    # viscosity must be positive
    with pytest.raises(SllbmError) as e:
        _sim(bad)
    assert e.value.code == -1
