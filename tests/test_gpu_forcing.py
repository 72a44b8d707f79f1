"""GPU tests of the Sec. 4.3 additions: Kupershtokh forcing against the
oracle and the closed-form uniform acceleration, mass rescaling, and the PI
controller on the mean streamwise momentum."""
import numpy as np
import pytest

from oracle import step as ost
from tests.oracle_cases import box_cfg, oracle_case
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _sim(cfg, prec, mode=0):
    from paper_2412_09051_gb300.sim import Sim
    return Sim(cfg, precision=prec, stream_mode=mode)


@pytest.mark.parametrize("name,over,prec,F", [("channel", dict(cells=(4, 6, 3)), "fp32", (0.05, 0.0, 0.01)),
                                              ("tgv2d", dict(cells=6), "fp64", (0.02, -0.01))])
@pytest.mark.parametrize("mode", [0, 1, 4])
def test_forced_steps_match_oracle(built_lib, name, over, prec, F, mode):
    cfg = get_config(name, **over)
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    par.force = np.array(F[:mesh.D])
    sim = _sim(cfg, prec, mode)
    sim.set_force(F)
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    tol = 1e-12 if prec == "fp64" else 1e-5
    for _ in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
    sim.step(3)
    fg, gg = sim.get_state()
    for a, b in ((fg, f), (gg, g)):
        s = np.maximum(np.abs(b).max(axis=1, keepdims=True), w[:, None])
        assert (np.abs(a - b) / s).max() < tol


@pytest.mark.parametrize("cells", [(32, 3, 2), (64, 3, 2)])
@pytest.mark.parametrize("mode,kernel", [(7, "k_step_rows_tmem"), (10, "k_step_rows_pairs")])
def test_forced_row_tiles_match_oracle(built_lib, cells, mode, kernel):
    """The row-tile kernels (rows of 64 and 128 nodes) with the body force:
    the forcing term enters in the relaxation pass of their collision."""
    cfg = get_config("channel", cells=cells)
    F = (0.05, 0.0, 0.01)
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    par.force = np.array(F)
    sim = _sim(cfg, "fp32", mode)
    assert sim.info.stream_mode == mode
    sim.set_force(F)
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    for _ in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
    sim.step(3)
    assert sim.step_kernel() == kernel
    fg, gg = sim.get_state()
    worst = 0.0
    for a, b in ((fg, f), (gg, g)):
        s = np.maximum(np.abs(b).max(axis=1, keepdims=True), w[:, None])
        worst = max(worst, float((np.abs(a - b) / s).max()))
    assert worst < 1e-5
    print(f"PARITY forced {kernel} {mesh.N}: populations {worst:.2e}")
    sim.close()


def test_uniform_acceleration(built_lib):
    """Closed form: u(t) = u0 + F t / rho for a uniform state in a periodic box."""
    F = np.array([0.02, 0.005])
    cfg = box_cfg(cells=(4, 4), L=(1.0, 1.0), dt=0.02)
    sim = _sim(cfg, "fp64")
    N = sim.N
    rho0, u0, T0 = 1.1, np.array([0.3, -0.2]), 0.9
    sim.init_state(np.full(N, rho0), np.tile(u0, (N, 1)), np.full(N, T0))
    sim.set_force(F)
    sim.step(9)
    r, u, T = sim.moments()
    assert np.abs(u - (u0 + 9 * F * cfg["dt"] / rho0)).max() < 1e-12
    assert np.abs(T - T0).max() < 1e-12 and np.abs(r - rho0).max() < 1e-12


def test_mass_rescaling(built_lib):
    cfg = get_config("channel", cells=(4, 6, 3))
    sim = _sim(cfg, "fp64")
    rho, u, T = initial_fields(cfg, sim.node_coords())
    sim.init_state(rho, u, T)
    sim.step(5)
    r0, u0, T0 = sim.moments()
    target = 1.02 * r0.sum()
    sim.rescale_mass(target)
    c, _ = sim.conservation()
    r1, u1, T1 = sim.moments()
    assert abs(c[0] - target) < 1e-12 * target
    assert np.abs(u1 - u0).max() < 1e-12 and np.abs(T1 - T0).max() < 1e-12


def test_pi_controller_spins_up_to_target(built_lib):
    """Sec. 4.3: the volume force is adjusted by a PI controller on the mean
    streamwise momentum.  From rest, the controlled channel reaches the
    target momentum (the uncontrolled one stays at rest) while mass
    rescaling every 10 steps keeps the total mass."""
    cfg = get_config("channel", cells=(4, 12, 3))
    free = _sim(cfg, "fp32")
    ctl = _sim(cfg, "fp32")
    N = free.N
    Tw = cfg["bcs"][0]["T"]
    for s in (free, ctl):
        s.init_state(np.ones(N), np.zeros((N, 3)), np.full(N, Tw))
    c0, _ = free.conservation()
    target = 0.05
    free.step(600)
    F = ctl.step_controlled(600, target, 0.0, kp=20.0, ki=100.0, control_every=5, rescale_every=10,
                            target_mass=c0[0])
    cf, _ = free.conservation()
    cc, _ = ctl.conservation()
    assert abs(cf[1] / N) < 1e-3 * target
    assert abs(cc[1] / N - target) < 0.1 * target
    assert np.isfinite(F).all()
    assert abs(cc[0] - c0[0]) < 1e-4 * c0[0]


def test_pi_controller_force_sequence_matches_host_law(built_lib):
    """The PI control law of Sec. 4.3 as read here, restated on the host in
    FP64 and replayed on the library's own FP64 momentum sums: every
    control_every steps e = target - mean(rho u_x), I += e control_every dt,
    F_x = F0 + kp e + ki I.  Stepping one control period per call, the force
    the library sets must equal the host's to 1e-12 at every update."""
    cfg = get_config("channel", cells=(4, 12, 3))
    sim = _sim(cfg, "fp32")
    N = sim.N
    Tw = cfg["bcs"][0]["T"]
    sim.init_state(np.ones(N), np.zeros((N, 3)), np.full(N, Tw))
    target, F0, kp, ki, every = 0.05, 1e-3, 20.0, 100.0, 5
    integral = 0.0
    forces = []
    for period in range(12):
        F = sim.step_controlled(every, target, F0, kp=kp, ki=ki, control_every=every, rescale_every=0,
                                target_mass=0.0)
        c, rc = sim.conservation(check=False)
        e = target - c[1] / N
        integral += e * every * cfg["dt"]
        Fh = F0 + kp * e + ki * integral
        assert abs(F[0] - Fh) <= 1e-12 * max(1.0, abs(Fh)), (period, F[0], Fh)
        assert F[1] == 0.0 and F[2] == 0.0
        forces.append(F[0])
    assert np.ptp(forces) > 1e-3                   # the force did change over the periods
    sim.close()
