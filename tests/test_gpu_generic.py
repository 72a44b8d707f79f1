"""GPU parity of the generic velocity-set kernels (generic.cu): D3Q125, the
product 5-point Gauss-Hermite rule (Sec. 3.2), and caller-supplied sets
through sllbm_create_desc, against the FP64 oracle, and a caller's copy of a
compiled set against that set's own kernels."""
import numpy as np
import pytest

from oracle import step as ost
from tests.oracle_cases import box_cfg, oracle_case
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _scale_err(a, b, w):
    s = np.maximum(np.abs(b).max(axis=1, keepdims=True), np.asarray(w)[:, None])
    return float((np.abs(a - b) / s).max())


def _d3q125(cfg):
    cfg = dict(cfg)
    cfg["velset"] = "D3Q125"
    return cfg


CASES = {
    # isothermal walls (bounce-back with the thermal correction), p = 2
    "channel_d3q125_fp64": (lambda: _d3q125(get_config("channel", cells=(3, 3, 2))), "fp64"),
    "channel_d3q125_fp32": (lambda: _d3q125(get_config("channel", cells=(3, 3, 2))), "fp32"),
    # equilibrium boundaries
    "mixing_d3q125_fp32": (lambda: _d3q125(get_config("mixing", cells=(3, 4, 2))), "fp32"),
    # periodic box of order 4 (the paper's order), Pr != 1, viscosity power law
    "box_d3q125_p4_fp64": (lambda: box_cfg(cells=(2, 2, 2), p=4, L=(1.0, 1.0, 1.0), dt=0.01, velset="D3Q125",
                                           mu=0.02, Pr=0.71, mu_exp=0.7), "fp64"),
    "box_d3q125_p3_fp32": (lambda: box_cfg(cells=(2, 2, 2), p=3, L=(1.0, 1.0, 1.0), dt=0.01, velset="D3Q125",
                                           mu=0.02, Pr=0.71), "fp32"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_d3q125_matches_oracle(built_lib, name):
    from paper_2412_09051_gb300.sim import Sim
    mk, prec = CASES[name]
    cfg = mk()
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision=prec)
    assert sim.Q == 125 and sim.info.stream_mode == 1
    xl, wl, ol = sim.velocity_set()
    assert np.abs(xl - xi).max() < 1e-15 and np.abs(wl - w).max() < 1e-15 and (ol == opp).all()
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    tol = 1e-12 if prec == "fp64" else 1e-5
    Tw = ost.isothermal_nodes(rec, par)
    worst = 0.0
    for k in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
        sim.step(1)
        assert sim.step_kernel() == "k_step_generic"
        fg, gg = sim.get_state()
        ef, eg = _scale_err(fg, f, w), _scale_err(gg, g, w)
        assert ef < tol and eg < tol, (k, ef, eg)
        worst = max(worst, ef, eg)
    r0, u0, T0 = ost.moments(f, g, xi, par.cv)
    r1, u1, T1 = sim.moments()
    em = max(np.abs(r1 - r0).max(), np.abs(T1 - T0).max(), np.abs(u1 - u0).max() / max(1.0, np.abs(u0).max()))
    assert em < tol
    # conservation sums (Sec. 3.1 moments summed over the nodes), both entry points
    D = mesh.D
    ref = np.concatenate([[r0.sum()], (r0[:, None] * u0).sum(0),
                          [float((r0 * (u0 ** 2).sum(1) + 2 * par.cv * r0 * T0).sum())]])
    import ctypes as C
    from paper_2412_09051_gb300 import capi
    static = np.zeros(D + 2)
    assert capi.lib().sllbm_conservation_static(sim.h, static.ctypes.data_as(C.c_void_p)) == 0
    for got in (sim.conservation()[0], static):
        assert np.abs(np.asarray(got) - ref).max() < tol * max(1.0, np.abs(ref).max()) * 10
    assert len(ref) == D + 2
    print(f"PARITY generic {name} {mesh.N}: populations {worst:.2e} moments {em:.2e}")
    sim.close()


def test_custom_copy_of_d3q45_equals_the_compiled_set(built_lib):
    """A caller's copy of D3Q45 (the oracle's abscissae and weights) runs the
    generic kernels; the compiled D3Q45 gather kernel gives the same FP64 step."""
    from oracle.velocity_sets import velocity_set
    from paper_2412_09051_gb300.sim import Sim
    base = get_config("channel", cells=(3, 3, 2))
    xi, w, _ = velocity_set("D3Q45")
    cust = dict(base, velset="CUSTOM", velset_xi=xi, velset_w=w)
    a, b = Sim(cust, precision="fp64"), Sim(base, precision="fp64", stream_mode=1)
    X = a.node_coords()
    rho, u, T = initial_fields(base, X)
    for s in (a, b):
        s.init_state(rho, u, T)
        s.step(4)
    assert a.step_kernel() == "k_step_generic" and b.step_kernel() == "k_step_gather"
    fa, ga = a.get_state()
    fb, gb = b.get_state()
    err = max(_scale_err(fa, fb, w), _scale_err(ga, gb, w))
    assert err < 1e-12, err
    print(f"PARITY custom D3Q45 vs compiled D3Q45, 4 channel steps (FP64): {err:.2e}")
    a.close()
    b.close()


def test_custom_d2q9_matches_oracle(built_lib):
    """The classic D2Q9 lattice given as a caller's set, on the Taylor-Green
    box (FP64), against the oracle with the same arrays."""
    from oracle.velocity_sets import velocity_set
    from paper_2412_09051_gb300.sim import Sim
    xi, w, _ = velocity_set("D2Q9")
    cfg = dict(get_config("tgv2d", cells=6), velset="CUSTOM", velset_xi=xi, velset_w=w)
    mesh, oxi, ow, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision="fp64")
    assert sim.Q == 9 and sim.step_kernel() in ("", "k_step_generic")
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, oxi, ow, par.cv)
    for _ in range(3):
        f, g = ost.step(mesh, rec, f, g, oxi, ow, par)
    sim.step(3)
    fg, gg = sim.get_state()
    err = max(_scale_err(fg, f, ow), _scale_err(gg, g, ow))
    assert err < 1e-12, err
    print(f"PARITY custom D2Q9 tgv2d: {err:.2e}")
    sim.close()
