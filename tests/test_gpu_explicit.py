"""GPU parity of the explicit mesh kind (SLLBM_MESH_EXPLICIT: the caller's
vertex coordinates per dimension) against the oracle, and against the
analytic channel on the channel's own vertices."""
import numpy as np
import pytest

from oracle import step as ost
from tests.oracle_cases import oracle_case
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _scale_err(a, b, w):
    s = np.maximum(np.abs(b).max(axis=1, keepdims=True), np.asarray(w)[:, None])
    return float((np.abs(a - b) / s).max())


def _explicit(base, vertices, bc_kinds=None):
    cfg = dict(base, mesh=dict(base["mesh"], kind=4, vertices=vertices))
    if bc_kinds is not None:
        cfg["bcs"] = [dict(base["bcs"][b], kind=bc_kinds[b]) for b in range(2)]
    return cfg


def test_explicit_on_channel_vertices_equals_the_channel(built_lib):
    """The channel (64-node rows) given as explicit vertex arrays: the same
    kernel and a bit-identical state after three steps."""
    from paper_2412_09051_gb300.sim import Sim
    base = get_config("channel", cells=(32, 3, 2))
    m = base["mesh"]
    a = Sim(base)
    X = a.node_coords()
    # the library's own vertices: the cell corners among its nodes (x fastest),
    # closed by L_d on the periodic dimensions as the channel builder does
    p, (C0, C1, C2), L = m["p"], m["cells"], m["length"]
    G = X.reshape(C2 * p, C1 * p + 1, C0 * p, 3)
    verts = [np.append(G[0, 0, ::p, 0], L[0] * C0 / C0), G[0, ::p, 0, 1], np.append(G[::p, 0, 0, 2], L[2] * C2 / C2)]
    cfg = _explicit(base, verts)
    b = Sim(cfg)
    assert np.array_equal(X, b.node_coords())
    for s in (a, b):
        s.init_state(*initial_fields(base, X))
        s.step(3)
    assert a.step_kernel() == b.step_kernel() == "k_step_rows_pairs"
    assert np.array_equal(a.get_state_raw(), b.get_state_raw())
    a.close()
    b.close()


def _rng_vertices(rng, C, L, start=0.0):
    """C cells of random widths (0.5 .. 1.5 of the mean) summing to L."""
    h = rng.uniform(0.5, 1.5, C)
    return start + np.concatenate([[0.0], np.cumsum(h / h.sum() * L)])


CASES = {
    # uniform periodic x, z, random wall-bounded y: every streaming mode applies
    "walls_random_y_fp32": ("fp32", lambda rng, c: [np.linspace(0, c["mesh"]["length"][0], 9),
                                                   _rng_vertices(rng, 5, 2.0), np.linspace(0, 1.0, 4)],
                            dict(cells=(8, 5, 3)), None),
    # random periodic x: the gather streaming
    "walls_random_x_fp64": ("fp64", lambda rng, c: [_rng_vertices(rng, 6, 4.0), _rng_vertices(rng, 4, 2.0),
                                                   np.linspace(0, 1.0, 3)],
                            dict(cells=(6, 4, 2)), None),
}


@pytest.mark.parametrize("name", list(CASES))
def test_explicit_mesh_matches_oracle(built_lib, name):
    from paper_2412_09051_gb300.sim import Sim
    prec, mkv, over, bck = CASES[name]
    rng = np.random.default_rng(31)
    base = get_config("channel", **over)
    cfg = _explicit(base, mkv(rng, base), bck)
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision=prec)
    assert np.abs(sim.node_coords() - mesh.X).max() < 1e-14
    gather = "random_x" in name
    assert (sim.info.stream_mode == 1) == gather
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    tol = 1e-12 if prec == "fp64" else 1e-5
    worst = 0.0
    for k in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
        sim.step(1)
        fg, gg = sim.get_state()
        ef, eg = _scale_err(fg, f, w), _scale_err(gg, g, w)
        assert ef < tol and eg < tol, (k, ef, eg)
        worst = max(worst, ef, eg)
    print(f"PARITY explicit {name} {mesh.N} ({sim.step_kernel()}): populations {worst:.2e}")
    sim.close()


def test_explicit_periodic_box_matches_oracle(built_lib):
    """A fully periodic 2D explicit mesh with random spacing in both
    dimensions (FP64, gather streaming)."""
    from paper_2412_09051_gb300.sim import Sim
    rng = np.random.default_rng(32)
    base = get_config("tgv2d", cells=6)
    cfg = _explicit(base, [_rng_vertices(rng, 6, base["mesh"]["length"][0]),
                           _rng_vertices(rng, 6, base["mesh"]["length"][1])])
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    sim = Sim(cfg, precision="fp64")
    assert sim.info.stream_mode == 1
    rho, u, T = initial_fields(cfg, mesh.X)
    sim.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    for _ in range(3):
        f, g = ost.step(mesh, rec, f, g, xi, w, par)
    sim.step(3)
    fg, gg = sim.get_state()
    err = max(_scale_err(fg, f, w), _scale_err(gg, g, w))
    assert err < 1e-12, err
    print(f"PARITY explicit periodic box {mesh.N}: {err:.2e}")
    sim.close()
