"""GPU parity at the full benchmark sizes, on sampled arrival nodes: one step
from the seeded initial state, each sampled node computed by the oracle."""
import numpy as np
import pytest

from oracle import step as ost
from oracle.departure import trace
from oracle.mesh import Mesh
from oracle.velocity_sets import velocity_set
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,over", [("channel", {}), ("mixing", {}), ("naca", {}), ("tgv2d", {}),
                                       # the paper's order p = 4 at the channel's node count (order-4 row tiles)
                                       ("channel", {"cells": (32, 24, 24), "p": 4})])
def test_fullsize_sampled_step(built_lib, name, over):
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config(name, **over)
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0),
                m.get("thickness", 0.12))
    xi, w, opp = velocity_set(cfg["velset"])
    par = ost.Params(cfg["dt"], cfg["gamma"], cfg["Pr"], cfg["mu_ref"], cfg["T_ref"], cfg["mu_exp"], cfg["bcs"])
    rho, u, T = initial_fields(cfg, mesh.X)
    rng = np.random.default_rng(11)
    nodes = np.unique(np.concatenate([rng.integers(0, mesh.n_nodes, 40),
                                      np.arange(min(40, mesh.n_nodes)),                  # low-y / wall row
                                      mesh.n_nodes - 1 - np.arange(min(40, mesh.n_nodes))]))
    rec = trace(mesh, xi, opp, cfg["dt"], cfg["bcs"], nodes=nodes)
    f1, g1 = ost.step_sample_from_fields(mesh, rec, rho, u, T, xi, w, par)
    sim = Sim(cfg)
    if over.get("p") == 4:
        assert sim.info.stream_mode == 10             # the order-4 two-nodes-per-thread row tiles, as bench.py runs it
    assert np.abs(sim.node_coords() - mesh.X).max() < 1e-12 * np.abs(mesh.X).max()
    sim.init_state(rho, u, T)
    sim.step(1)
    fg, gg = sim.get_state()
    tol = 1e-12 if cfg["precision"] == "fp64" else 1e-5
    worst = 0.0
    for a, b in ((fg[:, nodes], f1), (gg[:, nodes], g1)):
        s = np.maximum(np.abs(b).max(axis=1, keepdims=True), w[:, None])
        e = float((np.abs(a - b) / s).max())
        assert e < tol
        worst = max(worst, e)
    print(f"PARITY fullsize {cfg['name']}: {len(nodes)} sampled nodes, populations {worst:.2e}")
    sim.close()
