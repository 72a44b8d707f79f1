"""Domain decomposition along x on the GPU: two parts as two library contexts
in one process (sllbm_get_x_layers / sllbm_set_x_layers move the halo layers
on the device side of each context), against the single-domain run and the
FP64 oracle."""
import numpy as np
import pytest

from oracle import step as ost
from tests.oracle_cases import oracle_case
from workloads import get_config, initial_fields

pytestmark = pytest.mark.gpu


def _scale_err(a, b, w):
    s = np.maximum(np.abs(b).max(axis=1, keepdims=True), np.asarray(w)[:, None])
    return float((np.abs(a - b) / s).max())


@pytest.mark.parametrize("name,cells,parts", [("channel", (64, 3, 3), 2), ("channel", (12, 3, 2), 3),
                                              ("learned", 16, 2)])
def test_slab_parts_match_single_domain(built_lib, name, cells, parts):
    from oracle.velocity_sets import velocity_set
    from paper_2412_09051_gb300.sim import Sim
    from paper_2412_09051_gb300.slab import exchange_in_process, local_config, local_node_index, plan_for_config
    cfg = get_config(name, cells=cells)
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    rho, u, T = initial_fields(cfg, mesh.X)
    vmax = float(np.sqrt((xi ** 2).sum(1)).max())
    plans = [plan_for_config(cfg, parts, k, vmax) for k in range(parts)]
    sims, idxs = [], []
    for pl in plans:
        idx = local_node_index(pl, mesh.N[:mesh.D])
        s = Sim(local_config(cfg, pl))
        s.init_state(rho[idx], u[idx], T[idx])
        sims.append(s)
        idxs.append(idx)
    whole = Sim(cfg)
    whole.init_state(rho, u, T)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    for _ in range(3):
        for s in sims:
            s.step(1)
        exchange_in_process(sims, plans)
        whole.step(1)
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
    fw, gw = whole.get_state()
    worst_o, worst_w = 0.0, 0.0
    for s, pl, idx in zip(sims, plans, idxs):
        a, b = pl.interior
        fl, gl = s.get_state()
        sel = idx.reshape(-1, pl.nodes_x)[:, a:b].ravel()
        fl = fl.reshape(len(w), -1, pl.nodes_x)[:, :, a:b].reshape(len(w), -1)
        gl = gl.reshape(len(w), -1, pl.nodes_x)[:, :, a:b].reshape(len(w), -1)
        worst_o = max(worst_o, _scale_err(fl, f[:, sel], w), _scale_err(gl, g[:, sel], w))
        worst_w = max(worst_w, _scale_err(fl, fw[:, sel], w), _scale_err(gl, gw[:, sel], w))
    assert worst_o < 1e-5 and worst_w < 1e-5, (worst_o, worst_w)
    print(f"PARITY slab {name} {mesh.N} in {parts} parts ({sims[0].step_kernel()}): "
          f"vs oracle {worst_o:.2e}, vs one context ({whole.step_kernel()}) {worst_w:.2e}")
    for s in sims + [whole]:
        s.close()


def test_x_layers_round_trip(built_lib):
    """get_x_layers / set_x_layers: host and device buffers, exact copies."""
    import torch
    from paper_2412_09051_gb300.sim import Sim
    cfg = get_config("channel", cells=(8, 3, 2))
    s = Sim(cfg)
    s.init_state(*initial_fields(cfg, s.node_coords()))
    s.step(1)
    raw = s.get_state_raw()                                         # [Q, N, 2]
    Nx = s.info.nodes[0]
    lay = s.get_x_layers(3, 5)
    ref = raw.reshape(s.Q, -1, Nx, 2)[:, :, 3:8]
    assert np.array_equal(lay, ref)
    dev = torch.zeros(lay.shape, dtype=torch.float32, device="cuda")
    s.get_x_layers(3, 5, dev)
    torch.cuda.synchronize()
    assert np.array_equal(dev.cpu().numpy(), ref)
    s.set_x_layers(0, 5, lay)                                       # layers 3..7 copied onto 0..4
    raw2 = s.get_state_raw().reshape(s.Q, -1, Nx, 2)
    assert np.array_equal(raw2[:, :, 0:5], ref) and np.array_equal(raw2[:, :, 5:], raw.reshape(s.Q, -1, Nx, 2)[:, :, 5:])
    s.close()
