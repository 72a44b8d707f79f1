"""Domain decomposition along x (paper_2412_09051_gb300/slab.py) on the CPU.

The slab driver is engine-agnostic; here each part's engine is the FP64
oracle on the part's periodic slab-plus-halo mesh, and the parts are two gloo
ranks (world size 2) exchanging halo layers through torch.distributed after
every step.  The interior of every part must equal the single-domain oracle
run to FP64 rounding.  Plan arithmetic (partition, halo width, index maps)
is checked directly.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from oracle import step as ost
from tests.oracle_cases import box_cfg, oracle_case
from workloads import get_config, initial_fields


class OracleEngine:
    """A part stepped by the oracle: the engine interface of the slab driver
    (step, get_x_layers, set_x_layers) on full FP64 populations, layers as
    [Q, rows, nx, 2] (f, g)."""

    def __init__(self, cfg, rho, u, T):
        self.mesh, self.xi, self.w, self.opp, self.par, self.rec = oracle_case(cfg)
        self.f, self.g = ost.init_equilibrium(rho, u, T, self.xi, self.w, self.par.cv)
        self.Tw = ost.isothermal_nodes(self.rec, self.par)
        self.Nx = self.mesh.N[0]

    def _grid(self, a):
        return a.reshape(a.shape[0], -1, self.Nx)          # [Q, rows, Nx]

    def step(self, n):
        for _ in range(n):
            self.f, self.g = ost.step(self.mesh, self.rec, self.f, self.g, self.xi, self.w, self.par, Tw=self.Tw)

    def get_x_layers(self, x0, nx):
        return np.stack([self._grid(self.f)[:, :, x0:x0 + nx], self._grid(self.g)[:, :, x0:x0 + nx]], axis=-1).copy()

    def set_x_layers(self, x0, nx, buf):
        fg, gg = self._grid(self.f), self._grid(self.g)
        fg[:, :, x0:x0 + nx] = buf[..., 0]
        gg[:, :, x0:x0 + nx] = buf[..., 1]


CASES = {
    "box_d2q19": lambda: box_cfg(cells=(8, 4), p=2, L=(2 * np.pi, np.pi), dt=0.02, mu=0.02),
    "channel_d3q45": lambda: get_config("channel", cells=(6, 3, 2)),
}
STEPS = 3


def _max_speed(cfg):
    from oracle.velocity_sets import velocity_set
    xi, _, _ = velocity_set(cfg["velset"])
    return float(np.sqrt((xi ** 2).sum(1)).max())


def _global_fields(cfg):
    from oracle.mesh import Mesh
    m = cfg["mesh"]
    mesh = Mesh(m["kind"], m["p"], m["cells"], m["length"], m.get("stretch", 1.0), m.get("central", 0))
    return mesh, initial_fields(cfg, mesh.X)


def _part_engine(cfg, plan):
    from paper_2412_09051_gb300.slab import local_config, local_node_index
    mesh, (rho, u, T) = _global_fields(cfg)
    idx = local_node_index(plan, mesh.N[:mesh.D])
    return OracleEngine(local_config(cfg, plan), rho[idx], u[idx], T[idx]), idx


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, name, out):
    import torch.distributed as dist
    from paper_2412_09051_gb300.slab import TorchComm, plan_for_config, step_decomposed
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    cfg = CASES[name]()
    plan = plan_for_config(cfg, 2, rank, _max_speed(cfg))
    eng, idx = _part_engine(cfg, plan)
    step_decomposed(eng, plan, TorchComm(dist), STEPS)
    a, b = plan.interior
    out.put((rank, idx.reshape(-1, plan.nodes_x)[:, a:b].ravel(),
             eng._grid(eng.f)[:, :, a:b].reshape(len(eng.w), -1), eng._grid(eng.g)[:, :, a:b].reshape(len(eng.w), -1)))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("name", list(CASES))
def test_two_gloo_parts_match_single_domain(name):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, name, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict((r[0], r[1:]) for r in (q.get(timeout=600) for _ in range(2)))
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    cfg = CASES[name]()
    mesh, xi, w, opp, par, rec = oracle_case(cfg)
    _, (rho, u, T) = _global_fields(cfg)
    f, g = ost.init_equilibrium(rho, u, T, xi, w, par.cv)
    Tw = ost.isothermal_nodes(rec, par)
    for _ in range(STEPS):
        f, g = ost.step(mesh, rec, f, g, xi, w, par, Tw=Tw)
    covered = np.concatenate([res[0][0], res[1][0]])
    assert np.array_equal(np.sort(covered), np.arange(mesh.n_nodes))        # interiors tile the mesh
    worst = 0.0
    for r in (0, 1):
        idx, fp, gp = res[r]
        scale = np.abs(f).max(1, keepdims=True)
        worst = max(worst, float((np.abs(fp - f[:, idx]) / scale).max()), float((np.abs(gp - g[:, idx]) / scale).max()))
    assert worst < 1e-12, worst


def test_plan_arithmetic():
    from paper_2412_09051_gb300.slab import halo_cells, local_config, local_node_index, plan_slabs
    assert halo_cells(3.0, 0.01, 0.1) == 1 and halo_cells(3.0, 0.05, 0.1) == 2 and halo_cells(1.0, 0.1, 0.1) == 1
    plans = [plan_slabs(10, 3, k, 2, 1) for k in range(3)]
    assert [(pl.c0, pl.c1) for pl in plans] == [(0, 4), (4, 7), (7, 10)]
    pl = plans[0]
    assert pl.local_cells == 6 and pl.nodes_x == 12 and pl.interior == (2, 10)
    assert pl.global_x(0) == 18 and pl.global_x(2) == 0 and pl.global_x(11) == 9      # periodic images
    idx = local_node_index(pl, (20, 3))
    assert idx.shape == (36,) and idx[0] == 18 and idx[12] == 20 + 18
    cfg = get_config("channel", cells=(10, 3, 2))
    lc = local_config(cfg, pl)
    assert lc["mesh"]["cells"] == (6, 3, 2)
    assert abs(lc["mesh"]["length"][0] - 6 * cfg["mesh"]["length"][0] / 10) < 1e-15
    with pytest.raises(ValueError):
        plan_slabs(3, 3, 0, 2, 2)
