"""Domain decomposition of the step along the periodic x axis (slabs with halos).

The paper's runs are multi-node (Sec. 4; 3 to 32 nodes) but it does not describe
its decomposition.  Here the mesh is cut along its periodic x axis into
contiguous slabs of cells, one per part (one GPU each).  A part steps its slab
plus `halo` cells on each side as a periodic domain of its own, with the
unchanged single-GPU kernels: a departure point of an interior node lies at
most `halo` cells away, so interior nodes read only the part's own layers
(halo nodes are computed too, and are wrong).  After every step the halo node
layers are replaced by the neighbours' edge layers of the interior: one
point-to-point exchange per step, in ring order (the part to the left takes
my first interior layers, the part to the right my last ones).

The engine is any object with step(n), get_x_layers(x0, nx) and
set_x_layers(x0, nx, buf) (sim.Sim is one, through the C ABI); the
communicator moves one buffer to a neighbour and receives one (TorchComm over
torch.distributed: gloo on host buffers, NCCL on device buffers), and
exchange_in_process() serves parts that live in one process.
"""
import math
from dataclasses import dataclass


def halo_cells(max_speed, dt, cell_width):
    """Halo cells per side: a departure point lies within max|zeta| dt of its
    node, so its cell is at most ceil(max|zeta| dt / cell width) cells away;
    at least one cell."""
    return max(1, int(math.ceil(max_speed * dt / cell_width - 1e-12)))


@dataclass(frozen=True)
class SlabPlan:
    """Part `part` of `parts` of a periodic x axis of `cells_x` cells of order p."""
    cells_x: int
    parts: int
    part: int
    p: int
    halo: int
    c0: int          # first global cell of the part's interior
    c1: int          # one past its last

    @property
    def interior_cells(self):
        return self.c1 - self.c0

    @property
    def local_cells(self):
        return self.interior_cells + 2 * self.halo

    @property
    def nodes_x(self):
        return self.local_cells * self.p

    @property
    def halo_nodes(self):
        return self.halo * self.p

    @property
    def interior(self):
        """Local node range [a, b) of the interior along x."""
        return self.halo_nodes, self.halo_nodes + self.interior_cells * self.p

    def global_x(self, local_x):
        """Global node index along x of a local node index (periodic)."""
        return ((self.c0 - self.halo) * self.p + local_x) % (self.cells_x * self.p)


def plan_slabs(cells_x, parts, part, p, halo):
    """Contiguous slabs of cells_x // parts cells (the first cells_x % parts
    parts one more); each interior must hold at least `halo` cells, so that a
    halo is filled by the nearest neighbour alone."""
    base, extra = divmod(cells_x, parts)
    c0 = part * base + min(part, extra)
    c1 = c0 + base + (1 if part < extra else 0)
    if c1 - c0 < halo:
        raise ValueError(f"{cells_x} cells in {parts} parts leave fewer than {halo} halo cells per part")
    return SlabPlan(cells_x, parts, part, p, halo, c0, c1)


def plan_for_config(cfg, parts, part, max_speed):
    """The plan of a workload config (periodic x axis) for `parts` parts."""
    m = cfg["mesh"]
    width = m["length"][0] / m["cells"][0]
    return plan_slabs(m["cells"][0], parts, part, m["p"], halo_cells(max_speed, cfg["dt"], width))


def local_config(cfg, plan):
    """The config of the part's periodic domain: its local cells along x, the
    same cell width, everything else unchanged."""
    m = dict(cfg["mesh"])
    width = m["length"][0] / m["cells"][0]
    cells = list(m["cells"])
    length = list(m["length"])
    cells[0] = plan.local_cells
    length[0] = plan.local_cells * width
    m["cells"] = tuple(cells)
    m["length"] = tuple(length)
    out = dict(cfg)
    out["mesh"] = m
    out["name"] = f"{cfg['name']}_part{plan.part}of{plan.parts}"
    return out


def local_node_index(plan, nodes):
    """Global node indices of the part's local nodes (x fastest, then y, then
    z), for nodes = (global Nx, Ny[, Nz])."""
    import numpy as np
    gx = np.array([plan.global_x(k) for k in range(plan.nodes_x)])
    rest = 1
    for n in nodes[1:]:
        rest *= n
    return (gx[None, :] + nodes[0] * np.arange(rest)[:, None]).ravel()


class TorchComm:
    """Point-to-point moves over torch.distributed (the initialised default
    group): `shift` sends a buffer to rank dst and receives one from rank src."""

    def __init__(self, dist):
        self.dist = dist

    def shift(self, buf, dst, src, tag):
        import numpy as np
        import torch
        host = isinstance(buf, np.ndarray)
        t = torch.from_numpy(np.ascontiguousarray(buf)) if host else buf.contiguous()
        r = torch.empty_like(t)
        reqs = [self.dist.isend(t, dst, tag=tag), self.dist.irecv(r, src, tag=tag)]
        for q in reqs:
            q.wait()
        return r.numpy() if host else r


def exchange_halos(engine, plan, comm):
    """Refresh this part's halo layers from its neighbours (all parts call it
    together).  Two phases, each a shift around the ring: the first moves
    every part's last interior layers to the right neighbour's left halo, the
    second every part's first interior layers to the left neighbour's right halo."""
    hn, nx = plan.halo_nodes, plan.nodes_x
    a, b = plan.interior
    right = (plan.part + 1) % plan.parts
    left = (plan.part - 1) % plan.parts
    to_right = engine.get_x_layers(b - hn, hn)
    to_left = engine.get_x_layers(a, hn)
    if plan.parts == 1:
        from_left, from_right = to_right, to_left
    else:
        from_left = comm.shift(to_right, right, left, tag=1)
        from_right = comm.shift(to_left, left, right, tag=2)
    engine.set_x_layers(0, hn, from_left)
    engine.set_x_layers(nx - hn, hn, from_right)


def exchange_in_process(engines, plans):
    """The same exchange for all parts held by one process."""
    outs = []
    for e, pl in zip(engines, plans):
        a, b = pl.interior
        outs.append((e.get_x_layers(b - pl.halo_nodes, pl.halo_nodes), e.get_x_layers(a, pl.halo_nodes)))
    n = len(engines)
    for k, (e, pl) in enumerate(zip(engines, plans)):
        from_left = outs[(k - 1) % n][0]
        from_right = outs[(k + 1) % n][1]
        e.set_x_layers(0, pl.halo_nodes, from_left)
        e.set_x_layers(pl.nodes_x - pl.halo_nodes, pl.halo_nodes, from_right)


def step_decomposed(engine, plan, comm, n):
    """n steps of one part: a step, then the halo exchange."""
    for _ in range(n):
        engine.step(1)
        exchange_halos(engine, plan, comm)
