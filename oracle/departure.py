"""Departure points and boundary records (Sec. 3.1, Sec. 3.3), FP64 oracle.
TEST INFRASTRUCTURE ONLY.

For every arrival point (AP) x_n and velocity zeta_i the departure point (DP)
is x_n - dt zeta_i (Sec. 3.1).  The DP's cell is found by brute force: every
cell whose (enlarged) bounding box contains the point is tested with the
inverse cell map; the lowest cell id among the containing cells wins.  When no
cell contains the DP the trajectory has left the domain; the crossing
parameter t_W of x_n - t dt zeta_i with the boundary is found by 60 bisection
steps on "inside", giving the wall point x_W.  Then, by the boundary kind:

  equilibrium  f_i(AP) = f_i^eq(rho_w, u_w, T_w)                   (Sec. 3.3.1)
  bounce-back  f_i(AP) = f_ibar(x_W + iota), iota = zeta_i dt - (x_AP - x_W)
                                                                   (Sec. 3.3.2)
  isothermal   bounce-back plus the thermal correction of the node (Eq. thermalBC)
  outlet       f_i(AP) = f_i(x_AP + zeta_i dt)                     (Sec. 3.3.3)
  far field    equilibrium where x_W lies upstream of mid-chord, outlet downstream

Reading where the paper is silent: a reflected or mirrored point that again
leaves the domain is moved back along its segment to the last inside point
(60 bisection steps).
"""
import numpy as np
from scipy.spatial import cKDTree

from .mesh import KIND_NACA

BC_PERIODIC, BC_EQUILIBRIUM, BC_BOUNCEBACK, BC_ISOTHERMAL, BC_OUTLET, BC_FARFIELD = range(6)
REC_INTERIOR, REC_EQ, REC_BB, REC_BB_ISO, REC_OUTLET = range(5)


class Locator:
    """Brute-force point location (bounding-box prefilter + inverse map)."""

    def __init__(self, mesh):
        self.mesh = mesh
        if mesh.kind == KIND_NACA:
            nodes = mesh.cell_nodes(np.arange(mesh.n_cells))
            P = mesh.X[nodes]                       # [C, (p+1)^2, 2]
            lo, hi = P.min(1), P.max(1)
            self.center = 0.5 * (lo + hi)
            self.half = 0.5 * (hi - lo).max(1) * 1.25 + 1e-12

    def locate(self, x):
        """cells [M] (-1 outside) and reference coordinates [M, D]."""
        m = self.mesh
        x = m.wrap(np.atleast_2d(x))
        M = len(x)
        if m.kind != KIND_NACA:
            cc = np.zeros((M, m.D), dtype=np.int64)
            inside = np.ones(M, dtype=bool)
            for d in range(m.D):
                V = m.vertices[d]
                if not m.periodic[d]:
                    inside &= (x[:, d] >= V[0]) & (x[:, d] <= V[-1])
                cc[:, d] = np.clip(np.searchsorted(V, x[:, d], side="left") - 1, 0, m.cells[d] - 1)
            cell = m.cell_index(cc)
            xi, _ = m.inverse_map(cell, x)
            cell = np.where(inside, cell, -1)
            return cell, xi
        tree = cKDTree(x)
        lists = tree.query_ball_point(self.center, r=self.half, p=np.inf)
        pc = [(j, c) for c, lst in enumerate(lists) for j in lst]
        cell = np.full(M, -1, dtype=np.int64)
        xi_out = np.zeros((M, 2))
        if not pc:
            return cell, xi_out
        pc = np.array(pc, dtype=np.int64)
        pc = pc[np.lexsort((pc[:, 1], pc[:, 0]))]
        xi, ok = m.inverse_map(pc[:, 1], x[pc[:, 0]])
        inside = ok & (np.abs(xi).max(1) <= 1.0 + 1e-12)
        pc, xi = pc[inside], xi[inside]
        # lowest containing cell per point: pairs are sorted by (point, cell)
        first = np.ones(len(pc), dtype=bool)
        first[1:] = pc[1:, 0] != pc[:-1, 0]
        cell[pc[first, 0]] = pc[first, 1]
        xi_out[pc[first, 0]] = xi[first]
        return cell, xi_out


def _bisect(loc, x0, dirv, n_iter=60):
    """Largest t in [0,1] (to 2^-60) with x0 + t dirv inside, given x0 inside
    and x0 + dirv outside.  Returns (t_lo, t_hi)."""
    lo = np.zeros(len(x0))
    hi = np.ones(len(x0))
    for _ in range(n_iter):
        mid = 0.5 * (lo + hi)
        c, _ = loc.locate(x0 + mid[:, None] * dirv)
        ins = c >= 0
        lo = np.where(ins, mid, lo)
        hi = np.where(ins, hi, mid)
    return lo, hi


def boundary_id(mesh, xw, x_dp):
    """Which boundary the trajectory crossed: 0 = low side / wall, 1 = high side / far field."""
    if mesh.kind == KIND_NACA:
        r = np.linalg.norm(xw - np.array([0.5, 0.0]), axis=1)
        return (r > 0.5 * mesh.length[1]).astype(np.int64)
    V = mesh.vertices[1]
    return (x_dp[:, 1] > V[-1]).astype(np.int64)


def trace(mesh, xi_set, opp, dt, bcs, nodes=None):
    """Departure records for every (velocity i, node n), all velocities at once.

    bcs: list of two dicts (bid 0, bid 1) with key 'kind' (BC_* constant).
    nodes: optional subset of arrival nodes (default: all nodes).
    Returns dict of arrays [Q, N]: kind, src, bid, cell, tw, xi [Q, N, D], xsrc [Q, N, D].
    """
    loc = Locator(mesh)
    Q = len(xi_set)
    Xa = mesh.X if nodes is None else mesh.X[np.asarray(nodes)]
    N, D = len(Xa), mesh.D
    X = np.broadcast_to(Xa[None], (Q, N, D)).reshape(-1, D)
    step = np.broadcast_to((dt * xi_set)[:, None, :], (Q, N, D)).reshape(-1, D)
    vel = np.repeat(np.arange(Q), N)
    M = Q * N
    xdp = X - step
    cell, _ = loc.locate(xdp)
    kind = np.full(M, REC_INTERIOR)
    src = vel.copy()
    bid = np.full(M, -1)
    tw_all = np.full(M, np.nan)
    xsrc = mesh.wrap(xdp)
    outside = np.nonzero(cell < 0)[0]
    if len(outside):
        x0 = X[outside]
        st = step[outside]
        tlo, thi = _bisect(loc, x0, -st)
        tw = 0.5 * (tlo + thi)
        xw_in = x0 - tlo[:, None] * st
        xw = x0 - tw[:, None] * st
        b = boundary_id(mesh, xw, xdp[outside])
        tw_all[outside] = tw
        bid[outside] = b
        bk = np.array([bcs[k]["kind"] for k in b])
        if mesh.kind == KIND_NACA:
            ff = bk == BC_FARFIELD
            bk = np.where(ff & (xw[:, 0] < 0.5), BC_EQUILIBRIUM, np.where(ff, BC_OUTLET, bk))
        kind[outside[bk == BC_EQUILIBRIUM]] = REC_EQ
        # bounce-back / isothermal: reflected point x_W + iota
        sel = (bk == BC_BOUNCEBACK) | (bk == BC_ISOTHERMAL)
        if sel.any():
            nn = outside[sel]
            iota = st[sel] - (x0[sel] - xw[sel])
            xref = xw[sel] + iota
            c2, _ = loc.locate(xref)
            bad = c2 < 0
            if bad.any():
                a = xw_in[sel][bad]
                lo2, _ = _bisect(loc, a, xref[bad] - a)
                xref[bad] = a + lo2[:, None] * (xref[bad] - a)
            xsrc[nn] = mesh.wrap(xref)
            src[nn] = opp[vel[nn]]
            kind[nn] = np.where(bk[sel] == BC_ISOTHERMAL, REC_BB_ISO, REC_BB)
        # outlet: mirrored point x_AP + zeta_i dt
        sel = bk == BC_OUTLET
        if sel.any():
            nn = outside[sel]
            xm = x0[sel] + st[sel]
            c2, _ = loc.locate(xm)
            bad = c2 < 0
            if bad.any():
                a = x0[sel][bad]
                lo2, _ = _bisect(loc, a, xm[bad] - a)
                xm[bad] = a + lo2[:, None] * (xm[bad] - a)
            xsrc[nn] = mesh.wrap(xm)
            kind[nn] = REC_OUTLET
    # locate every source point (equilibrium records keep cell = -1)
    need = kind != REC_EQ
    c_all, xi_all = loc.locate(xsrc[need])
    cell_f = np.full(M, -1)
    xi_f = np.zeros((M, D))
    cell_f[need] = c_all
    xi_f[need] = xi_all
    assert (cell_f[need] >= 0).all(), "source point outside the mesh"
    shp = (Q, N)
    return dict(kind=kind.reshape(shp), src=src.reshape(shp), bid=bid.reshape(shp),
                cell=cell_f.reshape(shp), tw=tw_all.reshape(shp),
                xi=xi_f.reshape(Q, N, D), xsrc=xsrc.reshape(Q, N, D))
