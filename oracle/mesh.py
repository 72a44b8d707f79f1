"""Meshes of order-p Lagrange cells (Sec. 3.1, Eq. intf), FP64 oracle.
TEST INFRASTRUCTURE ONLY.

Every mesh here is logically structured: cells (c_0, .., c_{D-1}) with order-p
support points at the Gauss-Lobatto-Chebyshev positions xhat_k = -cos(pi k / p)
(Tab. 2 caption), shared between neighbouring cells (continuous numbering),
periodic dimensions identified.  Node linear index n = k_0 + N_0 (k_1 + N_1 k_2)
(first dimension fastest); cell linear index c = c_0 + C_0 (c_1 + C_1 c_2).

Kinds
  box      periodic in every dimension, uniform cells on [0, L_d)
  channel  x, z periodic uniform; y in [0, Ly] with tanh wall clustering
           y_j = (Ly/2) [1 - tanh(beta (1 - 2 j / C_y)) / tanh(beta)]
  mixing   x, z periodic uniform; y in [-Ly/2, Ly/2]: `central` uniform cells
           in the middle, cells growing by the factor `stretch` outside
  naca     2D O-grid around a NACA-00tt profile (closed trailing edge form of
           the thickness formula); the surface point of angle phi = 2 pi s / C_0
           has chord position x = 1 - psi, psi = (1 - cos phi)/2
           + 0.25 |sin phi| (1 + cos phi)/2, and y = sign(sin phi) y_t(x);
           dim 0 = around (periodic), dim 1 = radial
           with geometric growth `stretch` per cell up to a circle of radius R
           centred at mid-chord; cells are isoparametric of degree p over
           their own support points (curved cells).

  explicit axis-aligned cells on given vertex coordinates per dimension; x and
           z periodic, y periodic when `periodic_y`; a periodic dimension
           starts at 0 and its length is its last vertex.

For the box / channel / mixing / explicit kinds cells are axis-aligned boxes
and the cell map is affine per dimension.
"""
import math

import numpy as np

KIND_BOX, KIND_CHANNEL, KIND_MIXING, KIND_NACA, KIND_EXPLICIT = 0, 1, 2, 3, 4
TE_BLEND = 0.25


def glc_nodes(p):
    return -np.cos(np.pi * np.arange(p + 1) / p)


def lagrange_1d(p, xi):
    """Values of the p+1 Lagrange polynomials on the GLC nodes at xi (any shape)."""
    xh = glc_nodes(p)
    xi = np.asarray(xi, dtype=np.float64)
    out = []
    for a in range(p + 1):
        v = np.ones_like(xi)
        for m in range(p + 1):
            if m != a:
                v = v * (xi - xh[m]) / (xh[a] - xh[m])
        out.append(v)
    return np.stack(out, axis=-1)


def lagrange_1d_deriv(p, xi):
    xh = glc_nodes(p)
    xi = np.asarray(xi, dtype=np.float64)
    out = []
    for a in range(p + 1):
        tot = np.zeros_like(xi)
        for j in range(p + 1):
            if j == a:
                continue
            v = np.ones_like(xi) / (xh[a] - xh[j])
            for m in range(p + 1):
                if m != a and m != j:
                    v = v * (xi - xh[m]) / (xh[a] - xh[m])
            tot = tot + v
        out.append(tot)
    return np.stack(out, axis=-1)


def naca_half_thickness(x, t):
    """NACA 4-digit symmetric half thickness, closed trailing edge coefficient."""
    x = np.clip(x, 0.0, 1.0)
    return 5.0 * t * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2
                      + 0.2843 * x ** 3 - 0.1036 * x ** 4)


class Mesh:
    def __init__(self, kind, p, cells, length, stretch=1.0, central=0, thickness=0.12, vertices=None,
                 periodic_y=False):
        self.kind = kind
        self.p = p
        self.cells = tuple(int(c) for c in cells)
        self.D = len(self.cells)
        if kind == KIND_EXPLICIT:
            self._given = [np.asarray(v, dtype=np.float64) for v in vertices]
            length = [float(v[-1] - v[0]) for v in self._given]
        self.length = tuple(float(v) for v in length)
        self.stretch = float(stretch)
        self.central = int(central)
        self.thickness = float(thickness)
        D = self.D
        if kind == KIND_BOX:
            self.periodic = (True,) * D
        elif kind in (KIND_CHANNEL, KIND_MIXING):
            self.periodic = tuple(d != 1 for d in range(D))
        elif kind == KIND_NACA:
            assert D == 2
            self.periodic = (True, False)
        elif kind == KIND_EXPLICIT:
            self.periodic = tuple(d != 1 or bool(periodic_y) for d in range(D))
        else:
            raise ValueError(kind)
        self.N = tuple(c * p if per else c * p + 1 for c, per in zip(self.cells, self.periodic))
        self.n_nodes = int(np.prod(self.N))
        self.n_cells = int(np.prod(self.cells))
        if kind != KIND_NACA:
            self.vertices = [self._vertices_1d(d) for d in range(D)]
        self.X = self._node_coords()
        p1 = self.p + 1
        self._loc = np.array([np.unravel_index(j, (p1,) * D, order="F") for j in range(p1 ** D)])
        if kind == KIND_NACA:
            self.cellX = self.X[self.cell_nodes(np.arange(self.n_cells))]

    # ---------------------------------------------------------------- geometry
    def _vertices_1d(self, d):
        if self.kind == KIND_EXPLICIT:
            return self._given[d].copy()
        C, L = self.cells[d], self.length[d]
        j = np.arange(C + 1, dtype=np.float64)
        if d != 1 or self.kind == KIND_BOX:
            return L * j / C
        if self.kind == KIND_CHANNEL:
            b = self.stretch
            return 0.5 * L * (1.0 - np.tanh(b * (1.0 - 2.0 * j / C)) / math.tanh(b))
        # mixing layer: uniform centre, geometric growth outside
        nc = self.central
        side = (C - nc) // 2
        assert 2 * side + nc == C
        sizes = np.concatenate([self.stretch ** np.arange(side, 0, -1), np.ones(nc),
                                self.stretch ** np.arange(1, side + 1)])
        h = L / sizes.sum()
        v = np.concatenate([[0.0], np.cumsum(sizes * h)])
        return v - 0.5 * L

    def naca_logical_to_x(self, s, r):
        """Analytic O-grid map from logical (s around, r radial) in cell units."""
        Ca, Cr = self.cells
        R = self.length[1]
        ang = 2.0 * np.pi * np.asarray(s, dtype=np.float64) / Ca
        # chord position: cosine clustering at the leading edge (quadratic in the
        # angle there), a linear start at the trailing edge (no zero-speed corner)
        psi = 0.5 * (1.0 - np.cos(ang)) + TE_BLEND * np.abs(np.sin(ang)) * 0.5 * (1.0 + np.cos(ang))
        xs = 1.0 - psi
        sgn = np.where(np.sin(ang) >= 0.0, 1.0, -1.0)
        ys = sgn * naca_half_thickness(xs, self.thickness)
        xf = 0.5 + R * np.cos(ang)
        yf = R * np.sin(ang)
        q = self.stretch
        dr = (q ** np.asarray(r, dtype=np.float64) - 1.0) / (q ** Cr - 1.0)
        return np.stack([xs + dr * (xf - xs), ys + dr * (yf - ys)], axis=-1)

    def _node_logical(self, d, k):
        """Logical position (in cell units) of node index k along dimension d."""
        p = self.p
        xh = glc_nodes(p)
        c = np.minimum(k // p, self.cells[d] - 1)
        a = k - c * p
        return c + 0.5 * (xh[a] + 1.0)

    def _node_coords(self):
        D, p = self.D, self.p
        grids = np.meshgrid(*[np.arange(n) for n in self.N], indexing="ij")
        # node linear index has dim 0 fastest -> use Fortran order flatten
        ks = [g.ravel(order="F") for g in grids]
        if self.kind == KIND_NACA:
            s = self._node_logical(0, ks[0])
            r = self._node_logical(1, ks[1])
            return self.naca_logical_to_x(s, r)
        X = np.zeros((self.n_nodes, D))
        xh = glc_nodes(p)
        for d in range(D):
            V = self.vertices[d]
            k = ks[d]
            c = np.minimum(k // p, self.cells[d] - 1)
            a = k - c * p
            X[:, d] = V[c] + 0.5 * (xh[a] + 1.0) * (V[c + 1] - V[c])
        return X

    # ------------------------------------------------------------- numbering
    def node_index(self, k):
        """k: int array [..., D] of per-dimension node indices (wrapped)."""
        n = np.zeros(k.shape[:-1], dtype=np.int64)
        stride = 1
        for d in range(self.D):
            kd = k[..., d] % self.N[d] if self.periodic[d] else k[..., d]
            n = n + kd * stride
            stride *= self.N[d]
        return n

    def cell_coords(self, c):
        c = np.asarray(c, dtype=np.int64)
        out = []
        for d in range(self.D):
            out.append(c % self.cells[d])
            c = c // self.cells[d]
        return np.stack(out, axis=-1)

    def cell_index(self, cc):
        c = np.zeros(cc.shape[:-1], dtype=np.int64)
        stride = 1
        for d in range(self.D):
            c = c + cc[..., d] * stride
            stride *= self.cells[d]
        return c

    def cell_nodes(self, c):
        """Global node indices of the (p+1)^D support points of cells c [M];
        local ordering: first dimension fastest.  Shape [M, (p+1)^D]."""
        cc = self.cell_coords(c)
        p, D = self.p, self.D
        k = cc[:, None, :] * p + self._loc[None, :, :]
        return self.node_index(k)

    def basis(self, xi):
        """Tensor-product Lagrange basis at reference points xi [M, D] -> [M, (p+1)^D]."""
        p, D = self.p, self.D
        L = [lagrange_1d(p, xi[:, d]) for d in range(D)]
        out = L[0]
        for d in range(1, D):
            out = (out[:, None, :] * L[d][:, :, None]).reshape(len(xi), -1)
        return out

    def basis_grad(self, xi):
        """d basis / d xi_d -> [M, D, (p+1)^D]."""
        p, D = self.p, self.D
        L = [lagrange_1d(p, xi[:, d]) for d in range(D)]
        dL = [lagrange_1d_deriv(p, xi[:, d]) for d in range(D)]
        grads = []
        for e in range(D):
            parts = [dL[d] if d == e else L[d] for d in range(D)]
            out = parts[0]
            for d in range(1, D):
                out = (out[:, None, :] * parts[d][:, :, None]).reshape(len(xi), -1)
            grads.append(out)
        return np.stack(grads, axis=1)

    def cell_map(self, c, xi):
        """Physical position of reference points xi [M, D] in cells c [M]."""
        c = np.asarray(c)
        if self.kind == KIND_NACA:
            return np.einsum("mj,mjd->md", self.basis(xi), self.cellX[c])
        cc = self.cell_coords(c)
        out = np.zeros_like(xi)
        for d in range(self.D):
            V = self.vertices[d]
            lo, hi = V[cc[:, d]], V[cc[:, d] + 1]
            out[:, d] = lo + 0.5 * (xi[:, d] + 1.0) * (hi - lo)
        return out

    def cell_jacobian(self, c, xi):
        G = self.basis_grad(xi)
        return np.einsum("mej,mjd->mde", G, self.cellX[np.asarray(c)])

    def inverse_map(self, c, x, max_iter=50):
        """Reference coordinates of physical points x [M, D] in cells c [M]:
        closed form for affine cells, Newton from xi = 0 for curved cells."""
        c = np.asarray(c)
        if self.kind != KIND_NACA:
            cc = self.cell_coords(c)
            xi = np.zeros_like(x)
            for d in range(self.D):
                V = self.vertices[d]
                lo, hi = V[cc[:, d]], V[cc[:, d] + 1]
                xi[:, d] = 2.0 * (x[:, d] - lo) / (hi - lo) - 1.0
            return xi, np.ones(len(x), dtype=bool)
        xi = np.zeros_like(x)
        active = np.arange(len(x))
        for it in range(max_iter):
            if len(active) == 0:
                break
            ca, xa = c[active], xi[active]
            r = self.cell_map(ca, xa) - x[active]
            J = self.cell_jacobian(ca, xa)
            step = np.linalg.solve(J, r[:, :, None])[:, :, 0]
            step = np.clip(step, -1.0, 1.0)
            xa = np.clip(xa - step, -4.0, 4.0)
            xi[active] = xa
            done = np.abs(step).max(axis=1) < 1e-15
            # points that stay far outside the reference square cannot be inside
            far = (it >= 8) & (np.abs(xa).max(axis=1) > 2.0)
            active = active[~(done | far)]
        r = np.abs(self.cell_map(c, xi) - x).max(axis=1)
        ok = r < 1e-12
        return xi, ok

    def wrap(self, x):
        """Wrap periodic coordinates of physical points into the domain
        (box / channel / mixing: [lo_d, lo_d + L_d))."""
        x = x.copy()
        if self.kind == KIND_NACA:
            return x
        for d in range(self.D):
            if self.periodic[d]:
                x[:, d] = np.mod(x[:, d], self.length[d])
        return x
