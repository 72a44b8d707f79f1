"""Pins of the oracle meshes and interpolation (Sec. 3.1 Eq. intf)."""
import math

import numpy as np
import pytest

from oracle.departure import Locator
from oracle.mesh import KIND_BOX, KIND_CHANNEL, KIND_MIXING, KIND_NACA, Mesh, glc_nodes, lagrange_1d


def test_glc_nodes():
    """Tab. 2 caption: Gauss-Lobatto-Chebyshev points; p = 3 -> {-1, -1/2, 1/2, 1}."""
    assert np.allclose(glc_nodes(3), [-1, -0.5, 0.5, 1], atol=1e-15)
    assert np.allclose(glc_nodes(2), [-1, 0, 1], atol=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_lagrange_cardinal_and_partition(p):
    x = glc_nodes(p)
    assert np.abs(lagrange_1d(p, x) - np.eye(p + 1)).max() < 1e-14
    t = np.linspace(-1, 1, 37)
    assert np.abs(lagrange_1d(p, t).sum(1) - 1).max() < 1e-14


def _meshes():
    return [Mesh(KIND_BOX, 2, (4, 3), (2.0, 1.5)),
            Mesh(KIND_CHANNEL, 2, (3, 4, 2), (3.0, 2.0, 1.0), stretch=2.0),
            Mesh(KIND_MIXING, 2, (2, 8, 2), (4.0, 10.0, 2.0), stretch=1.1, central=4),
            Mesh(KIND_NACA, 3, (16, 6), (1.0, 20.0), stretch=1.3)]


@pytest.mark.parametrize("mesh", _meshes(), ids=["box", "channel", "mixing", "naca"])
def test_polynomial_reproduction(mesh):
    """Interpolating nodal values of a degree-p polynomial in the reference
    coordinates reproduces it exactly anywhere in the cell (affine cells: also a
    degree-p polynomial of x)."""
    rng = np.random.default_rng(0)
    p, D = mesh.p, mesh.D
    cc = np.stack([rng.integers(0, mesh.cells[d] - (1 if mesh.periodic[d] else 0), size=20)
                   for d in range(D)], axis=1)    # away from the periodic seam
    cells = mesh.cell_index(cc)
    xi = rng.uniform(-1, 1, size=(20, D))
    nodes = mesh.cell_nodes(cells)
    L = mesh.basis(xi)
    if mesh.kind == KIND_NACA:
        # a polynomial of degree p in each reference coordinate, evaluated at the cell's support points
        xh = glc_nodes(p)
        loc = mesh._loc
        coef = rng.normal(size=(p + 1, p + 1))
        vals = np.array([[sum(coef[a, b] * xh[loc[j, 0]] ** a * xh[loc[j, 1]] ** b
                              for a in range(p + 1) for b in range(p + 1)) for j in range(len(loc))]] * 20)
        exact = np.array([sum(coef[a, b] * x[0] ** a * x[1] ** b for a in range(p + 1) for b in range(p + 1))
                          for x in xi])
        assert np.abs((L * vals).sum(1) - exact).max() < 1e-12
        return
    X = mesh.X
    c = rng.normal(size=D)

    def poly(x):
        return 0.3 + (x * c).sum(-1) ** p + x[..., 0] ** p

    xphys = mesh.cell_map(cells, xi)
    got = (L * poly(X[nodes])).sum(1)
    assert np.abs(got - poly(xphys)).max() < 1e-11


def test_channel_tanh_vertices():
    m = Mesh(KIND_CHANNEL, 2, (4, 8, 4), (1.0, 2.0, 1.0), stretch=2.0)
    V = m.vertices[1]
    j = np.arange(9)
    assert np.allclose(V, 1.0 - np.tanh(2.0 * (1 - 2 * j / 8)) / math.tanh(2.0), atol=1e-15)
    assert V[0] == 0.0 and abs(V[-1] - 2.0) < 1e-15
    assert np.all(np.diff(V)[:4] > 0) and np.diff(V)[0] < np.diff(V)[3]


def test_mixing_vertices():
    m = Mesh(KIND_MIXING, 2, (2, 12, 2), (1.0, 10.0, 1.0), stretch=1.1, central=4)
    h = np.diff(m.vertices[1])
    assert abs(m.vertices[1][0] + 5) < 1e-14 and abs(m.vertices[1][-1] - 5) < 1e-13
    assert np.allclose(h[4:8], h[4]) and np.allclose(h[8:] / h[7:-1], 1.1)


def test_naca_surface_and_jacobian():
    """Wall nodes lie on the NACA-0012 half-thickness curve; the O-grid maps
    with positive Jacobian everywhere; the far field is a circle of radius R."""
    m = Mesh(KIND_NACA, 3, (32, 12), (1.0, 20.0), stretch=1.2)
    Na = m.N[0]
    wall = m.X[:Na]
    x = wall[:, 0]
    yt = 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x ** 2 + 0.2843 * x ** 3 - 0.1036 * x ** 4)
    assert np.abs(np.abs(wall[:, 1]) - yt).max() < 1e-14
    assert abs(yt.max() - 0.06) < 2e-3          # 12 % thickness
    ff = m.X[-Na:]
    assert np.allclose(np.linalg.norm(ff - np.array([0.5, 0.0]), axis=1), 20.0)
    c = np.arange(m.n_cells)
    dets = []
    for xi in ([-1, -1], [1, 1], [0, 0], [1, -1], [-1, 1]):
        J = m.cell_jacobian(c, np.tile(np.array(xi, float), (m.n_cells, 1)))
        dets.append(np.linalg.det(J))
    dets = np.concatenate(dets)
    assert (dets < 0).all()                      # one orientation everywhere, never singular


def test_newton_inverse_map():
    m = Mesh(KIND_NACA, 3, (16, 6), (1.0, 20.0), stretch=1.3)
    rng = np.random.default_rng(1)
    c = rng.integers(0, m.n_cells, 50)
    xi = rng.uniform(-1, 1, (50, 2))
    x = m.cell_map(c, xi)
    xi2, ok = m.inverse_map(c, x)
    assert ok.all() and np.abs(xi2 - xi).max() < 1e-10
    assert np.abs(m.cell_map(c, xi2) - x).max() < 1e-12


def test_locator_finds_points():
    m = Mesh(KIND_NACA, 3, (16, 6), (1.0, 20.0), stretch=1.3)
    rng = np.random.default_rng(2)
    c = rng.integers(0, m.n_cells, 40)
    xi = rng.uniform(-0.9, 0.9, (40, 2))
    x = m.cell_map(c, xi)
    loc = Locator(m)
    cc, xr = loc.locate(x)
    assert (cc == c).all() and np.abs(xr - xi).max() < 1e-10
    cc, _ = loc.locate(np.array([[0.5, 0.0], [30.0, 0.0]]))   # inside the profile / beyond the far field
    assert (cc == -1).all()


def test_explicit_mesh_reproduces_the_analytic_kinds():
    """The explicit kind on the vertices of a channel (walls in y) or a box
    (periodic y) gives the same nodes, counts and periodicity: its
    construction is pinned to the analytic kinds'."""
    import numpy as np
    from oracle.mesh import KIND_BOX, KIND_CHANNEL, KIND_EXPLICIT, Mesh
    ch = Mesh(KIND_CHANNEL, 2, (4, 5, 3), (6.0, 2.0, 3.0), stretch=2.0)
    ex = Mesh(KIND_EXPLICIT, 2, (4, 5, 3), (0.0, 0.0, 0.0), vertices=ch.vertices)
    assert ex.periodic == ch.periodic and ex.N == ch.N and ex.length == ch.length
    assert np.array_equal(ex.X, ch.X)
    bx = Mesh(KIND_BOX, 3, (3, 4), (2.0, 1.5))
    ex = Mesh(KIND_EXPLICIT, 3, (3, 4), (0.0, 0.0), vertices=bx.vertices, periodic_y=True)
    assert ex.periodic == (True, True) and np.array_equal(ex.X, bx.X)
