"""Pins of the statistics oracle (Sec. 4.2-4.4 definitions) by closed forms."""
import math

import numpy as np
import pytest

from oracle import stats
from oracle.mesh import Mesh


def _fields_cos(mesh, eps, A, B, U0, T0, th):
    x = mesh.X[:, 0]
    k = 2 * math.pi / mesh.length[0]
    c, s = np.cos(k * x), np.sin(k * x)
    rho = 1.0 + eps * c
    u = np.zeros((mesh.n_nodes, mesh.D))
    u[:, 0] = U0 + A * c
    u[:, 1] = B * s
    T = T0 + th * c
    return rho, u, T


@pytest.mark.parametrize("p", [2, 4])
def test_favre_and_reynolds_closed_forms(p):
    """rho = 1 + e cos kx, u = U0 + A cos kx, v = B sin kx, T = T0 + th cos kx
    on equally spaced x nodes over one period (p = 2 GLC nodes are equally
    spaced; p = 4 nodes are not, so there only the Favre identities that do
    not use the discrete orthogonality are checked)."""
    mesh = Mesh(0, p, (8, 3), (2.0, 1.0))
    e, A, B, U0, T0, th = 0.2, 0.3, 0.25, 0.7, 1.1, 0.05
    rho, u, T = _fields_cos(mesh, e, A, B, U0, T0, th)
    pr = stats.plane_profiles(mesh, rho, u, T)
    assert pr["y"].shape == (mesh.N[1],)
    if p == 2:
        assert np.allclose(pr["rho"], 1.0, atol=1e-14)
        assert np.allclose(pr["u"][:, 0], U0, atol=1e-14)
        assert np.allclose(pr["u_favre"][:, 0], U0 + e * A / 2, atol=1e-14)
        assert np.allclose(pr["u_favre"][:, 1], 0.0, atol=1e-14)
        assert np.allclose(pr["T"], T0, atol=1e-14)
        assert np.allclose(pr["p"], T0 + e * th / 2, atol=1e-14)
        assert np.allclose(pr["R"][:, 0, 0], A * A * (0.5 - e * e / 4), atol=1e-14)
        assert np.allclose(pr["R"][:, 1, 1], B * B / 2, atol=1e-14)
        assert np.allclose(pr["R"][:, 0, 1], 0.0, atol=1e-14)
    # identities that hold on any node set: mean(rho u'') = 0, R symmetric and
    # R = mean(rho u u) / rho_bar - u~ u~
    r = stats._planes(mesh, rho)
    U = stats._planes(mesh, u)
    assert np.abs((r[:, :, None] * (U - pr["u_favre"][:, None, :])).mean(1)).max() < 1e-14
    assert np.abs(pr["R"] - np.swapaxes(pr["R"], 1, 2)).max() < 1e-17
    R2 = (r[:, :, None, None] * U[:, :, :, None] * U[:, :, None, :]).mean(1) / pr["rho"][:, None, None] \
        - pr["u_favre"][:, :, None] * pr["u_favre"][:, None, :]
    assert np.abs(pr["R"] - R2).max() < 1e-14


def test_thickness_exact_for_a_linear_profile():
    """rho = 1, u1 = c (y - 1) on the channel's stretched p = 4 y cells over
    [0, 2]: delta_theta = 1/2 - 2 c^2 / (3 du^2) and delta_omega = du / |c|,
    exactly (the interpolant reproduces the quadratic integrand)."""
    mesh = Mesh(1, 4, (2, 5, 2), (1.0, 2.0, 1.0), 2.0)
    c, du = -0.6, 1.7
    u = np.zeros((mesh.n_nodes, 3))
    u[:, 0] = c * (mesh.X[:, 1] - 1.0)
    pr = stats.plane_profiles(mesh, np.ones(mesh.n_nodes), u, np.ones(mesh.n_nodes))
    th, om = stats.mixing_thickness(mesh, pr, du, 1.0)
    assert abs(th - (0.5 - 2 * c * c / (3 * du * du))) < 1e-14
    assert abs(om - du / abs(c)) < 1e-12


def test_thickness_of_a_tanh_profile_converges():
    """u1 = (du/2) tanh(-y / (2a)), rho = rho0: delta_theta = a and
    delta_omega = 4 a in the continuum; the discrete values converge."""
    a, du = 0.25, 1.3
    errs = []
    for cells in (16, 48):
        mesh = Mesh(2, 2, (2, cells, 2), (1.0, 8.0, 1.0), 1.0, cells)
        u = np.zeros((mesh.n_nodes, 3))
        u[:, 0] = 0.5 * du * np.tanh(-mesh.X[:, 1] / (2 * a))
        pr = stats.plane_profiles(mesh, np.ones(mesh.n_nodes), u, np.ones(mesh.n_nodes))
        th, om = stats.mixing_thickness(mesh, pr, du, 1.0)
        errs.append((abs(th - a) / a, abs(om - 4 * a) / (4 * a)))
    assert errs[1][0] < 1e-5 and errs[1][1] < 2e-2
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1]


def test_pressure_coefficient():
    g, ma, p0 = 1.4, 1.5, 0.8
    assert np.allclose(stats.pressure_coefficient([1.0, 2.0], [0.8, 0.4], p0, ma, g), 0.0)
    e = 0.03
    cp = stats.pressure_coefficient([1.0], [p0 * (1 + e)], p0, ma, g)
    assert abs(cp[0] - e / (0.5 * g * ma * ma)) < 1e-15


def test_plane_nodes_are_the_boundary_planes():
    mesh = Mesh(1, 2, (3, 2, 2), (1.0, 2.0, 1.0), 2.0)
    for side, y in ((0, 0.0), (1, 2.0)):
        n = stats.plane_nodes(mesh, side)
        assert len(n) == mesh.N[0] * mesh.N[2] and len(set(n)) == len(n)
        assert np.allclose(mesh.X[n, 1], y)


def test_averages_over_states():
    """Time averages: one state repeated gives the instantaneous profiles; the
    Reynolds means of two states are the averages of their means; R over two
    states includes the fluctuation between them (u1 = +-A in the two states
    of a uniform field: R_11 = A^2)."""
    mesh = Mesh(0, 2, (6, 3), (2.0, 1.0))
    rho, u, T = _fields_cos(mesh, 0.1, 0.2, 0.1, 0.5, 1.0, 0.02)
    one = stats.plane_profiles(mesh, rho, u, T)
    rep = stats.plane_profiles_over_states(mesh, [(rho, u, T)] * 3)
    for k in ("rho", "u", "u_favre", "T", "p", "R"):
        assert np.abs(one[k] - rep[k]).max() < 1e-15
    u2 = u * 1.3
    two = stats.plane_profiles_over_states(mesh, [(rho, u, T), (rho, u2, T)])
    assert np.abs(two["u"] - 0.5 * (one["u"] + stats.plane_profiles(mesh, rho, u2, T)["u"])).max() < 1e-15
    A = 0.3
    ones = np.ones(mesh.n_nodes)
    ua, ub = np.zeros((mesh.n_nodes, 2)), np.zeros((mesh.n_nodes, 2))
    ua[:, 0], ub[:, 0] = A, -A
    pr = stats.plane_profiles_over_states(mesh, [(ones, ua, ones), (ones, ub, ones)])
    assert np.allclose(pr["u_favre"][:, 0], 0.0, atol=1e-16) and np.allclose(pr["R"][:, 0, 0], A * A, rtol=1e-15)
