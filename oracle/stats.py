"""Flow statistics of the paper's experiments, FP64 numpy (test infrastructure:
only tests/, smoke() and bench.py's CPU leg use this package).

Written from the definitions of the paper:
  Reynolds average (Sec. 4.3): arithmetic mean over the homogeneous directions
      x and z, per node plane of constant y index;
  Favre average (Sec. 4.3): phi~ = mean(rho phi) / mean(rho);
  Reynolds stresses (Eq. rij): mean(rho) R_ab = mean(rho u_a'' u_b''),
      u'' = u - u~;
  momentum thickness (Sec. 4.4): delta_theta = 1 / (rho0 du^2) * integral over
      y of rho_bar (du/2 - u1~)(du/2 + u1~);
  vorticity thickness (Sec. 4.4): delta_omega = du / max |d u1_bar / dy|;
  pressure coefficient (Sec. 4.2): C_P = (p - p0) / (gamma/2 p0 Ma^2), p = rho T.
Readings: the y integral is that of the piecewise order-p interpolant of the
plane values on the mesh's y cells; d/dy is the derivative of that interpolant
at the nodes, the largest magnitude over every (cell, node) pair.

Parity: pinned by closed forms in tests/test_oracle_stats.py.
"""
import numpy as np

from .mesh import KIND_NACA, glc_nodes, lagrange_1d, lagrange_1d_deriv


def _planes(mesh, a):
    """a [N, ...] -> [N1, N0 * N2, ...] grouped by y index (nodes x fastest)."""
    N0, N1 = mesh.N[0], mesh.N[1]
    N2 = mesh.N[2] if mesh.D == 3 else 1
    a = np.asarray(a).reshape((N2, N1, N0) + np.shape(a)[1:])
    return np.moveaxis(a, 1, 0).reshape((N1, N2 * N0) + np.shape(a)[3:])


def plane_profiles(mesh, rho, u, T):
    """Per y-node plane: y, rho_bar, u_bar [N1, D], u_favre [N1, D], T_bar,
    p_bar (p = rho T), R [N1, D, D] (Favre Reynolds stresses)."""
    return plane_profiles_over_states(mesh, [(rho, u, T)])


def plane_profiles_over_states(mesh, states):
    """plane_profiles with the averages taken over x, z and a list of states
    [(rho, u, T), ...] (Reynolds averages over the homogeneous directions and
    time): every state contributes its nodes of each plane as samples."""
    if mesh.kind == KIND_NACA:
        raise ValueError("plane statistics need an axis-aligned mesh")
    r = np.concatenate([_planes(mesh, s[0]) for s in states], axis=1)
    U = np.concatenate([_planes(mesh, s[1]) for s in states], axis=1)
    t = np.concatenate([_planes(mesh, s[2]) for s in states], axis=1)
    rb = r.mean(axis=1)
    ub = U.mean(axis=1)
    uf = (r[:, :, None] * U).mean(axis=1) / rb[:, None]
    up = U - uf[:, None, :]                               # u'' = u - u~
    R = (r[:, :, None, None] * up[:, :, :, None] * up[:, :, None, :]).mean(axis=1) / rb[:, None, None]
    y = _planes(mesh, mesh.X)[:, 0, 1]
    return dict(y=y, rho=rb, u=ub, u_favre=uf, T=t.mean(axis=1), p=(r * t).mean(axis=1), R=R)


def _y_cells(mesh):
    """(cell lower vertex, upper vertex, node indices [p+1]) for every y cell."""
    p = mesh.p
    V = mesh.vertices[1]
    N1 = mesh.N[1]
    return [(V[c], V[c + 1], np.array([(c * p + a) % N1 for a in range(p + 1)])) for c in range(mesh.cells[1])]


def mixing_thickness(mesh, prof, du, rho0):
    """(delta_theta, delta_omega) from plane_profiles output."""
    p = mesh.p
    xg, wg = np.polynomial.legendre.leggauss(8)          # exact for the interpolant's degree <= 2p < 15
    Lg = lagrange_1d(p, xg)                              # [8, p+1]
    I = prof["rho"] * (0.5 * du - prof["u_favre"][:, 0]) * (0.5 * du + prof["u_favre"][:, 0])
    u1 = prof["u"][:, 0]
    dL = lagrange_1d_deriv(p, glc_nodes(p))              # [node a, basis b]
    theta, slope = 0.0, 0.0
    for lo, hi, j in _y_cells(mesh):
        h = hi - lo
        theta += 0.5 * h * float(wg @ (Lg @ I[j]))
        slope = max(slope, float(np.abs(dL @ u1[j]).max()) * 2.0 / h)
    return theta / (rho0 * du * du), du / slope


def pressure_coefficient(rho, T, p0, mach, gamma):
    """C_P = (p - p0) / (gamma/2 p0 Ma^2) with p = rho T."""
    return (np.asarray(rho) * np.asarray(T) - p0) / (0.5 * gamma * p0 * mach * mach)


def plane_nodes(mesh, side):
    """Node indices of the plane y index 0 (side 0) or N1 - 1 (side 1), x fastest
    then z (for the O-grid: the airfoil surface and the far-field ring)."""
    j = 0 if side == 0 else mesh.N[1] - 1
    N0, N1 = mesh.N[0], mesh.N[1]
    N2 = mesh.N[2] if mesh.D == 3 else 1
    kx, kz = np.meshgrid(np.arange(N0), np.arange(N2), indexing="xy")
    return (kx + N0 * (j + N1 * kz)).ravel()
