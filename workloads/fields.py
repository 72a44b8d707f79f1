"""Seeded macroscopic initial fields evaluated at caller-supplied node coordinates."""
import math

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.Philox(int(seed)))


def initial_fields(cfg, X, seed=None):
    """rho [N], u [N, D], T [N] for the config's initial condition at nodes X [N, D]."""
    ini = cfg["init"]
    kind = ini["kind"]
    X = np.asarray(X, dtype=np.float64)
    N, D = X.shape
    rho = np.ones(N)
    T = np.ones(N)
    u = np.zeros((N, D))
    if kind == "taylor_green":
        U = ini["U"]
        x, y = X[:, 0], X[:, 1]
        u[:, 0] = U * np.sin(x) * np.cos(y)
        u[:, 1] = -U * np.cos(x) * np.sin(y)
        p = 1.0 + 0.25 * U * U * (np.cos(2 * x) + np.cos(2 * y))
        rho = p / T
    elif kind == "naca_freestream":
        U = ini["U"]
        u[:, 0] = U
        u[:, 1] = 0.1 * U * np.sin(1.3 * X[:, 1] + 0.1)
    elif kind == "channel_laminar":
        ub, amp = ini["ub"], ini["amp"]
        T = np.full(N, ini.get("T", 1.0))
        y = X[:, 1]
        shape = 1.0 - (y - 1.0) ** 2
        u[:, 0] = 1.5 * ub * shape
        r = _rng(ini["seed"] if seed is None else seed).uniform(-1.0, 1.0, size=(N, D))
        u += amp * ub * shape[:, None] * r
    elif kind == "mixing_layer":
        # tanh profile with delta_omega0 = 1 (delta_theta0 = 1/4) plus the
        # solenoidal broadband disturbance of Sec. 4.4, max |u'| = amp * du
        du, amp = ini["du"], ini["amp"]
        y = X[:, 1]
        u[:, 0] = 0.5 * du * np.tanh(-y / 1.0 * 2.0)
        u += spectral_broadband(X, amp * du, 0.25, ini["seed"] if seed is None else seed)
    elif kind == "isentropic_vortex":
        # Shu's isentropic vortex of strength eps advected by a uniform stream
        mach = ini["mach"]
        r = _rng(ini["seed"] if seed is None else seed)
        L = 2.0 * math.pi
        xc, yc = r.uniform(0.3 * L, 0.7 * L, size=2)
        U0 = mach * math.sqrt(1.4)
        eps = ini.get("eps", 2.5)
        R = ini.get("R", 1.0)                       # core radius
        if "center" in ini:
            xc, yc = ini["center"]
        dx, dy = (X[:, 0] - xc) / R, (X[:, 1] - yc) / R
        r2 = dx * dx + dy * dy
        e = np.exp(0.5 * (1.0 - r2))
        u[:, 0] = U0 - eps / (2.0 * math.pi) * e * dy
        u[:, 1] = eps / (2.0 * math.pi) * e * dx
        T = 1.0 - 0.4 * eps * eps / (8.0 * 1.4 * math.pi ** 2) * e * e
        rho = T ** (1.0 / 0.4)
    elif kind == "shear_layer":
        mach = ini["mach"]
        U0 = mach * math.sqrt(1.4)
        y = X[:, 1]
        L = 2.0 * math.pi
        u[:, 0] = U0 * np.tanh((y - 0.5 * L) / 0.3)
        r = _rng(ini.get("seed", 0) if seed is None else seed).uniform(-1.0, 1.0, size=2)
        u[:, 1] = 0.05 * U0 * (np.sin(X[:, 0] + r[0]) + 0.5 * np.sin(2 * X[:, 0] + r[1]))
    else:
        raise ValueError(kind)
    return rho, u, T


def _grid_of(X):
    """Axes and per-node indices of nodes that form a tensor-product grid."""
    N, D = X.shape
    axes, idx = [], []
    for d in range(D):
        a = np.unique(np.round(X[:, d], 12))
        axes.append(a)
        idx.append(np.searchsorted(a, np.round(X[:, d], 12)))
    if int(np.prod([len(a) for a in axes])) != N:
        raise ValueError("nodes do not form a tensor-product grid")
    return axes, idx


def spectral_broadband(X, amp_abs, dtheta0, seed, kdecay=24.0):
    """Solenoidal broadband velocity disturbance after the recipe of Sec. 4.4:
    a random vector potential with values uniform in [0, 1] on the node grid
    (one scalar potential in 2D), scaled in spectral space by exp(-|k| / 24)
    (k: integer wavenumbers of the node grid, one period per grid length in
    each direction), multiplied by exp(-(x2 / (2 dtheta0))^2) and differentiated:
    u' = curl(g Xi).  Derivatives are spectral in node-index space times
    d(index)/dx from the node spacing (the grid may be stretched).  Scaled so
    that max |u'| = amp_abs.  X: [N, D] nodes on a tensor-product grid."""
    N, D = X.shape
    axes, idx = _grid_of(X)
    shape = tuple(len(a) for a in axes)               # (n0, n1[, n2]) in x, y, z order
    r = _rng(seed)
    ncomp = 3 if D == 3 else 1
    xi0 = r.uniform(0.0, 1.0, size=(ncomp,) + shape)
    kv = np.meshgrid(*[np.fft.fftfreq(n) * n for n in shape], indexing="ij")
    kabs = np.sqrt(sum(k * k for k in kv))
    F = np.fft.fftn(xi0, axes=tuple(range(1, D + 1))) * np.exp(-kabs / kdecay)
    Xi = np.fft.ifftn(F, axes=tuple(range(1, D + 1))).real
    # d(Xi)/dx_d: spectral derivative in index space / (dx_d / d index)
    dXi = []
    for d in range(D):
        ik = 2j * np.pi * kv[d] / shape[d]
        dd = np.fft.ifftn(F * ik, axes=tuple(range(1, D + 1))).real
        h = np.gradient(axes[d])                      # dx_d per index step
        sh = [1] * (D + 1)
        sh[d + 1] = -1
        dXi.append(dd / h.reshape(sh))
    y = axes[1]
    g = np.exp(-(y / (2.0 * dtheta0)) ** 2)
    gp = -y / (2.0 * dtheta0 ** 2) * g                 # dg/dy
    sh = [1] * D
    sh[1] = -1
    g, gp = g.reshape(sh), gp.reshape(sh)
    if D == 2:
        psi, (dpx, dpy) = Xi[0], (dXi[0][0], dXi[1][0])
        comp = [g * dpy + gp * psi, -g * dpx]
    else:
        # curl(g Xi) = g curl(Xi) + grad(g) x Xi, grad(g) = (0, g', 0)
        Xx, Xy, Xz = Xi
        comp = [g * (dXi[1][2] - dXi[2][1]) + gp * Xz,
                g * (dXi[2][0] - dXi[0][2]),
                g * (dXi[0][1] - dXi[1][0]) - gp * Xx]
    up = np.stack([c[tuple(idx)] for c in comp], axis=1)
    m = np.abs(up).max()
    return up * (amp_abs / m) if m > 0 else up


def random_state_perturbation(Q, N, seed, amp):
    """Seeded uniform perturbation [Q, N] in [-amp, amp] (for parity tests that
    start from a non-equilibrium state)."""
    return amp * _rng(seed).uniform(-1.0, 1.0, size=(Q, N))
