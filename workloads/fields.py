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
        du, amp = ini["du"], ini["amp"]
        y = X[:, 1]
        u[:, 0] = 0.5 * du * np.tanh(-y / 1.0 * 2.0)
        env = np.exp(-(y / 2.0) ** 2)
        r = _rng(ini["seed"] if seed is None else seed).uniform(-1.0, 1.0, size=(N, D))
        u += amp * du * env[:, None] * r
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


def random_state_perturbation(Q, N, seed, amp):
    """Seeded uniform perturbation [Q, N] in [-amp, amp] (for parity tests that
    start from a non-equilibrium state)."""
    return amp * _rng(seed).uniform(-1.0, 1.0, size=(Q, N))
