"""Velocity sets of the SLLBM (Sec. 3.2), FP64 oracle.  TEST INFRASTRUCTURE ONLY.

The paper uses cubature rules of quadrature degree 9 for the Gaussian weight
omega(xi) = (2 pi)^(-D/2) exp(-|xi|^2 / 2): D2Q19 and D3Q45 (Sec. 3.2), D2Q25
(product Gauss-Hermite, Sec. 3.2 / Sec. 4.1) and, for the classic-LBM special
case named in Sec. 2, D2Q9.  The abscissae of D2Q19 / D3Q45 are not printed in
the paper; the rules below are closed-form fully symmetric degree-9 rules:

  D2Q19  rest point, ring A at angles k*60 deg with r^2 = (48 - 8 sqrt15)/7,
         ring B at 30 + k*60 deg with r = 2 sqrt2, ring C at k*60 deg with
         r^2 = (48 + 8 sqrt15)/7.
  D3Q125 product of the 5-point Gauss-Hermite rule (nodes 0, +-sqrt(5 -+
         sqrt10), the roots of He_5), x fastest, then y, then z: the 3D
         member of the product family whose 2D member D2Q25 the paper uses;
         exact to degree 9 in each variable.
  D3Q45  rest point, shell A: icosahedron (cyclic perms of (0, +-phi, +-1))
         at radius sqrt3, shell B: dodecahedron ((+-1)^3 and cyclic perms of
         (0, +-1/phi, +-phi)) at radius 3, shell C: icosahedron of the same
         orientation as shell A (cyclic perms of (0, +-phi, +-1)) at radius
         sqrt15.

Here only the abscissae are stated; the weights are obtained by solving the
(linear) moment equations sum_i w_i xi_i^k = E_omega[xi^k] for all monomials of
degree <= 9, which is what "quadrature degree 9" means (Sec. 3.2).  Tests pin
the result against the moments, the closed-form weights and the symmetry.

Ordering (shared convention of the library's population layout): index 0 is
the rest velocity; inside every shell the first half are the representatives
listed below and the second half their negatives in the same order, so the
opposite of index k in a shell of n points is k + n/2 (mod n).
"""
import itertools
import math

import numpy as np

PHI = (1.0 + math.sqrt(5.0)) / 2.0


def gaussian_moment_1d(k):
    """E[xi^k] for the standard normal: 0 for odd k, (k-1)!! for even k."""
    if k % 2:
        return 0.0
    return float(np.prod(np.arange(k - 1, 0, -2))) if k > 0 else 1.0


def gaussian_moment(mono):
    """E_omega[prod_d xi_d^mono_d] for the D-dimensional standard normal."""
    return float(np.prod([gaussian_moment_1d(k) for k in mono]))


def monomials(D, degree):
    return [m for m in itertools.product(range(degree + 1), repeat=D) if sum(m) <= degree]


def _shell(reps, radius):
    reps = np.asarray(reps, dtype=np.float64)
    reps = reps / np.linalg.norm(reps, axis=1)[:, None] * radius
    return np.vstack([reps, -reps])


def _cyc(a, b):
    """Cyclic permutations of (0, a, b)."""
    return [(0.0, a, b), (b, 0.0, a), (a, b, 0.0)]


def abscissae(name):
    """Abscissae xi_i (Q x D) in the documented order."""
    if name == "D2Q9":
        s = math.sqrt(3.0)
        pts = [(0, 0), (s, 0), (0, s), (s, s), (-s, s), (-s, 0), (0, -s), (-s, -s), (s, -s)]
        return np.array(pts, dtype=np.float64)
    if name == "D2Q25":
        r1 = math.sqrt(5.0 - math.sqrt(10.0))
        r2 = math.sqrt(5.0 + math.sqrt(10.0))
        nodes = [0.0, r1, r2, -r1, -r2]
        return np.array([(a, b) for b in nodes for a in nodes], dtype=np.float64)
    if name == "D3Q125":
        r1 = math.sqrt(5.0 - math.sqrt(10.0))
        r2 = math.sqrt(5.0 + math.sqrt(10.0))
        nodes = [0.0, r1, r2, -r1, -r2]
        return np.array([(a, b, c) for c in nodes for b in nodes for a in nodes], dtype=np.float64)
    if name == "D2Q19":
        ra = math.sqrt((48.0 - 8.0 * math.sqrt(15.0)) / 7.0)
        rb = 2.0 * math.sqrt(2.0)
        rc = math.sqrt((48.0 + 8.0 * math.sqrt(15.0)) / 7.0)
        pts = [np.zeros((1, 2))]
        for r, a0 in ((ra, 0.0), (rb, math.pi / 6.0), (rc, 0.0)):
            ang = a0 + np.arange(6) * math.pi / 3.0
            pts.append(np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1))
        return np.vstack(pts)
    if name == "D3Q45":
        shell_a = _cyc(PHI, 1.0) + _cyc(-PHI, 1.0)
        shell_a = [shell_a[0], shell_a[3], shell_a[1], shell_a[4], shell_a[2], shell_a[5]]
        shell_b = [(1, 1, 1), (1, 1, -1), (1, -1, 1), (-1, 1, 1)]
        t = _cyc(1.0 / PHI, PHI) + _cyc(-1.0 / PHI, PHI)
        shell_b += [t[0], t[3], t[1], t[4], t[2], t[5]]
        shell_c = _cyc(PHI, 1.0) + _cyc(-PHI, 1.0)
        shell_c = [shell_c[0], shell_c[3], shell_c[1], shell_c[4], shell_c[2], shell_c[5]]
        return np.vstack([np.zeros((1, 3)),
                          _shell(shell_a, math.sqrt(3.0)),
                          _shell(shell_b, 3.0),
                          _shell(shell_c, math.sqrt(15.0))])
    raise ValueError(name)


def _orbits(name, xi):
    """Groups of indices that share one weight (the symmetry orbits)."""
    Q = len(xi)
    if name == "D2Q9":
        r2 = np.round((xi ** 2).sum(1), 9)
        return [np.nonzero(r2 == v)[0] for v in np.unique(r2)]
    if name in ("D2Q25", "D3Q125"):
        key = [tuple(sorted(np.round(np.abs(x), 9))) for x in xi]
        uniq = sorted(set(key))
        return [np.array([i for i in range(Q) if key[i] == u]) for u in uniq]
    if name == "D2Q19":
        return [np.array([0])] + [np.arange(1 + 6 * k, 7 + 6 * k) for k in range(3)]
    if name == "D3Q45":
        return [np.array([0]), np.arange(1, 13), np.arange(13, 33), np.arange(33, 45)]
    raise ValueError(name)


def velocity_set(name):
    """Return (xi [Q,D], w [Q], opp [Q]) with weights solved from the moment
    equations of the Gaussian weight (degree 9 for the cubature sets, degree 5
    for D2Q9)."""
    xi = abscissae(name)
    Q, D = xi.shape
    if name == "D3Q125":
        # a product rule: the 1D weights of the 5 Gauss-Hermite nodes solve
        # the 1D moment equations of degree 0 .. 4 (a Vandermonde system;
        # with the roots of He_5 as nodes the rule is then exact to degree
        # 9), and the 3D weight is the product over the coordinates.  (The
        # symmetric degree-9 equations in 3D do not fix its 10 orbit weights.)
        x = abscissae("D2Q25")[:5, 0]
        V = np.vander(x, 5, increasing=True).T
        w1 = np.linalg.solve(V, np.array([gaussian_moment_1d(k) for k in range(5)]))
        w = np.array([w1[i % 5] * w1[(i // 5) % 5] * w1[i // 25] for i in range(Q)])
        opp = np.array([int(np.argmin(np.abs(xi + xi[i]).sum(1))) for i in range(Q)])
        return xi, w, opp
    orbits = _orbits(name, xi)
    degree = 5 if name == "D2Q9" else 9
    mons = monomials(D, degree)
    A = np.zeros((len(mons), len(orbits)))
    b = np.zeros(len(mons))
    for r, m in enumerate(mons):
        val = np.prod(xi ** np.array(m), axis=1)
        for c, orb in enumerate(orbits):
            A[r, c] = val[orb].sum()
        b[r] = gaussian_moment(m)
    scale = 1.0 / np.maximum(1.0, np.abs(A).max(axis=1))
    As, bs = A * scale[:, None], b * scale
    wo, *_ = np.linalg.lstsq(As, bs, rcond=None)
    # one step of iterative refinement in the scaled system
    dw, *_ = np.linalg.lstsq(As, bs - As @ wo, rcond=None)
    wo = wo + dw
    w = np.zeros(Q)
    for c, orb in enumerate(orbits):
        w[orb] = wo[c]
    opp = np.array([int(np.argmin(np.abs(xi + xi[i]).sum(1))) for i in range(Q)])
    return xi, w, opp


def custom_set(xi, w):
    """A caller's set (xi [Q,D], w [Q]) with its opposites, for oracle cases
    of the library's SLLBM_VELSET_CUSTOM kind."""
    xi = np.asarray(xi, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    opp = np.array([int(np.argmin(np.abs(xi + xi[i]).sum(1))) for i in range(len(xi))])
    return xi, w, opp


def moment_error(xi, w, degree):
    """max over monomials of degree <= `degree` of |sum w xi^k - E[xi^k]|."""
    D = xi.shape[1]
    err = 0.0
    for m in monomials(D, degree):
        err = max(err, abs(float((w * np.prod(xi ** np.array(m), axis=1)).sum()) - gaussian_moment(m)))
    return err
