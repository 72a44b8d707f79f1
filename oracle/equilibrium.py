"""Hermite equilibrium of order N = 4 (Sec. 3.1), FP64 oracle.  TEST INFRASTRUCTURE ONLY.

f_i^eq = w_i sum_{n=0}^{4} (1/n!) a^(n) : H^(n)(xi_i)       (Sec. 3.1, equilibrium)
g_i^eq = T (2 c_v - D) f_i^eq                               (Sec. 3.1, g-equilibrium)

The paper omits the coefficients a^(n) (it refers to Wilde et al. 2020 and
Shan et al. 2006).  They are the Hermite coefficients of the Maxwellian
M(rho, u, theta) about the reference state rho0 = T0 = 1 (Grad expansion):
  a0 = rho
  a1 = rho u
  a2 = rho (u u + (theta-1) delta)
  a3 = rho (u u u + (theta-1) sym(delta u))
  a4 = rho (u u u u + (theta-1) sym(delta u u) + (theta-1)^2 sym(delta delta))
where sym(.) sums over the distinct index placements.  H^(n) are the
probabilists' Hermite tensors.  Everything here is written with explicit
tensors and einsum contractions, node-vectorised: rho [N], u [N, D], T [N].
Abscissae are zeta_i = sqrt(T0) xi_i with T0 = 1.
"""
import numpy as np


def _delta(D):
    return np.eye(D)


def hermite_tensors(xi):
    """H^(0..4) evaluated at every abscissa: shapes [Q], [Q,D], [Q,D,D], ..."""
    Q, D = xi.shape
    d = _delta(D)
    H0 = np.ones(Q)
    H1 = xi.copy()
    H2 = np.einsum("qa,qb->qab", xi, xi) - d[None]
    xxx = np.einsum("qa,qb,qc->qabc", xi, xi, xi)
    sym_dx = (np.einsum("ab,qc->qabc", d, xi) + np.einsum("ac,qb->qabc", d, xi)
              + np.einsum("bc,qa->qabc", d, xi))
    H3 = xxx - sym_dx
    x4 = np.einsum("qa,qb,qc,qd->qabcd", xi, xi, xi, xi)
    sym_dxx = (np.einsum("ab,qc,qd->qabcd", d, xi, xi) + np.einsum("ac,qb,qd->qabcd", d, xi, xi)
               + np.einsum("ad,qb,qc->qabcd", d, xi, xi) + np.einsum("bc,qa,qd->qabcd", d, xi, xi)
               + np.einsum("bd,qa,qc->qabcd", d, xi, xi) + np.einsum("cd,qa,qb->qabcd", d, xi, xi))
    sym_dd = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
              + np.einsum("ad,bc->abcd", d, d))
    H4 = x4 - sym_dxx + sym_dd[None]
    return H0, H1, H2, H3, H4


def maxwell_coefficients(rho, u, T):
    """Hermite coefficients a^(0..4) of the Maxwellian, node-vectorised."""
    N, D = u.shape
    d = _delta(D)
    t = T - 1.0
    a0 = rho
    a1 = rho[:, None] * u
    uu = np.einsum("na,nb->nab", u, u)
    a2 = rho[:, None, None] * (uu + t[:, None, None] * d[None])
    uuu = np.einsum("na,nb,nc->nabc", u, u, u)
    sym_du = (np.einsum("ab,nc->nabc", d, u) + np.einsum("ac,nb->nabc", d, u)
              + np.einsum("bc,na->nabc", d, u))
    a3 = rho[:, None, None, None] * (uuu + t[:, None, None, None] * sym_du)
    u4 = np.einsum("na,nb,nc,nd->nabcd", u, u, u, u)
    sym_duu = (np.einsum("ab,nc,nd->nabcd", d, u, u) + np.einsum("ac,nb,nd->nabcd", d, u, u)
               + np.einsum("ad,nb,nc->nabcd", d, u, u) + np.einsum("bc,na,nd->nabcd", d, u, u)
               + np.einsum("bd,na,nc->nabcd", d, u, u) + np.einsum("cd,na,nb->nabcd", d, u, u))
    sym_dd = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
              + np.einsum("ad,bc->abcd", d, d))
    a4 = rho[:, None, None, None, None] * (u4 + t[:, None, None, None, None] * sym_duu
                                           + (t * t)[:, None, None, None, None] * sym_dd[None])
    return a0, a1, a2, a3, a4


def feq(rho, u, T, xi, w):
    """f^eq [Q, N] for node arrays rho [N], u [N, D], T [N]."""
    rho = np.asarray(rho, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    H = hermite_tensors(xi)
    a = maxwell_coefficients(rho, u, T)
    s = (np.einsum("n,q->qn", a[0], H[0])
         + np.einsum("na,qa->qn", a[1], H[1])
         + np.einsum("nab,qab->qn", a[2], H[2]) / 2.0
         + np.einsum("nabc,qabc->qn", a[3], H[3]) / 6.0
         + np.einsum("nabcd,qabcd->qn", a[4], H[4]) / 24.0)
    return w[:, None] * s


def geq(rho, u, T, xi, w, cv):
    D = xi.shape[1]
    return np.asarray(T)[None, :] * (2.0 * cv - D) * feq(rho, u, T, xi, w)


def maxwellian_moment(rho, u, T, mono):
    """Closed-form moment E[prod (u_d + sqrt(T) z_d)^k_d] * rho of the Maxwellian,
    from binomial expansion and 1D standard-normal moments (used as a pin)."""
    from math import comb
    from .velocity_sets import gaussian_moment_1d
    val = rho
    for d, k in enumerate(mono):
        s = 0.0
        for j in range(k + 1):
            s += comb(k, j) * u[d] ** (k - j) * T ** (j / 2.0) * gaussian_moment_1d(j)
        val = val * s
    return val
