"""Pins of the oracle equilibrium (Sec. 3.1): Maxwellian moments to order 4,
g-equilibrium, Hermite orthogonality."""
import math

import numpy as np
import pytest

from oracle.equilibrium import feq, geq, hermite_tensors, maxwellian_moment
from oracle.velocity_sets import monomials, velocity_set


@pytest.mark.parametrize("name", ["D2Q19", "D3Q45", "D2Q25"])
def test_maxwellian_moments_to_order_4(name):
    """Degree-9 rule x order-4 expansion: moments up to order 4 equal the
    Maxwellian's (closed form from 1D normal moments)."""
    xi, w, _ = velocity_set(name)
    D = xi.shape[1]
    rng = np.random.default_rng(3)
    for _ in range(4):
        rho = rng.uniform(0.5, 2.0)
        u = rng.uniform(-0.8, 0.8, size=D)
        T = rng.uniform(0.6, 1.6)
        f = feq(np.array([rho]), u[None], np.array([T]), xi, w)[:, 0]
        for m in monomials(D, 4):
            ref = maxwellian_moment(rho, u, T, m)
            got = (f * np.prod(xi ** np.array(m), axis=1)).sum()
            assert abs(got - ref) < 1e-11 * max(1.0, abs(ref)), (m, got, ref)


def test_fifth_moment_not_reproduced():
    """Order-4 truncation: an odd fifth-order moment differs from the Maxwellian."""
    xi, w, _ = velocity_set("D2Q19")
    rho, u, T = 1.0, np.array([0.5, 0.0]), 1.2
    f = feq(np.array([rho]), u[None], np.array([T]), xi, w)[:, 0]
    m = (5, 0)
    assert abs((f * xi[:, 0] ** 5).sum() - maxwellian_moment(rho, u, T, m)) > 1e-4


def test_rest_state_is_weights():
    xi, w, _ = velocity_set("D3Q45")
    f = feq(np.ones(1), np.zeros((1, 3)), np.ones(1), xi, w)[:, 0]
    assert np.abs(f - w).max() < 1e-15


def test_g_equilibrium_energy():
    """sum g^eq = (2 c_v - D) rho T and total energy 2 rho E = rho |u|^2 + 2 rho c_v T."""
    xi, w, _ = velocity_set("D2Q19")
    cv = 2.5
    rho, u, T = np.array([1.3]), np.array([[0.3, -0.4]]), np.array([1.1])
    f = feq(rho, u, T, xi, w)[:, 0]
    g = geq(rho, u, T, xi, w, cv)[:, 0]
    assert abs(g.sum() - (2 * cv - 2) * rho[0] * T[0]) < 1e-13
    e2 = ((xi ** 2).sum(1) * f).sum() + g.sum()
    assert abs(e2 - (rho[0] * (u ** 2).sum() + 2 * rho[0] * cv * T[0])) < 1e-13


def test_hermite_orthogonality():
    """sum_i w_i H^(m)_i H^(n)_i = 0 for m != n (m + n <= 9) and the textbook
    norm sum w H2_ab H2_cd = delta_ac delta_bd + delta_ad delta_bc."""
    xi, w, _ = velocity_set("D3Q45")
    H = hermite_tensors(xi)
    d = np.eye(3)
    assert abs(np.einsum("q,qa->a", w, H[1]).max()) < 1e-14
    assert np.abs(np.einsum("q,qab,qc->abc", w, H[2], H[1])).max() < 1e-13
    assert np.abs(np.einsum("q,qab,qcde->abcde", w, H[2], H[3])).max() < 1e-12
    n2 = np.einsum("q,qab,qcd->abcd", w, H[2], H[2])
    assert np.abs(n2 - (np.einsum("ac,bd->abcd", d, d) + np.einsum("ad,bc->abcd", d, d))).max() < 1e-12
