"""Pins of the oracle velocity sets (Sec. 3.2): cubature degree, closed-form
weights, symmetry.  The weights are solved from moment equations inside the
oracle; the closed forms below are independent facts about the rules."""
import math

import numpy as np
import pytest

from oracle.velocity_sets import gaussian_moment, moment_error, monomials, velocity_set


@pytest.mark.parametrize("name,deg", [("D2Q19", 9), ("D3Q45", 9), ("D2Q25", 9), ("D2Q9", 5), ("D3Q125", 9)])
def test_exact_to_degree(name, deg):
    xi, w, opp = velocity_set(name)
    assert moment_error(xi, w, deg) < 1e-11
    assert (w > 0).all()
    assert abs(w.sum() - 1.0) < 1e-14


@pytest.mark.parametrize("name,deg", [("D2Q19", 10), ("D3Q45", 10), ("D2Q25", 10), ("D2Q9", 6), ("D3Q125", 10)])
def test_not_exact_beyond_degree(name, deg):
    """The rules are exactly of the stated degree (Sec. 3.2: N = 9), not more."""
    xi, w, _ = velocity_set(name)
    assert moment_error(xi, w, deg) > 1e-3


def test_sizes_match_paper():
    """Sec. 3.2: 19 points in 2D and 45 points in 3D for degree 9; D2Q25 product rule."""
    assert velocity_set("D2Q19")[0].shape == (19, 2)
    assert velocity_set("D3Q45")[0].shape == (45, 3)
    assert velocity_set("D2Q25")[0].shape == (25, 2)


def test_closed_form_weights():
    _, w, _ = velocity_set("D3Q45")
    assert np.allclose(w[0], 28 / 135, rtol=0, atol=1e-13)
    assert np.allclose(w[1:13], 25 / 432, rtol=0, atol=1e-13)
    assert np.allclose(w[13:33], 1 / 216, rtol=0, atol=1e-13)
    assert np.allclose(w[33:45], 1 / 2160, rtol=0, atol=1e-13)
    _, w, _ = velocity_set("D2Q19")
    assert abs(w[0] - 31 / 96) < 1e-13 and np.allclose(w[7:13], 1 / 128, atol=1e-13)
    # D2Q25 = tensor product of the 5-point Gauss-Hermite rule
    r10 = math.sqrt(10)
    w1 = {0: 8 / 15, 1: (7 + 2 * r10) / 60, 2: (7 - 2 * r10) / 60, 3: (7 + 2 * r10) / 60, 4: (7 - 2 * r10) / 60}
    _, w, _ = velocity_set("D2Q25")
    for i in range(25):
        assert abs(w[i] - w1[i % 5] * w1[i // 5]) < 1e-13
    _, w, _ = velocity_set("D2Q9")
    assert np.allclose(sorted(set(np.round(w, 12))), [1 / 36, 1 / 9, 4 / 9])


def test_gauss_hermite_nodes_are_roots_of_He5():
    xi, _, _ = velocity_set("D2Q25")
    x = np.unique(np.round(xi[:, 0], 12))
    he5 = x ** 5 - 10 * x ** 3 + 15 * x
    assert np.abs(he5).max() < 1e-10


@pytest.mark.parametrize("name", ["D2Q9", "D2Q19", "D2Q25", "D3Q45", "D3Q125"])
def test_opposites(name):
    xi, w, opp = velocity_set(name)
    assert np.abs(xi[opp] + xi).max() < 1e-14
    assert (opp[opp] == np.arange(len(xi))).all()
    assert np.allclose(w[opp], w)


def test_shell_radii():
    xi, _, _ = velocity_set("D3Q45")
    r2 = (xi ** 2).sum(1)
    assert np.allclose(r2[1:13], 3) and np.allclose(r2[13:33], 9) and np.allclose(r2[33:], 15)
    xi, _, _ = velocity_set("D2Q19")
    r2 = (xi ** 2).sum(1)
    assert np.allclose(r2[1:7], (48 - 8 * math.sqrt(15)) / 7) and np.allclose(r2[7:13], 8)


def test_second_moment_isotropy():
    """sum w xi_a xi_b = delta_ab (the lattice temperature T0 = 1)."""
    for name in ("D2Q19", "D3Q45", "D2Q25"):
        xi, w, _ = velocity_set(name)
        assert np.abs(np.einsum("q,qa,qb->ab", w, xi, xi) - np.eye(xi.shape[1])).max() < 1e-13


def test_d3q125_is_the_gauss_hermite_product():
    """D3Q125: every weight is the product of the three 1D 5-point
    Gauss-Hermite weights of its coordinates (closed form; the oracle solves
    the weights from the moment equations), nodes x fastest, then y, then z;
    each coordinate a root of He_5."""
    r10 = math.sqrt(10)
    r1, r2 = math.sqrt(5 - r10), math.sqrt(5 + r10)
    nodes = [0.0, r1, r2, -r1, -r2]
    w1 = [8 / 15, (7 + 2 * r10) / 60, (7 - 2 * r10) / 60, (7 + 2 * r10) / 60, (7 - 2 * r10) / 60]
    xi, w, _ = velocity_set("D3Q125")
    assert xi.shape == (125, 3)
    for i in range(125):
        a, b, c = i % 5, (i // 5) % 5, i // 25
        assert np.abs(xi[i] - [nodes[a], nodes[b], nodes[c]]).max() < 1e-15
        assert abs(w[i] - w1[a] * w1[b] * w1[c]) < 1e-14
    x = np.unique(np.round(xi.ravel(), 12))
    assert np.abs(x ** 5 - 10 * x ** 3 + 15 * x).max() < 1e-10
    # a product rule integrates x^8 y^8 z^8 exactly although its degree is 24
    assert abs(float((w * (xi ** 8).prod(1)).sum()) - 105.0 ** 3) < 1e-7 * 105.0 ** 3
