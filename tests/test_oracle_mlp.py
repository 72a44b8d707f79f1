"""Pins of the oracle learned-collision pieces: orthonormal moment basis,
conservation projection, the network and the correction against a
hand-evaluated one-path network, gradients against central finite
differences, bfloat16 rounding."""
import math

import numpy as np
import pytest

from oracle.mlp import HIDDEN, MLP, bf16_round, conservation_basis, moment_basis, projector
from oracle.velocity_sets import velocity_set


@pytest.mark.parametrize("name", ["D2Q19", "D3Q45"])
def test_moment_basis_orthonormal(name):
    xi, w, _ = velocity_set(name)
    Phi = moment_basis(xi, w)
    assert Phi.shape == (len(w), len(w))
    assert np.abs((Phi * w) @ Phi.T - np.eye(len(w))).max() < 1e-10
    assert np.allclose(Phi[0], 1.0)                    # first basis function: the constant
    assert np.allclose(Phi[1], xi[:, 0]) and np.allclose(Phi[2], xi[:, 1])   # then xi (unit second moments)


@pytest.mark.parametrize("name", ["D2Q19", "D3Q45"])
def test_projection_conserves(name):
    xi, w, _ = velocity_set(name)
    P = projector(xi, w)
    C = conservation_basis(xi)
    o = np.random.default_rng(0).normal(size=(len(w), 7))
    d = w[:, None] * (P @ o)
    assert np.abs(C @ d).max() < 1e-13
    assert np.abs(P @ P - P).max() < 1e-12             # a projector
    assert np.abs((P @ o)[:, :1] - o[:, :1]).max() > 1e-3


def _net(Q, seed=0):
    r = np.random.default_rng(seed)
    return MLP(r.normal(0, 0.3, (HIDDEN, Q)), r.normal(0, 0.1, HIDDEN), r.normal(0, 0.2, (HIDDEN, HIDDEN)),
               r.normal(0, 0.1, HIDDEN), r.normal(0, 0.2, (Q, HIDDEN)), r.normal(0, 0.1, Q), np.ones(Q), 1.0)


@pytest.mark.parametrize("name", ["D2Q19", "D3Q45"])
def test_correction_one_path_network_closed_form(name):
    """A network with a single path from input to output has a closed form.
    Input: f^neq = alpha w Phi_k (a multiple of one basis function), so the
    moments are z = alpha e_k (orthonormal basis) and the scaled input is
    x_k = s alpha.  Layers: only W1[j0, k] = a, b1[j0] = beta1,
    W2[j1, j0] = b, b2[j1] = beta2 are non-zero, and W3[:, j1] = c v with
    v = Phi_k, b3 = beta3 (1, .., 1).  Then
      o = c tanh(b tanh(a s alpha + beta1) + beta2) v + beta3 1,
    the projection keeps v (the xi_0 xi_1 moment: by the reflection symmetry
    of the set it is weighted-orthogonal to 1, xi and |xi|^2) and removes the
    constant, so delta f_i = w_i sigma c tanh(b tanh(a s alpha + beta1) + beta2) v_i.
    A transposed basis, a dropped bias, a missing tanh, the output scaling
    without w_i or sigma, or no projection each break it."""
    xi, w, _ = velocity_set(name)
    Q = len(w)
    Phi = moment_basis(xi, w)
    P = projector(xi, w)
    D = xi.shape[1]
    k = 4 if D == 2 else 5                       # graded order: 1, xi (D), xi_0^2, xi_0 xi_1
    v = Phi[k]
    assert np.abs(v * np.sqrt((w * v * v).sum()) - v).max() < 1e-12      # unit weighted norm
    assert np.abs(v - xi[:, 0] * xi[:, 1] / np.sqrt((w * (xi[:, 0] * xi[:, 1]) ** 2).sum())).max() < 1e-12
    j0, j1 = 7, 11
    a, b, c, beta1, beta2, beta3, s, sigma = 0.8, -1.3, 0.6, 0.2, -0.1, 0.9, 2.5, 0.03
    W1 = np.zeros((HIDDEN, Q)); W1[j0, k] = a
    b1 = np.zeros(HIDDEN); b1[j0] = beta1
    W2 = np.zeros((HIDDEN, HIDDEN)); W2[j1, j0] = b
    b2 = np.zeros(HIDDEN); b2[j1] = beta2
    W3 = np.zeros((Q, HIDDEN)); W3[:, j1] = c * v
    b3 = np.full(Q, beta3)
    s_in = np.ones(Q); s_in[k] = s
    net = MLP(W1, b1, W2, b2, W3, b3, s_in, sigma)
    alphas = np.array([0.07, -0.15, 0.0])
    fneq = (w * v)[:, None] * alphas[None, :]
    df = net.correction(fneq, xi, w, Phi, P)
    for n, al in enumerate(alphas):
        T = math.tanh(b * math.tanh(a * s * al + beta1) + beta2)
        assert np.abs(df[:, n] - w * sigma * c * T * v).max() < 1e-15, (n, al)
    # the forward pass alone, on the same inputs: o = c T v + beta3
    o, (x, h1, h2) = net.forward((Phi @ fneq).T * s_in)
    for n, al in enumerate(alphas):
        T = math.tanh(b * math.tanh(a * s * al + beta1) + beta2)
        assert np.abs(o[n] - (c * T * v + beta3)).max() < 1e-14
        assert abs(h1[n, j0] - math.tanh(a * s * al + beta1)) < 1e-15
        assert np.abs(np.delete(h1[n], j0)).max() == 0.0


def test_gradients_finite_difference():
    xi, w, _ = velocity_set("D2Q19")
    Q = len(w)
    P = projector(xi, w)
    net = _net(Q)
    r = np.random.default_rng(1)
    x = r.normal(0, 1, (5, Q))
    y = r.normal(0, 1, (5, Q))
    _, grads = net.loss_and_grads(x, y, P, w)
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    for name, gr in zip(names, grads):
        A = getattr(net, name)
        for idx in [tuple(r.integers(0, s) for s in A.shape) for _ in range(6)]:
            h = 1e-6
            old = A[idx]
            A[idx] = old + h
            lp, _ = net.loss_and_grads(x, y, P, w)
            A[idx] = old - h
            lm, _ = net.loss_and_grads(x, y, P, w)
            A[idx] = old
            assert abs((lp - lm) / (2 * h) - gr[idx]) < 1e-7 * max(1.0, abs(gr[idx])), (name, idx)


def test_bf16_round():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.14159265, 1e-3])
    r = bf16_round(v)
    assert r[0] == 1.0 and r[1] == 1.0 + 2 ** -7 or r[1] == 1.0      # tie -> even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] + 3.140625) < 1e-12
    assert np.all(np.abs(r - v) <= np.abs(v) * 2 ** -8)
