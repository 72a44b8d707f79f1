"""Pins of the oracle learned-collision pieces: orthonormal moment basis,
conservation projection, gradients against central finite differences,
bfloat16 rounding."""
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
