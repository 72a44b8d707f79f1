"""Pins of the synthetic input generators (CPU): the solenoidal broadband
disturbance of the mixing layer (Sec. 4.4) and its envelope."""
import numpy as np
import pytest

from workloads.fields import spectral_broadband


def _grid(shape, h):
    ax = [np.arange(n) * hh - 0.5 * n * hh for n, hh in zip(shape, h)]
    G = np.meshgrid(*ax, indexing="ij")
    # nodes x fastest, as the meshes number them
    return np.stack([g.transpose(tuple(range(len(shape)))[::-1]).ravel() for g in G], axis=1)


def _spectral_div(X, u, shape, h):
    """Divergence of node field u on a uniform periodic grid, spectrally."""
    D = len(shape)
    div = np.zeros(shape)
    for d in range(D):
        f = u[:, d].reshape(shape[::-1]).transpose(tuple(range(D))[::-1])   # index (i0, i1[, i2])
        k = np.fft.fftfreq(shape[d]) * shape[d]
        sh = [1] * D
        sh[d] = -1
        ik = (2j * np.pi * k / shape[d]).reshape(sh)
        div += np.fft.ifftn(np.fft.fftn(f) * ik).real / h[d]
    return div


@pytest.mark.parametrize("shape,h", [((16, 12, 10), (0.5, 0.25, 0.4)), ((24, 20), (0.3, 0.2))])
def test_disturbance_is_solenoidal(shape, h):
    """With a flat envelope (dtheta0 -> infinity) the curl of the filtered
    potential has zero divergence to rounding (spectral derivatives commute)."""
    X = _grid(shape, h)
    u = spectral_broadband(X, 0.1, 1e9, seed=3)
    div = _spectral_div(X, u, shape, h)
    assert np.abs(div).max() < 1e-12 * np.abs(u).max() / min(h)
    assert abs(np.abs(u).max() - 0.1) < 1e-15


def test_disturbance_amplitude_envelope_and_seed():
    shape, h = (16, 64, 8), (0.5, 0.125, 0.5)
    X = _grid(shape, h)
    dth = 0.25
    u = spectral_broadband(X, 0.05, dth, seed=7)
    assert abs(np.abs(u).max() - 0.05) < 1e-15
    # confined to the shear layer: g(8 dtheta0) = exp(-16)
    far = np.abs(X[:, 1]) > 8 * dth
    assert np.abs(u[far]).max() < 1e-5 * 0.05
    near = np.abs(X[:, 1]) < dth
    assert np.abs(u[near]).max() > 0.1 * 0.05
    assert np.array_equal(u, spectral_broadband(X, 0.05, dth, seed=7))
    assert not np.allclose(u, spectral_broadband(X, 0.05, dth, seed=8))


def test_grid_required():
    X = np.random.default_rng(0).uniform(size=(50, 2))
    with pytest.raises(ValueError):
        spectral_broadband(X, 0.1, 0.25, seed=0)
