"""Pins of the oracle's acquisition operator (Eq. 1) against closed forms,
numpy's FFT on a Cartesian special case, adjointness and the KB kernel's
error bound."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kb, nufft


def _rand(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_beatty_beta_values():
    # beta = pi sqrt((W/os)^2 (os - 1/2)^2 - 0.8): 8.996 (W=4), 13.855 (W=6) at os=2
    assert kb.beatty_beta(4, 2) == pytest.approx(8.99615, abs=1e-5)
    assert kb.beatty_beta(6, 2) == pytest.approx(13.85510, abs=1e-4)


@pytest.mark.parametrize("width", [4, 6])
def test_psi_hat_matches_quadrature(width):
    beta = kb.beatty_beta(width, 2)
    for f in [0.0, 0.05, 0.1, 0.2, 0.25, 0.4]:
        val, _ = integrate.quad(lambda u: kb.psi(u, width, beta) * math.cos(2 * math.pi * f * u),
                                -width / 2, width / 2, epsabs=1e-12, epsrel=1e-12, limit=200)
        assert kb.psi_hat(np.array([f]), width, beta)[0] == pytest.approx(val, rel=1e-9)


def test_taps_are_w_nearest_nodes():
    u = np.array([3.3, -0.5, 7.0, 0.0, 511.9])
    m = kb.taps(u, 4)
    assert m.shape == (5, 4)
    assert np.all(np.abs(u[:, None] - m) <= 2.0)
    np.testing.assert_array_equal(m[0], [2, 3, 4, 5])


def test_nudft_delta_is_phase_ramp():
    rng = np.random.default_rng(0)
    ny, nx = 12, 16
    x = np.zeros((1, ny, nx), complex)
    y0, x0 = 3, 5                      # array index; centred coordinate = index - n/2
    x[0, y0, x0] = 2.0 - 1.0j
    k = rng.uniform(-np.pi, np.pi, (1, 40, 2))
    y = nufft.nudft_forward(x, k)
    expect = (2.0 - 1.0j) * np.exp(-1j * (k[0, :, 0] * (x0 - nx // 2) + k[0, :, 1] * (y0 - ny // 2)))
    np.testing.assert_allclose(y[0], expect, rtol=1e-13, atol=1e-13)


def test_nudft_on_cartesian_grid_is_fft():
    rng = np.random.default_rng(1)
    n = 8
    x = _rand(rng, 1, n, n)
    m = np.arange(n) - n // 2
    my, mx = np.meshgrid(m, m, indexing="ij")
    k = np.stack([2 * np.pi * mx.ravel() / n, 2 * np.pi * my.ravel() / n], -1)[None]
    y = nufft.nudft_forward(x, k)[0].reshape(n, n)
    F = np.fft.fft2(x[0])
    # centred coordinates shift the phase by (-1)^(mx + my)
    expect = F[my % n, mx % n] * (-1.0) ** (mx + my)
    np.testing.assert_allclose(y, expect, rtol=1e-11, atol=1e-11)


def test_nudft_adjointness():
    rng = np.random.default_rng(2)
    x = _rand(rng, 3, 10, 14)
    k = rng.uniform(-np.pi, np.pi, (3, 50, 2))
    r = _rand(rng, 3, 50)
    lhs = np.vdot(nufft.nudft_forward(x, k), r)
    rhs = np.vdot(x, nufft.nudft_adjoint(r, k, 10, 14))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("width,bound", [(4, 2e-3), (6, 1e-4)])
def test_kb_forward_within_kernel_bound(width, bound):
    rng = np.random.default_rng(3)
    n = 24
    x = _rand(rng, 2, n, n)
    k = rng.uniform(-np.pi, np.pi, (2, 300, 2))
    g = nufft.KBGrid(n, n, os=2, width=width)
    y0 = nufft.nudft_forward(x, k)
    y1 = nufft.kb_forward(x, k, g)
    assert np.linalg.norm(y1 - y0) / np.linalg.norm(y0) < bound


@pytest.mark.parametrize("width,bound", [(4, 2e-3), (6, 1e-4)])
def test_kb_adjoint_within_kernel_bound(width, bound):
    rng = np.random.default_rng(4)
    n = 20
    r = _rand(rng, 2, 256)
    k = rng.uniform(-np.pi, np.pi, (2, 256, 2))
    g = nufft.KBGrid(n, n, os=2, width=width)
    x0 = nufft.nudft_adjoint(r, k, n, n)
    x1 = nufft.kb_adjoint(r, k, g)
    assert np.linalg.norm(x1 - x0) / np.linalg.norm(x0) < bound


def test_kb_adjointness():
    rng = np.random.default_rng(5)
    g = nufft.KBGrid(16, 24, os=2, width=4)
    x = _rand(rng, 2, 16, 24)
    k = rng.uniform(-np.pi, np.pi, (2, 120, 2))
    r = _rand(rng, 2, 120)
    lhs = np.vdot(nufft.kb_forward(x, k, g), r)
    rhs = np.vdot(x, nufft.kb_adjoint(r, k, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_kb_edge_samples_wrap():
    # samples at the band edge (k = -pi) and exactly on grid nodes still agree with the NUDFT
    rng = np.random.default_rng(6)
    n = 16
    x = _rand(rng, 1, n, n)
    k = np.array([[[-np.pi, -np.pi], [-np.pi, 0.0], [0.0, 0.0], [np.pi / 2, -np.pi / 4],
                   [2 * np.pi * 3 / 32, 2 * np.pi * 5 / 32]]])
    g = nufft.KBGrid(n, n, os=2, width=6)
    np.testing.assert_allclose(nufft.kb_forward(x, k, g), nufft.nudft_forward(x, k),
                               rtol=0, atol=2e-4 * np.abs(x).sum())
