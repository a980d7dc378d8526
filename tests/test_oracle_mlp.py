"""Pins of the learned-matcher oracle (oracle/mlp.py) to facts outside it.

* GELU against its closed-form values (GELU(0) = 0, GELU(z) -> z, -> 0 in the
  tails, GELU(1) = Phi(1)) and its derivative against central differences.
* The backward pass against central finite differences of the loss, on a
  small network (every parameter) and on the full 20-256-256-256-3 network
  (a random sample of parameters in every layer and every bias).
* The forward pass against an explicit per-unit loop on a tiny network.
* One Adam step against its closed form at t = 1 (the first step moves
  every parameter by lr sign(g) up to eps).
"""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_forms_and_derivative():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    phi1 = 0.5 * (1 + math.erf(1 / math.sqrt(2)))
    assert abs(mlp.gelu(np.array([1.0]))[0] - phi1) < 1e-15
    assert abs(mlp.gelu(np.array([12.0]))[0] - 12.0) < 1e-12
    assert abs(mlp.gelu(np.array([-12.0]))[0]) < 1e-12
    z = np.linspace(-4, 4, 33)
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(z), fd, atol=1e-8)


def _fd_check(theta, X, T, sizes, idx, h=1e-6, rtol=1e-6):
    y, cache = mlp.forward(theta, X, sizes)
    g = mlp.backward(theta, cache, y, T, sizes)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss(mlp.forward(tp, X, sizes)[0], T) - mlp.loss(mlp.forward(tm, X, sizes)[0], T)) / (2 * h)
        assert abs(g[i] - fd) <= rtol * max(1.0, abs(fd)) + 1e-9, (i, g[i], fd)


def test_backward_matches_finite_differences_small_network():
    sizes = (5, 7, 6, 4, 3)
    rng = np.random.default_rng(0)
    theta = mlp.init(1, sizes) + 0.1 * rng.standard_normal(mlp.n_params(sizes))
    X = rng.standard_normal((9, 5))
    T = rng.standard_normal((9, 3))
    _fd_check(theta, X, T, sizes, range(mlp.n_params(sizes)))


def test_backward_matches_finite_differences_full_network():
    rng = np.random.default_rng(2)
    theta = mlp.init(3)
    theta += 0.01 * rng.standard_normal(theta.size)          # non-zero biases
    X = rng.standard_normal((6, 20))
    T = rng.standard_normal((6, 3))
    # a sample of weights and biases of every layer
    idx, at = [], 0
    for i, o in zip(mlp.SIZES[:-1], mlp.SIZES[1:]):
        idx += list(at + rng.choice(o * i, 6, replace=False)) + list(at + o * i + rng.choice(o, 3, replace=False))
        at += o * i + o
    _fd_check(theta, X, T, mlp.SIZES, idx, h=1e-5, rtol=1e-5)


def test_forward_matches_explicit_unit_loop():
    sizes = (3, 4, 2)
    rng = np.random.default_rng(4)
    theta = rng.standard_normal(mlp.n_params(sizes))
    x = rng.standard_normal(3)
    (W1, b1), (W2, b2) = mlp.unpack(theta, sizes)
    hidden = []
    for u in range(4):
        z = b1[u] + sum(W1[u, k] * x[k] for k in range(3))
        hidden.append(z * 0.5 * (1 + math.erf(z / math.sqrt(2))))
    out = [b2[o] + sum(W2[o, u] * hidden[u] for u in range(4)) for o in range(2)]
    np.testing.assert_allclose(mlp.forward(theta, x[None], sizes)[0][0], out, rtol=1e-14)


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(5)
    theta = rng.standard_normal(50)
    g = rng.standard_normal(50)
    new, m, v = mlp.adam_step(theta, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    # at t = 1, mhat = g and vhat = g^2, so the step is lr g / (|g| + eps)
    np.testing.assert_allclose(new, theta - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)


def test_features_targets_and_decoding():
    rng = np.random.default_rng(6)
    a = rng.standard_normal((40, 10)) + 1j * rng.standard_normal((40, 10))
    a[3] = 0
    x, nrm = mlp.features(a)
    assert x.shape == (40, 20)
    np.testing.assert_allclose(np.linalg.norm(np.delete(x, 3, 0), axis=1), 1.0, rtol=1e-14)
    assert np.all(x[3] == 0) and nrm[3] == 0
    np.testing.assert_allclose(x[0, 0::2] + 1j * x[0, 1::2], a[0] / np.linalg.norm(a[0]), rtol=1e-14)
    ranges = (100.0, 4000.0, 10.0, 500.0, 0.3)
    t1 = np.array([100.0, 4000.0, 632.45553203]); t2 = np.array([10.0, 500.0, 70.71067812])
    y = mlp.encode(t1, t2, np.array([0.3, 0.6, 0.15]), ranges)
    np.testing.assert_allclose(y[:2, :2], [[-1, -1], [1, 1]], atol=1e-14)      # range ends
    np.testing.assert_allclose(y[2, :2], [0.0, 0.0], atol=1e-8)               # geometric midpoints
    d1, d2, pd = mlp.decode(y, np.array([1.0, 2.0, 4.0]), ranges)
    np.testing.assert_allclose(d1, t1, rtol=1e-12)
    np.testing.assert_allclose(d2, t2, rtol=1e-12)
    np.testing.assert_allclose(pd, [0.3, 1.2, 0.6], rtol=1e-12)


def test_noiseless_training_targets_recover_pd():
    """At infinite SNR alpha = rho sig Phi, so rho / ||alpha|| = 1 / ||sig Phi||."""
    rng = np.random.default_rng(7)
    T, K, n = 30, 4, 12
    phi, _ = np.linalg.qr(rng.standard_normal((T, K)) + 1j * rng.standard_normal((T, K)))
    sig = rng.standard_normal((n, T)) + 1j * rng.standard_normal((n, T))
    rho = rng.uniform(0.5, 1.0, n)
    t1t2 = np.stack([np.full(n, 1000.0), np.full(n, 100.0)], -1)
    ranges = (100.0, 4000.0, 10.0, 500.0, 1.0)
    x, y = mlp.training_set(sig, t1t2, rho, np.full(n, 300.0), np.zeros((n, K)), phi, ranges)
    np.testing.assert_allclose(y[:, 2], 1.0 / np.linalg.norm(sig @ phi, axis=1), rtol=1e-12)
    a = sig @ phi
    np.testing.assert_allclose(x[:, 0::2] + 1j * x[:, 1::2], a / np.linalg.norm(a, axis=1)[:, None], rtol=1e-12)


def test_round_bf16():
    # exactly representable values (8 significant bits) are unchanged
    exact = np.array([1.0, -2.5, 0.15625, 3.0 * 2 ** -20, 255.0, -0.0])
    np.testing.assert_array_equal(mlp.round_bf16(exact), exact)
    # halfway cases go to the even neighbour: 1 + 2^-8 lies between 1 and 1 + 2^-7
    assert mlp.round_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert mlp.round_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    # otherwise the relative error is at most the unit roundoff 2^-8 (8 significant bits)
    v = np.random.default_rng(8).standard_normal(10000) * 10.0
    assert np.max(np.abs(mlp.round_bf16(v) - v) / np.abs(v)) <= 2 ** -8 * (1 + 1e-6)
