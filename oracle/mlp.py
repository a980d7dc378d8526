"""Learned signal-to-parameter matcher (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper's related work (Section I) cites replacing dictionary matching by
a fully connected network that maps a fingerprint to its tissue parameters.
This module writes out the plain definitions the GPU learned matcher must
reproduce: a multilayer perceptron with GELU hidden units, its loss and its
gradient by the chain rule, and one Adam step (Kingma and Ba, 2015), all in
float64, with loops over layers only.

Model: x [B, 20] (the K = 10 complex subspace coefficients of a fingerprint
divided by their norm, as (Re, Im) pairs) -> 3 hidden layers of 256 GELU
units -> 3 outputs (normalised log T1, log T2 and PD per unit input norm).
Parameters are packed layer by layer as W_l [out][in] row-major, then b_l
[out] (the layout of the device library).

GELU(z) = z Phi(z) with Phi the standard normal CDF (the exact form with
erf, not the tanh approximation); GELU'(z) = Phi(z) + z phi(z).
Loss: L = 1 / (2 B) sum_{batch, outputs} (y - t)^2.
"""
from __future__ import annotations

import math

import numpy as np

SIZES = (20, 256, 256, 256, 3)

_erf = np.vectorize(math.erf, otypes=[np.float64])


def n_params(sizes=SIZES):
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unpack(theta, sizes=SIZES):
    """[(W [out, in], b [out])] views of the packed parameter vector."""
    theta = np.asarray(theta, np.float64)
    out, at = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = theta[at:at + o * i].reshape(o, i)
        at += o * i
        b = theta[at:at + o]
        at += o
        out.append((W, b))
    assert at == theta.size
    return out


def pack(layers):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def init(seed, sizes=SIZES):
    """He-style uniform initialisation: W ~ U(-sqrt(6 / in), sqrt(6 / in)), b = 0."""
    rng = np.random.default_rng(seed)
    layers = []
    for i, o in zip(sizes[:-1], sizes[1:]):
        lim = math.sqrt(6.0 / i)
        layers.append((rng.uniform(-lim, lim, (o, i)), np.zeros(o)))
    return pack(layers)


def gelu(z):
    return z * 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def round_bf16(v):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), via
    the float32 value: the upper 16 bits of its IEEE encoding after adding
    0x7fff plus the lowest kept bit.  Finite inputs only."""
    f = np.asarray(v, np.float64).astype(np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, sizes=SIZES, act_bf16=False):
    """(y [B, 3], cache): cache holds every layer's input and pre-activation.
    act_bf16: every layer's input rounded to bfloat16 (the tensor-core
    inference, whose operands are BF16)."""
    layers = unpack(theta, sizes)
    h = np.asarray(X, np.float64)
    cache = []
    for li, (W, b) in enumerate(layers):
        if act_bf16:
            h = round_bf16(h)
        z = h @ W.T + b
        cache.append((h, z))
        h = gelu(z) if li < len(layers) - 1 else z
    return h, cache


def loss(y, t):
    y, t = np.asarray(y, np.float64), np.asarray(t, np.float64)
    return float(np.sum((y - t) ** 2) / (2.0 * y.shape[0]))


def backward(theta, cache, y, t, sizes=SIZES):
    """Packed gradient dL/dtheta by the chain rule, layer by layer from the output."""
    layers = unpack(theta, sizes)
    B = y.shape[0]
    dz = (np.asarray(y, np.float64) - np.asarray(t, np.float64)) / B      # output layer is linear
    grads = [None] * len(layers)
    for li in range(len(layers) - 1, -1, -1):
        W, _ = layers[li]
        h, _ = cache[li]
        grads[li] = (dz.T @ h, dz.sum(axis=0))        # dL/dW = dz^T h, dL/db = sum over the batch
        if li > 0:
            dh = dz @ W                                # dL/d(input of layer li)
            dz = dh * gelu_grad(cache[li - 1][1])      # through the previous layer's GELU
    return pack(grads)


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step t >= 1): biased moments, bias correction, scaled step."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ---------------------------------------------------------------------------
# Inputs and targets of the learned matcher
# ---------------------------------------------------------------------------
def features(alpha):
    """(x [n, 2K], norm [n]): the subspace coefficients divided by their norm, as
    (Re, Im) pairs (an all-zero fingerprint gives x = 0, norm 0)."""
    alpha = np.asarray(alpha, np.complex128)
    nrm = np.linalg.norm(alpha, axis=1)
    a = np.where(nrm[:, None] > 0, alpha / np.where(nrm > 0, nrm, 1.0)[:, None], 0.0)
    return np.stack([a.real, a.imag], axis=-1).reshape(alpha.shape[0], -1), nrm


def encode(t1, t2, c, ranges):
    """Targets (u1, u2, u3): log T1 and log T2 mapped affinely from [log Tmin,
    log Tmax] to [-1, 1], and c / pd_scale with c = rho / ||alpha||.
    ranges = (t1min, t1max, t2min, t2max, pd_scale)."""
    t1min, t1max, t2min, t2max, pd_scale = ranges
    u1 = 2.0 * (np.log(t1) - math.log(t1min)) / (math.log(t1max) - math.log(t1min)) - 1.0
    u2 = 2.0 * (np.log(t2) - math.log(t2min)) / (math.log(t2max) - math.log(t2min)) - 1.0
    return np.stack([u1, u2, np.asarray(c, np.float64) / pd_scale], axis=-1)


def decode(y, norm, ranges):
    """(t1, t2, pd) from network outputs y [n, 3] and the inputs' norms."""
    t1min, t1max, t2min, t2max, pd_scale = ranges
    y = np.asarray(y, np.float64)
    t1 = np.exp(math.log(t1min) + 0.5 * (y[:, 0] + 1.0) * (math.log(t1max) - math.log(t1min)))
    t2 = np.exp(math.log(t2min) + 0.5 * (y[:, 1] + 1.0) * (math.log(t2max) - math.log(t2min)))
    return t1, t2, y[:, 2] * pd_scale * np.asarray(norm, np.float64)


def training_set(sig, t1t2, rho, snr_db, noise, phi, ranges):
    """(x [n, 2K], y [n, 3]) of noisy subspace fingerprints.

    sig [n, T]: the noiseless signals of the drawn (T1, T2); alpha = rho sig Phi
    (the compression of the recon, X = alpha Phi^H); complex noise of unit
    variance per coefficient, scaled to the drawn SNR of the coefficient
    vector: sigma^2 = ||alpha||^2 / K 10^(-snr / 10)."""
    K = phi.shape[1]
    a = np.asarray(rho, np.float64)[:, None] * (np.asarray(sig, np.complex128) @ np.asarray(phi, np.complex128))
    sigma = np.linalg.norm(a, axis=1) / math.sqrt(K) * 10.0 ** (-np.asarray(snr_db, np.float64) / 20.0)
    a = a + sigma[:, None] * np.asarray(noise, np.complex128)
    x, nrm = features(a)
    c = np.asarray(rho, np.float64) / nrm
    t1t2 = np.asarray(t1t2, np.float64)
    return x, encode(t1t2[:, 0], t1t2[:, 1], c, ranges)
