"""Kaiser-Bessel interpolation kernel (oracle, FP64).

The paper hands its NUFFT to a GPU library (Sec. III-D, Implementation
Details); the kernel here is the standard Kaiser-Bessel choice such libraries
use:

    psi(u) = I0(beta sqrt(1 - (2u/W)^2)),  |u| <= W/2   (grid units)

with Beatty et al. (2005)'s shape parameter
    beta = pi sqrt((W/os)^2 (os - 1/2)^2 - 0.8)
and its continuous Fourier transform (Jackson et al. 1991)
    psi_hat(f) = W sinh(sqrt(beta^2 - (pi W f)^2)) / sqrt(beta^2 - (pi W f)^2)
(the sin form when the root is imaginary), f in cycles per grid unit.
"""
from __future__ import annotations

import math

import numpy as np


def beatty_beta(width: int, os: float) -> float:
    return math.pi * math.sqrt((width / os) ** 2 * (os - 0.5) ** 2 - 0.8)


def psi(u, width: int, beta: float):
    """Kernel value at offset u (grid units); zero for |u| > W/2."""
    u = np.asarray(u, dtype=np.float64)
    arg = 1.0 - (2.0 * u / width) ** 2
    out = np.i0(beta * np.sqrt(np.clip(arg, 0.0, None)))
    return np.where(np.abs(u) <= width / 2.0, out, 0.0)


def psi_hat(f, width: int, beta: float):
    """Continuous Fourier transform of psi at frequency f (cycles / grid unit)."""
    f = np.asarray(f, dtype=np.float64)
    z2 = beta ** 2 - (math.pi * width * f) ** 2
    out = np.empty_like(f)
    pos = z2 > 0
    z = np.sqrt(np.abs(z2))
    out[pos] = width * np.sinh(z[pos]) / z[pos]
    neg = z2 < 0
    out[neg] = width * np.sin(z[neg]) / z[neg]
    out[z2 == 0] = width
    return out


def taps(u, width: int):
    """Integer grid nodes used for coordinate u: the W nodes floor(u - W/2) + 1 ...

    Returns an int64 array [..., W] (not yet wrapped modulo the grid size).
    """
    u = np.asarray(u, dtype=np.float64)
    m0 = np.floor(u - width / 2.0).astype(np.int64) + 1
    return m0[..., None] + np.arange(width)
