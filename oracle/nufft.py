"""Acquisition operator A = F_u (one coil, C = I) of Eq. 1 (oracle, FP64).

Image layout: x[..., ny, nx] with centred coordinates n = (nx - Nx/2,
ny - Ny/2).  A sample position is k = (kx, ky) in radians per voxel.

* ``nudft_forward`` / ``nudft_adjoint``: the exact non-uniform DFT,
      y_j = sum_n x_n exp(-i k_j . n),   x_n = sum_j y_j exp(+i k_j . n).
  No density compensation, no scaling: X^0 = A^* b literally (Algorithm 1).
* ``kb_forward`` / ``kb_adjoint``: the Kaiser-Bessel gridding approximation of
  the same operator, the computation a GPU NUFFT library performs
  (Sec. III-D):  deapodise by psi_hat, zero-pad to the os-times oversampled
  grid, FFT, and interpolate each sample from its W x W nearest grid nodes
  (periodic wrap).  The adjoint runs the transposed steps: spread, inverse FFT
  (unnormalised), crop, deapodise.
"""
from __future__ import annotations

import numpy as np

from . import kb


def _centred(n):
    return np.arange(n, dtype=np.float64) - n // 2


def nudft_forward(x, k):
    """x [T, ny, nx] complex, k [T, ns, 2] -> y [T, ns] (exact)."""
    x = np.asarray(x, dtype=np.complex128)
    T, ny, nx = x.shape
    cx, cy = _centred(nx), _centred(ny)
    y = np.empty(k.shape[:2], dtype=np.complex128)
    for t in range(T):
        ex = np.exp(-1j * np.outer(k[t, :, 0], cx))      # [ns, nx]
        ey = np.exp(-1j * np.outer(k[t, :, 1], cy))      # [ns, ny]
        y[t] = np.einsum("jy,yx,jx->j", ey, x[t], ex)
    return y


def nudft_adjoint(y, k, ny, nx):
    """y [T, ns], k [T, ns, 2] -> x [T, ny, nx] (exact adjoint of nudft_forward)."""
    y = np.asarray(y, dtype=np.complex128)
    T = y.shape[0]
    cx, cy = _centred(nx), _centred(ny)
    x = np.empty((T, ny, nx), dtype=np.complex128)
    for t in range(T):
        ex = np.exp(1j * np.outer(k[t, :, 0], cx))
        ey = np.exp(1j * np.outer(k[t, :, 1], cy))
        x[t] = np.einsum("j,jy,jx->yx", y[t], ey, ex)
    return x


class KBGrid:
    """Fixed parameters of the gridding NUFFT for one image size."""

    def __init__(self, ny, nx, os=2, width=4):
        self.ny, self.nx, self.os, self.width = ny, nx, os, width
        self.gy, self.gx = os * ny, os * nx
        self.beta = kb.beatty_beta(width, os)
        # deapodisation: psi_hat at the image's centred coordinates
        self.dx = kb.psi_hat(_centred(nx) / self.gx, width, self.beta)
        self.dy = kb.psi_hat(_centred(ny) / self.gy, width, self.beta)

    def grid_coords(self, k):
        """Sample positions in grid units: u = k G / (2 pi)."""
        return k[..., 0] * self.gx / (2 * np.pi), k[..., 1] * self.gy / (2 * np.pi)

    def weights(self, kt):
        """Interpolation nodes and weights of one frame's samples."""
        ux, uy = self.grid_coords(kt)
        mx = kb.taps(ux, self.width)                     # [ns, W]
        my = kb.taps(uy, self.width)
        wx = kb.psi(ux[:, None] - mx, self.width, self.beta)
        wy = kb.psi(uy[:, None] - my, self.width, self.beta)
        return mx % self.gx, my % self.gy, wx, wy

    def pad(self, img):
        """Place a centred [ny, nx] image on the [gy, gx] grid (index n mod G)."""
        g = np.zeros((self.gy, self.gx), dtype=np.complex128)
        iy = np.arange(self.ny) - self.ny // 2
        ix = np.arange(self.nx) - self.nx // 2
        g[np.ix_(iy % self.gy, ix % self.gx)] = img
        return g

    def crop(self, g):
        iy = np.arange(self.ny) - self.ny // 2
        ix = np.arange(self.nx) - self.nx // 2
        return g[np.ix_(iy % self.gy, ix % self.gx)]


def kb_forward(x, k, grid: KBGrid):
    """Gridding approximation of nudft_forward.  x [T, ny, nx], k [T, ns, 2]."""
    x = np.asarray(x, dtype=np.complex128)
    T = x.shape[0]
    y = np.empty(k.shape[:2], dtype=np.complex128)
    deapod = np.outer(grid.dy, grid.dx)
    for t in range(T):
        spectrum = np.fft.fft2(grid.pad(x[t] / deapod))
        mx, my, wx, wy = grid.weights(k[t])
        # y_j = sum_a sum_b wy[j,a] wx[j,b] G[my[j,a], mx[j,b]]
        vals = spectrum[my[:, :, None], mx[:, None, :]]
        y[t] = np.einsum("ja,jb,jab->j", wy, wx, vals)
    return y


def kb_adjoint(y, k, grid: KBGrid):
    """Exact adjoint of kb_forward.  y [T, ns] -> x [T, ny, nx]."""
    y = np.asarray(y, dtype=np.complex128)
    T = y.shape[0]
    x = np.empty((T, grid.ny, grid.nx), dtype=np.complex128)
    deapod = np.outer(grid.dy, grid.dx)
    for t in range(T):
        g = np.zeros((grid.gy, grid.gx), dtype=np.complex128)
        mx, my, wx, wy = grid.weights(k[t])
        contrib = wy[:, :, None] * wx[:, None, :] * y[t][:, None, None]
        np.add.at(g, (np.broadcast_to(my[:, :, None], contrib.shape),
                      np.broadcast_to(mx[:, None, :], contrib.shape)), contrib)
        img = np.fft.ifft2(g) * (grid.gy * grid.gx)   # unnormalised e^{+i} sum
        x[t] = grid.crop(img) / deapod
    return x
