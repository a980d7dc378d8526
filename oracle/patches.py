"""Patch extraction Q_q, Casorati Q and its adjoint Q^* (oracle).

Sec. III-A: Q_q(X) extracts the p x p x L patch at spatial location q; Q(X)
arranges all patches as the columns of a Casorati matrix; Q^* is the adjoint
(scatter-add of each patch back to its location).  The patch stride is printed
garbled ("s = p|2"); with the paper's own p = 11, s = 5 (Sec. III-D) it reads
s = floor(p / 2), and any stride can be passed here.  Patch origins along one
axis are 0, s, 2s, ... <= n - p, plus n - p when (n - p) is not a multiple of
s, so that every voxel is covered.

Layout: images are [ny, nx, T] (one fingerprint per voxel along the last
axis); patch i has origin (oy[i // nox], ox[i % nox]); a patch is stored as
[p*p, T] with row index py * p + px.
"""
from __future__ import annotations

import numpy as np


def origins(n: int, p: int, s: int):
    o = list(range(0, n - p + 1, s))
    if o[-1] != n - p:
        o.append(n - p)
    return np.asarray(o, dtype=np.int64)


class PatchGrid:
    def __init__(self, ny, nx, p, s):
        self.ny, self.nx, self.p, self.s = ny, nx, p, s
        self.oy, self.ox = origins(ny, p, s), origins(nx, p, s)
        self.count = len(self.oy) * len(self.ox)

    def origin(self, i):
        return self.oy[i // len(self.ox)], self.ox[i % len(self.ox)]

    def extract(self, img):
        """Q(X): img [ny, nx, T] -> patches [Np, p*p, T]."""
        p = self.p
        out = np.empty((self.count, p * p) + img.shape[2:], dtype=img.dtype)
        for i in range(self.count):
            y0, x0 = self.origin(i)
            out[i] = img[y0:y0 + p, x0:x0 + p].reshape((p * p,) + img.shape[2:])
        return out

    def adjoint(self, patches):
        """Q^*: patches [Np, p*p, T] -> img [ny, nx, T] (scatter-add)."""
        p = self.p
        img = np.zeros((self.ny, self.nx) + patches.shape[2:], dtype=patches.dtype)
        for i in range(self.count):
            y0, x0 = self.origin(i)
            img[y0:y0 + p, x0:x0 + p] += patches[i].reshape((p, p) + patches.shape[2:])
        return img

    def coverage(self):
        """Number of patches covering each voxel: Q^*(Q(1))."""
        return self.adjoint(self.extract(np.ones((self.ny, self.nx, 1))))[..., 0]
