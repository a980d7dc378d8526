"""Dictionary D, look-up table and temporal subspace (oracle, FP64).

Eq. 3: d_m = B(eta_m; theta) with PD = 1, one row per (T1, T2) pair; the LUT
records the pair of each row.

The fingerprint-manifold projection P_S(X) = X d^dagger d (Eq. 14) needs an
orthonormal basis d "approximated by the precomputed dictionary".  The basis
here is the top-K right singular vectors of D (M x T): Phi = V[:, :K]
(T x K, orthonormal columns), so P_S(X) = X Phi Phi^H for X with one
fingerprint per row.
"""
from __future__ import annotations

import numpy as np

from . import epg


def simulate(lut, fa, tr, te=2.94, ti=20.0):
    """D [M, T] for lut [M, 2] = (T1, T2) in ms."""
    lut = np.asarray(lut, dtype=np.float64)
    return epg.fisp(lut[:, 0], lut[:, 1], fa, tr, te=te, ti=ti)


def subspace(D, rank):
    """Phi [T, K]: the top-K right singular vectors of D (numpy SVD, FP64)."""
    _, _, vh = np.linalg.svd(np.asarray(D, dtype=np.complex128), full_matrices=False)
    return vh[:rank].conj().T


def project(X, phi):
    """P_S(X) = X Phi Phi^H for fingerprints X [..., T] (Eq. 14)."""
    return (X @ phi) @ phi.conj().T
