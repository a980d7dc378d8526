"""Locally-low-rank steps (oracle, FP64).

Eq. 18: the P subproblem (Eq. 16) is solved patch by patch by singular value
thresholding: with Q_qi(X^n) = sum sigma U V^H,
    P_qi = sum max(sigma - 1/beta, 0) U V^H.
Eq. 19: the X subproblem (Eq. 17) is quadratic.  Eq. 19 prints
    X = (Z + mu lambda2 beta Q^*(P)) / (1 + mu lambda2 beta),
which is its exact minimiser only when Q^* Q = I.  With overlapping patches
Q^* Q = diag(cnt) (cnt = patches covering the voxel), and the exact
minimiser of Eq. 17 divides voxel-wise by (1 + mu lambda2 beta cnt); that is
the reading used, and ``literal=True`` reproduces the printed denominator.
"""
from __future__ import annotations

import numpy as np


def svt(P, tau):
    """Singular value thresholding of one matrix (numpy SVD)."""
    u, s, vh = np.linalg.svd(P, full_matrices=False)
    return (u * np.maximum(s - tau, 0.0)) @ vh


def svt_patches(patches, tau):
    return np.stack([svt(p, tau) for p in patches])


def nuclear_norms(patches):
    return np.array([np.linalg.svd(p, compute_uv=False).sum() for p in patches])


def x_update(Z, QtP, cnt, mu, lam2, beta, literal=False):
    """Eq. 19 (voxel-wise denominators unless ``literal``).  Z, QtP [ny, nx, T]."""
    c = mu * lam2 * beta
    den = (1.0 + c) if literal else (1.0 + c * cnt)[..., None]
    return (Z + c * QtP) / den
