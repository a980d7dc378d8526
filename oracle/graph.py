"""Parameter-manifold patch graph and Laplacian (oracle, FP64).

Eq. 7: w_ij = exp(-||Q_qi(M) - Q_qj(M)||_F^2 / sigma^2), distances taken
between patches of the matched parameter maps M, not of the fingerprints.
Eq. 9-10: L = D - W with D the diagonal degree matrix D_ii = sum_j w_ij.
Eq. 8-9: J_MS(X) = Tr(Q(X) L Q(X)^H); its gradient term in Eq. 12 is
Q^*(Q(X) L).

Readings where the paper is silent:
* features: each voxel contributes (T1 / T1max, T2 / T2max), the maxima
  taken over the dictionary's look-up table, so both maps weigh alike; the
  ratios are rounded (half to even) to 12-bit fixed point, q = rint(4096 T /
  Tmax), and squared distances are summed exactly in integers.  Matched maps
  are piecewise constant, so many patch distances tie exactly; exact integer
  distances make every device break those ties the same way (lowest index).
  12 bits resolve T1 to ~1 ms at 4000 ms, finer than any dictionary grid;
* graph: each patch keeps its k nearest patches (self excluded, ties to the
  lower index) and W = (K + K^T) / 2 with K_ij = w_ij on those edges, which
  makes W symmetric as Eq. 10 requires (Eq. 9 prints the dense graph);
* sigma^2 (never given): the median of the non-zero squared kNN distances,
  1 when all are zero;
* max(L) in the lambda_1 update of Algorithm 1: the largest entry of L, which
  is the largest degree.
"""
from __future__ import annotations

import numpy as np


QSCALE = 4096          # fixed-point scale of the features


def features(t1map, t2map, grid, t1max, t2max):
    """Integer patch vectors [Np, 2 p^2] (fixed point of T / Tmax) from maps [ny, nx]."""
    m = np.stack([np.rint(np.asarray(t1map, np.float64) / float(t1max) * QSCALE),
                  np.rint(np.asarray(t2map, np.float64) / float(t2max) * QSCALE)], axis=-1)
    return grid.extract(m.astype(np.int64)).reshape(grid.count, -1)


def knn(F, k):
    """(nbr [Np, k] int, d2 [Np, k]) of the k nearest rows, self excluded.

    Integer features give exact integer distances; float features are summed in
    float64."""
    F = np.asarray(F)
    exact = np.issubdtype(F.dtype, np.integer)
    F = F.astype(np.int64 if exact else np.float64)
    n = F.shape[0]
    nbr = np.empty((n, k), dtype=np.int64)
    d2 = np.empty((n, k), dtype=F.dtype)
    for i in range(n):
        di = np.sum((F - F[i]) ** 2, axis=1)
        if exact:
            di[i] = np.iinfo(np.int64).max
        else:
            di[i] = np.inf
        order = np.argsort(di, kind="stable")[:k]
        nbr[i], d2[i] = order, di[order]
    return nbr, d2


def sigma2(d2):
    nz = d2[d2 > 0]
    return float(np.median(nz)) if nz.size else 1.0


def adjacency(nbr, d2, s2):
    """W = (K + K^T)/2 with K_ij = exp(-d2_ij / sigma^2) on the kNN edges."""
    n = nbr.shape[0]
    K = np.zeros((n, n))
    for i in range(n):
        K[i, nbr[i]] = np.exp(-d2[i] / s2)
    return 0.5 * (K + K.T)


def laplacian(W):
    """L = D - W (Eq. 9), D_ii = sum_j W_ij."""
    W = np.asarray(W, np.float64)
    return np.diag(W.sum(axis=1)) - W


def build(t1map, t2map, grid, k, t1max, t2max):
    """Laplacian [Np, Np] of the kNN patch graph of the maps, and sigma^2.

    Distances are reported in units of (T / Tmax)^2 (integer distance / 4096^2)."""
    F = features(t1map, t2map, grid, t1max, t2max)
    nbr, d2i = knn(F, k)
    d2 = d2i.astype(np.float64) / float(QSCALE * QSCALE)
    s2 = sigma2(d2)
    return laplacian(adjacency(nbr, d2, s2)), s2


def graph_term(img, L, grid):
    """Q^*(Q(X) L) for X as [ny, nx, T]: column j of Q(X)L is sum_i Q_i L_ij."""
    Qx = grid.extract(img)                                   # [Np, p^2, T]
    QL = np.einsum("ipt,ij->jpt", Qx, L)
    return grid.adjoint(QL)


def trace_term(img, L, grid):
    """Tr(Q(X) L Q(X)^H) = sum_ij L_ij <Q_j, Q_i> (real for symmetric real L)."""
    Qx = grid.extract(img).reshape(grid.count, -1)
    G = Qx.conj() @ Qx.T                                     # G_ij = <Q_i, Q_j>
    return float(np.real(np.sum(L * G)))
