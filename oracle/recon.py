"""Algorithm 1 (MS-LLR reconstruction), oracle, FP64, full-frame data.

The MRF data X is held as [ny, nx, T] (all T frames), every operator is
applied literally:

  Z^n     = P_S(X^n - mu [A^*(A X^n - b) + lambda1 Q^*(Q(X^n) L^n)])   (Eq. 12)
  P^{n+1} = SVT_{1/beta}(Q_qi(X^n)) for every patch                    (Eq. 18)
  X^{n+1} = (Z^n + mu lambda2 beta Q^*(P^{n+1})) / (1 + mu lambda2 beta cnt)  (Eq. 19)
  cost(n) = 1/2 ||A X - b||^2 + lambda1 Tr(Q(X) L Q(X)^H) + lambda2 sum ||Q_qi(X)||_*
  stop if cost(n-1)/cost(n) - 1 < tol (tol > 0 only)
  M^{n+1} = Phi_D(X^{n+1});  L^{n+1} from M^{n+1};  lambda1 from max(L^{n+1})

Readings (the paper leaves these open):
* the problem is posed over X in S (Eq. 11, 13), so the initial iterate is
  placed in S: X^0 = P_S(A^* b);
* mu = 1 is a valid step only for ||A|| <= 1 and the SVT threshold 1/beta
  depends on the data scale; A is therefore used as A / a with a = ||A P_S||_2
  (power iteration), and the data are scaled by gamma so that the largest PD
  matched from X^0 is ``pd_target`` (100, the paper's PD scale);
* Algorithm 1 prints lambda1^n = lambda1^0 x max(L^n) "for a finer balance of
  the regularisation terms".  With mu = 1 the product makes the graph part of
  the Eq. 12 step exceed the stability bound (mu lambda1 ||Q^* Q L|| grows
  with max(L)^2 and reaches ~12 on a 10-nearest-patch graph; the cost then
  oscillates).  The reading used divides instead, lambda1 = lambda1^0 / max(L),
  which balances the term by normalising the Laplacian to a unit largest entry;
  ``literal_lam1=True`` reproduces the printed product.  lambda1 of the first
  iteration comes from L^0.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import graph, llr, match, nufft, patches


@dataclass
class Params:
    mu: float = 1.0
    lam1_0: float = 0.1
    lam2: float = 0.1
    beta: float = 0.2
    patch: int = 8
    stride: int = 4
    knn: int = 10
    power_iters: int = 20
    pd_target: float = 100.0
    a_norm: float = 0.0       # > 0: use this ||A P_S|| instead of estimating it
    x_scale: float = 0.0      # > 0: use this gamma instead of deriving it
    tol: float = 0.0          # > 0: enable the cost-ratio stopping rule
    literal_xupdate: bool = False
    literal_lam1: bool = False   # True: lambda1 = lambda1^0 * max(L) as printed


class MSLLR:
    def __init__(self, b, k, grid: nufft.KBGrid, phi, D, lut, params: Params):
        self.b = np.asarray(b, np.complex128)
        self.k = np.asarray(k, np.float64)
        self.grid = grid
        self.phi = np.asarray(phi, np.complex128)
        self.D = np.asarray(D, np.complex128)
        self.lut = np.asarray(lut, np.float64)
        self.p = params
        self.pg = patches.PatchGrid(grid.ny, grid.nx, params.patch, params.stride)
        self.cnt = self.pg.coverage()
        self.t1max, self.t2max = self.lut[:, 0].max(), self.lut[:, 1].max()
        self.cost, self.lam1_hist, self.sigma2_hist = [], [], []

    # --- operators ---------------------------------------------------------
    def A_raw(self, X):
        return nufft.kb_forward(np.moveaxis(X, -1, 0), self.k, self.grid)

    def AH_raw(self, y):
        return np.moveaxis(nufft.kb_adjoint(y, self.k, self.grid), 0, -1)

    def A(self, X):
        return self.A_raw(X) / self.a

    def AH(self, y):
        return self.AH_raw(y) / self.a

    def PS(self, X):
        return (X @ self.phi) @ self.phi.conj().T

    def opnorm(self):
        """||A P_S||_2 by power iteration on coefficient images [ny, nx, K]."""
        K = self.phi.shape[1]
        v = np.ones((self.grid.ny, self.grid.nx, K), np.complex128)
        v /= np.linalg.norm(v)
        lam = 0.0
        for _ in range(self.p.power_iters):
            w = self.AH_raw(self.A_raw(v @ self.phi.conj().T)) @ self.phi
            lam = float(np.real(np.vdot(v, w)))
            v = w / np.linalg.norm(w)
        return float(np.sqrt(lam))

    def match(self, X):
        idx, t1, t2, pd = match.match(X.reshape(-1, X.shape[-1]), self.D, self.lut)
        sh = X.shape[:2]
        return idx.reshape(sh), t1.reshape(sh), t2.reshape(sh), pd.reshape(sh)

    def update_graph(self):
        _, t1, t2, _ = self.maps
        self.L, s2 = graph.build(t1, t2, self.pg, self.p.knn, self.t1max, self.t2max)
        lmax = float(self.L.max())
        if self.p.literal_lam1:
            self.lam1 = self.p.lam1_0 * lmax
        else:
            self.lam1 = self.p.lam1_0 / lmax if lmax > 0 else 0.0
        self.sigma2_hist.append(s2)
        self.lam1_hist.append(self.lam1)

    # --- Algorithm 1 -------------------------------------------------------
    def init(self):
        self.a = self.p.a_norm if self.p.a_norm > 0 else self.opnorm()
        self.bs = self.b / self.a
        X0 = self.PS(self.AH(self.bs))
        idx, t1, t2, pd = self.match(X0)
        if self.p.x_scale > 0:
            self.gamma = self.p.x_scale
        else:
            self.gamma = self.p.pd_target / pd.max() if pd.max() > 0 else 1.0
        self.X = X0 * self.gamma
        self.bs = self.bs * self.gamma
        self.maps = (idx, t1, t2, pd * self.gamma)
        self.update_graph()
        return self

    def objective(self, X):
        r = self.A(X) - self.bs
        data = 0.5 * float(np.sum(np.abs(r) ** 2))
        ms = graph.trace_term(X, self.L, self.pg)
        llr_ = float(llr.nuclear_norms(self.pg.extract(X)).sum())
        return data + self.lam1 * ms + self.p.lam2 * llr_

    def gradient(self, X):
        """The bracket of Eq. 12: A^*(A X - b) + lambda1 Q^*(Q(X) L), with L and
        lambda1 of the current pass."""
        r = self.A(X) - self.bs
        return self.AH(r) + self.lam1 * graph.graph_term(X, self.L, self.pg)

    def z_step(self, X):
        """Eq. 12: Z = P_S(X - mu [gradient])."""
        return self.PS(X - self.p.mu * self.gradient(X))

    def iterate(self):
        """One pass of the loop body; returns False when the stopping rule fires."""
        p, X = self.p, self.X
        Z = self.z_step(X)
        P = llr.svt_patches(self.pg.extract(X), 1.0 / p.beta)
        self.X = llr.x_update(Z, self.pg.adjoint(P), self.cnt, p.mu, p.lam2, p.beta,
                              literal=p.literal_xupdate)
        self.cost.append(self.objective(self.X))
        if p.tol > 0 and len(self.cost) > 1 and self.cost[-2] / self.cost[-1] - 1.0 < p.tol:
            return False
        self.maps = self.match(self.X)
        self.update_graph()
        return True

    def run(self, iters):
        for _ in range(iters):
            if not self.iterate():
                break
        idx, t1, t2, pd = self.maps
        return idx, t1, t2, pd / self.gamma
