"""FISP signal evolution B(eta; theta) by extended phase graphs (oracle, FP64).

Eq. 2 models a voxel as rho B(eta; theta) with B the Bloch-equation response
to the excitation train theta = (FA, TR, TE); Eq. 3 builds the dictionary
from B with PD = 1.  The paper names the FISP sequence with TE = 2.94 ms
(Sec. IV) but not the simulator; this oracle uses the extended-phase-graph
formalism (Weigel 2015) with the state vector (F+_k, F-_k, Z_k), k = 0..T:

per repetition t
  1. RF pulse of flip FA_t about x (phase 0):
        F+' = c^2 F+ + s^2 F- - i sin(a) Z
        F-' = s^2 F+ + c^2 F- + i sin(a) Z
        Z'  = -i/2 sin(a) F+ + i/2 sin(a) F- + cos(a) Z      (c, s = cos, sin of a/2)
  2. relaxation over TE: F *= E2, Z_k *= E1 (k >= 1), Z_0 = Z_0 E1 + 1 - E1
  3. signal: F+_0
  4. relaxation over TR_t - TE
  5. one full dephasing (unbalanced FISP gradient): F+_k <- F+_{k-1},
     F-_k <- F-_{k+1}, F+_0 <- conj(F-_0).
The magnetisation starts at equilibrium, is inverted (Z_0 = -1) and relaxes
for TI before the train.  All T+1 states are kept: no truncation.
"""
from __future__ import annotations

import numpy as np


def fisp(t1, t2, fa_deg, tr, te=2.94, ti=20.0, inversion=True):
    """Signals [M, T] complex128 for parameter arrays t1, t2 [M] (ms)."""
    t1 = np.atleast_1d(np.asarray(t1, dtype=np.float64))
    t2 = np.atleast_1d(np.asarray(t2, dtype=np.float64))
    fa = np.deg2rad(np.asarray(fa_deg, dtype=np.float64))
    tr = np.asarray(tr, dtype=np.float64)
    M, T = t1.shape[0], fa.shape[0]
    S = T + 2
    Fp = np.zeros((M, S), dtype=np.complex128)
    Fm = np.zeros((M, S), dtype=np.complex128)
    Z = np.zeros((M, S), dtype=np.complex128)

    def relax(tau):
        e1 = np.exp(-tau / t1)[:, None]
        e2 = np.exp(-tau / t2)[:, None]
        Fp[:] *= e2
        Fm[:] *= e2
        Z[:] *= e1
        Z[:, 0] += 1.0 - e1[:, 0]

    Z[:, 0] = -1.0 if inversion else 1.0
    if inversion:
        relax(ti)
    out = np.empty((M, T), dtype=np.complex128)
    for t in range(T):
        a = fa[t]
        c2, s2, sa, ca = np.cos(a / 2) ** 2, np.sin(a / 2) ** 2, np.sin(a), np.cos(a)
        fp = c2 * Fp + s2 * Fm - 1j * sa * Z
        fm = s2 * Fp + c2 * Fm + 1j * sa * Z
        z = -0.5j * sa * Fp + 0.5j * sa * Fm + ca * Z
        Fp[:], Fm[:], Z[:] = fp, fm, z
        relax(te)
        out[:, t] = Fp[:, 0]
        relax(tr[t] - te)
        Fp[:, 1:] = Fp[:, :-1].copy()
        Fm[:, :-1] = Fm[:, 1:].copy()
        Fm[:, -1] = 0.0
        Fp[:, 0] = np.conj(Fm[:, 0])
    return out
