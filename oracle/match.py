"""Dictionary matching Phi_D of Eq. 5 (oracle, FP64).

For each voxel fingerprint x (one row of X):
    k   = argmax_m |<d_m, x>| / ||d_m||          (see reading below)
    eta = LUT[k]
    rho = max(Re <d_k, x> / ||d_k||^2, 0)
with <a, b> = sum_t conj(a_t) b_t.

Reading: Eq. 5 prints ||d_k||_2^2 in the argmax denominator, which makes the
score depend on each atom's scale and favours small-norm atoms; the argmax
here uses ||d_k||_2 (cosine similarity with unit-normalised atoms, the usual
MRF rule), and ``literal_norm2=True`` reproduces the printed form.  The PD
line uses ||d_k||^2 as printed.  Ties go to the lowest index, so an all-zero
fingerprint maps to atom 0 with PD 0.
"""
from __future__ import annotations

import numpy as np


def match(X, D, lut, atom_norm2=None, literal_norm2=False):
    """X [N, L], D [M, L], lut [M, 2] -> (idx [N], t1 [N], t2 [N], pd [N]).

    ``atom_norm2`` overrides ||d_m||^2 (used when D holds subspace-compressed
    atoms d_m Phi while the norms stay those of the full atoms).
    """
    X = np.asarray(X, dtype=np.complex128)
    D = np.asarray(D, dtype=np.complex128)
    n2 = np.sum(np.abs(D) ** 2, axis=1) if atom_norm2 is None else np.asarray(atom_norm2, np.float64)
    s = X @ D.conj().T                                    # [N, M]: <d_m, x_n>
    denom = n2 if literal_norm2 else np.sqrt(n2)
    score = np.abs(s) / denom[None, :]
    idx = np.argmax(score, axis=1)                        # first maximum = lowest index
    sk = s[np.arange(X.shape[0]), idx]
    pd = np.maximum(sk.real / n2[idx], 0.0)
    lut = np.asarray(lut, dtype=np.float64)
    return idx, lut[idx, 0], lut[idx, 1], pd


def scores(X, D, atom_norm2=None):
    """The full score matrix |<d_m, x_n>| / ||d_m|| [N, M] (for tie checks)."""
    X = np.asarray(X, dtype=np.complex128)
    D = np.asarray(D, dtype=np.complex128)
    n2 = np.sum(np.abs(D) ** 2, axis=1) if atom_norm2 is None else np.asarray(atom_norm2, np.float64)
    return np.abs(X @ D.conj().T) / np.sqrt(n2)[None, :]
