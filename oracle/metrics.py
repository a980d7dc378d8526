"""Quality metrics (oracle).

Eq. 20: SNR = -10 log10(||X - X_hat||_F^2 / ||X||_F^2).
Eq. 21: NMSE = ||m_hat - m||^2 / ||m||^2 for one parameter map; NRMSE is its
square root.  ``mask`` restricts both to the object (air has no T1/T2).
"""
from __future__ import annotations

import numpy as np


def snr(x, x_hat):
    x, x_hat = np.asarray(x), np.asarray(x_hat)
    return float(-10.0 * np.log10(np.sum(np.abs(x - x_hat) ** 2) / np.sum(np.abs(x) ** 2)))


def nmse(m, m_hat, mask=None):
    m, m_hat = np.asarray(m, np.float64), np.asarray(m_hat, np.float64)
    if mask is not None:
        m, m_hat = m[mask], m_hat[mask]
    return float(np.sum((m_hat - m) ** 2) / np.sum(m ** 2))


def nrmse(m, m_hat, mask=None):
    return float(np.sqrt(nmse(m, m_hat, mask)))
