"""Pins of the oracle's SVT (Eq. 18), X update (Eq. 19) and metrics (Eq. 20-21)."""
import numpy as np
import pytest

from oracle import llr, metrics, patches


def _nuc(P):
    return np.linalg.svd(P, compute_uv=False).sum()


def test_svt_is_the_proximal_point():
    # SVT_{1/beta}(Q) minimises ||P||_* + beta/2 ||P - Q||^2 (Eq. 16)
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((9, 5)) + 1j * rng.standard_normal((9, 5))
    beta = 0.7
    P = llr.svt(Q, 1.0 / beta)
    f = lambda M: _nuc(M) + 0.5 * beta * np.sum(np.abs(M - Q) ** 2)
    f0 = f(P)
    for s in [1e-1, 1e-2, 1e-3]:
        for _ in range(30):
            E = rng.standard_normal(Q.shape) + 1j * rng.standard_normal(Q.shape)
            assert f(P + s * E) >= f0 - 1e-12


def test_svt_special_cases():
    rng = np.random.default_rng(1)
    Q = rng.standard_normal((8, 4)) + 1j * rng.standard_normal((8, 4))
    np.testing.assert_allclose(llr.svt(Q, 0.0), Q, atol=1e-12)
    np.testing.assert_allclose(llr.svt(Q, 1e6), 0.0, atol=0)
    u = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    v = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    R1 = np.outer(u, v.conj())
    s = np.linalg.norm(u) * np.linalg.norm(v)
    np.testing.assert_allclose(llr.svt(R1, 0.25 * s), 0.75 * R1, atol=1e-12)


def test_x_update_is_exact_minimiser():
    # brute force: minimise 1/(2 mu)||X - Z||^2 + lam2 beta/2 sum ||P_i - Q_i(X)||^2
    # as one stacked least-squares problem built from explicit patch selectors
    rng = np.random.default_rng(2)
    pg = patches.PatchGrid(6, 6, 3, 2)
    mu, lam2, beta = 1.0, 0.3, 0.5
    Z = rng.standard_normal((6, 6, 2)) + 1j * rng.standard_normal((6, 6, 2))
    P = rng.standard_normal((pg.count, 9, 2)) + 1j * rng.standard_normal((pg.count, 9, 2))
    rows, rhs = [np.eye(36) / np.sqrt(mu)], [Z.reshape(36, 2) / np.sqrt(mu)]
    for i in range(pg.count):
        y0, x0 = pg.origin(i)
        S = np.zeros((9, 36))
        for py in range(3):
            for px in range(3):
                S[py * 3 + px, (y0 + py) * 6 + (x0 + px)] = 1.0
        rows.append(np.sqrt(lam2 * beta) * S)
        rhs.append(np.sqrt(lam2 * beta) * P[i])
    A = np.vstack(rows)
    B = np.vstack(rhs)
    Xbf = np.linalg.lstsq(A, B, rcond=None)[0].reshape(6, 6, 2)
    X = llr.x_update(Z, pg.adjoint(P), pg.coverage(), mu, lam2, beta)
    np.testing.assert_allclose(X, Xbf, atol=1e-12)


def test_x_update_literal_equals_exact_without_overlap():
    rng = np.random.default_rng(3)
    pg = patches.PatchGrid(8, 8, 4, 4)
    Z = rng.standard_normal((8, 8, 2))
    P = rng.standard_normal((pg.count, 16, 2))
    a = llr.x_update(Z, pg.adjoint(P), pg.coverage(), 1.0, 0.1, 0.2)
    b = llr.x_update(Z, pg.adjoint(P), pg.coverage(), 1.0, 0.1, 0.2, literal=True)
    np.testing.assert_allclose(a, b, atol=1e-15)


def test_metrics_closed_forms():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((5, 5, 3)) + 1j * rng.standard_normal((5, 5, 3))
    assert metrics.snr(x, 1.01 * x) == pytest.approx(40.0, abs=1e-9)
    m = rng.uniform(1, 2, (4, 4))
    assert metrics.nmse(m, 1.1 * m) == pytest.approx(0.01, rel=1e-12)
    assert metrics.nrmse(m, 1.1 * m) == pytest.approx(0.1, rel=1e-12)
    mask = np.zeros((4, 4), bool)
    mask[0] = True
    m2 = m.copy()
    m2[1:] = 0
    assert metrics.nmse(m, np.where(mask, m * 1.2, 7.0), mask) == pytest.approx(0.04, rel=1e-12)
