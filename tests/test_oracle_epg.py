"""Pins of the oracle's FISP simulation B(eta; theta) (Eq. 2-3).

The EPG recursion is checked against an independent isochromat simulation of
the Bloch equation (rotation matrices, relaxation and per-TR precession of
n_iso spins spread over one full dephasing cycle), which is exact when n_iso
exceeds the number of repetitions, and against closed forms."""
import math

import numpy as np
import pytest

from oracle import epg


def bloch_isochromats(t1, t2, fa_deg, tr, te, ti, n_iso=128, inversion=True):
    """Mean transverse magnetisation of n_iso isochromats, one per dephasing phase."""
    theta = 2 * np.pi * np.arange(n_iso) / n_iso
    M = np.zeros((n_iso, 3))
    M[:, 2] = 1.0

    def relax(tau):
        e1, e2 = math.exp(-tau / t1), math.exp(-tau / t2)
        M[:, 0] *= e2
        M[:, 1] *= e2
        M[:, 2] = M[:, 2] * e1 + (1.0 - e1)

    if inversion:
        M[:, 2] = -1.0
        relax(ti)
    out = []
    for a_deg, trt in zip(fa_deg, tr):
        a = math.radians(a_deg)
        R = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
        M[:] = M @ R.T
        relax(te)
        out.append(np.mean(M[:, 0] + 1j * M[:, 1]))
        relax(trt - te)
        c, s = np.cos(theta), np.sin(theta)
        mx, my = M[:, 0].copy(), M[:, 1].copy()
        M[:, 0] = c * mx - s * my
        M[:, 1] = s * mx + c * my
    return np.array(out)


@pytest.mark.parametrize("t1,t2", [(800.0, 80.0), (1500.0, 300.0), (300.0, 30.0), (4000.0, 500.0)])
def test_epg_equals_isochromat_bloch(t1, t2):
    rng = np.random.default_rng(7)
    T = 40
    fa = rng.uniform(5, 70, T)
    tr = rng.uniform(12, 15, T)
    s_epg = epg.fisp([t1], [t2], fa, tr, te=2.94, ti=20.0)[0]
    s_iso = bloch_isochromats(t1, t2, fa, tr, 2.94, 20.0, n_iso=128)
    np.testing.assert_allclose(s_epg, s_iso, rtol=0, atol=1e-12)


def test_single_pulse_closed_form():
    t1, t2, a = 900.0, 70.0, 35.0
    s = epg.fisp([t1], [t2], [a], [14.0], te=2.94, ti=20.0)[0, 0]
    expect = -1j * math.sin(math.radians(a)) * (1 - 2 * math.exp(-20.0 / t1)) * math.exp(-2.94 / t2)
    assert s == pytest.approx(expect, abs=1e-15)
    s = epg.fisp([t1], [t2], [a], [14.0], te=2.94, inversion=False)[0, 0]
    assert s == pytest.approx(-1j * math.sin(math.radians(a)) * math.exp(-2.94 / t2), abs=1e-15)


def test_saturation_recovery_closed_form():
    # 90 deg pulses with TR >> T2: no transverse memory, Z recovers from 0 each TR
    t1, t2, T, TR = 700.0, 8.0, 6, 1500.0
    s = epg.fisp([t1], [t2], [90.0] * T, [TR] * T, te=2.94, ti=20.0)[0]
    e2te = math.exp(-2.94 / t2)
    assert s[0] == pytest.approx(-1j * (1 - 2 * math.exp(-20.0 / t1)) * e2te, abs=1e-14)
    for n in range(1, T):
        assert s[n] == pytest.approx(-1j * (1 - math.exp(-TR / t1)) * e2te, abs=1e-14)


def test_no_relaxation_second_pulse():
    # T1, T2 -> infinity: S_1 = -i sin a, S_2 = -i sin a cos a (dephased F cannot refocus yet)
    a = 40.0
    s = epg.fisp([1e30], [1e30], [a, a], [10.0, 10.0], te=2.94, inversion=False)[0]
    sa, ca = math.sin(math.radians(a)), math.cos(math.radians(a))
    assert s[0] == pytest.approx(-1j * sa, abs=1e-14)
    assert s[1] == pytest.approx(-1j * sa * ca, abs=1e-14)


def test_pd_one_and_vectorised_over_atoms():
    fa = np.linspace(5, 60, 30)
    tr = np.full(30, 13.0)
    many = epg.fisp([500.0, 1200.0], [50.0, 100.0], fa, tr)
    one = epg.fisp([1200.0], [100.0], fa, tr)
    np.testing.assert_allclose(many[1], one[0], rtol=0, atol=0)
    assert np.all(np.abs(many) <= 1.0 + 1e-12)
