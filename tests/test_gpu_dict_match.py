"""GPU parity of the EPG dictionary (Eq. 2-3) and matching (Eq. 5)."""
import numpy as np
import pytest

import synth
from oracle import epg, match as omatch
from gpu_util import as_f32_inputs, c64, dev, f32, mrf, np_, rand_c, rel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("T", [1, 2, 7, 100, 1000])
def test_epg_matches_oracle(T):
    m = mrf()
    fa, tr = synth.fisp_train(T, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(100, 4000, 7), synth.log_grid(10, 500, 6))
    lut, fa, tr = as_f32_inputs(lut, fa, tr)
    D = np_(m.epg_fisp(f32(lut), f32(fa), f32(tr)))
    D0 = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    for i in range(len(lut)):
        assert rel(D[i], D0[i]) < 2e-5, (i, lut[i])


def test_epg_no_inversion():
    m = mrf()
    fa, tr = synth.fisp_train(50, seed=3)
    lut = np.array([[800.0, 60.0], [2000.0, 200.0]])
    lut, fa, tr = as_f32_inputs(lut, fa, tr)
    D = np_(m.epg_fisp(f32(lut), f32(fa), f32(tr), inversion=False))
    assert rel(D, epg.fisp(lut[:, 0], lut[:, 1], fa, tr, inversion=False)) < 2e-5


@pytest.fixture(scope="module")
def dict100():
    fa, tr = synth.fisp_train(100, seed=2)
    lut = synth.workload_grid(synth.WORKLOADS["mrf64_t100"])
    D = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    (D,) = as_f32_inputs(D)
    return lut, D


def _valid_choice(X, D, gidx, oidx, atom_norm2=None, rtol=1e-5):
    """Indices must agree except at near-ties, where the GPU's pick must score within rtol of the best."""
    sc = omatch.scores(X, D, atom_norm2)
    rows = np.arange(len(X))
    best = sc[rows, oidx]
    mine = sc[rows, gidx]
    diff = gidx != oidx
    assert np.all(mine[diff] >= best[diff] * (1 - rtol)), np.nonzero(diff)[0][:10]
    return diff.mean()


def test_noiseless_atoms_bit_exact(dict100):
    m = mrf()
    lut, D = dict100
    rng = np.random.default_rng(0)
    pd = rng.uniform(0.5, 1.0, len(D))
    X = as_f32_inputs(D * pd[:, None])[0]
    idx, pdh, t1t2 = m.match(c64(X), c64(D), f32(lut))
    idx = np_(idx)
    np.testing.assert_array_equal(idx, np.arange(len(D)))
    np.testing.assert_allclose(np_(pdh), pd, rtol=2e-5)
    np.testing.assert_array_equal(np_(t1t2), lut.astype(np.float32))


def test_noisy_matches_oracle_several_tiles_ragged(dict100):
    m = mrf()
    lut, D = dict100
    rng = np.random.default_rng(1)
    n = 1000
    pick = rng.integers(0, len(D), n)
    X = D[pick] * rng.uniform(0.2, 2.0, (n, 1)) + 0.05 * rand_c(rng, n, D.shape[1])
    X[:7] = 0.0                                       # air: index 0, PD 0
    X[7] = -D[3]                                      # negative phase: PD clamped to 0
    (X,) = as_f32_inputs(X)
    idx, pd, _ = m.match(c64(X), c64(D), f32(lut))
    idx, pd = np_(idx), np_(pd)
    oidx, _, _, opd = omatch.match(X, D, lut)
    assert _valid_choice(X, D, idx, oidx) < 0.01
    same = idx == oidx
    np.testing.assert_allclose(pd[same], opd[same], rtol=1e-4, atol=1e-6)
    assert np.all(idx[:7] == 0) and np.all(pd[:7] == 0)
    assert idx[7] == 3 and pd[7] == 0


def test_ragged_sizes_and_given_norms():
    m = mrf()
    rng = np.random.default_rng(2)
    n, mm, L = 333, 131, 37
    D = rand_c(rng, mm, L)
    X = rand_c(rng, n, L)
    n2 = rng.uniform(0.5, 3.0, mm)
    lut = rng.uniform(10, 1000, (mm, 2))
    D, X, n2, lut = as_f32_inputs(D, X, n2, lut)
    idx, pd, _ = m.match(c64(X), c64(D), f32(lut), atom_norm2=f32(n2))
    oidx, _, _, opd = omatch.match(X, D, lut, atom_norm2=n2)
    idx = np_(idx)
    _valid_choice(X, D, idx, oidx, atom_norm2=n2)
    same = idx == oidx
    np.testing.assert_allclose(np_(pd)[same], opd[same], rtol=1e-4, atol=1e-6)


def test_literal_norm2_flag():
    m = mrf()
    D = np.array([[2.0, 0.0], [1.0, 0.0], [0.0, 1.0]], complex)
    lut = np.array([[1.0, 1.0], [2.0, 2.0], [3.0, 3.0]])
    x = np.array([[1.0, 0.1]], complex)
    assert np_(m.match(c64(x), c64(D), f32(lut))[0])[0] == 0
    assert np_(m.match(c64(x), c64(D), f32(lut), precision=0x100)[0])[0] == 1
