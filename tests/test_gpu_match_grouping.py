"""Tensor-core matching (Eq. 5, subspace-length fingerprints): a row's
winner cannot depend on how the rows are grouped.  The matcher tiles the
rows in blocks of 128, runs the blocks in waves over the SMs and keeps a
candidate list per row; matching any slice of the rows on its own (other
block boundaries, other waves, a ragged last block) must give the same
indices and inner products, bit for bit.  Checked with more row blocks than
two waves of blocks, with a dictionary of a single atom tile, and against
the FP32 matcher and the FP64 oracle up to near ties."""
import numpy as np
import pytest
import torch

import synth
from oracle import dictionary, epg, match as omatch
from gpu_util import as_f32_inputs, c64, f32, mrf, np_, rand_c

pytestmark = pytest.mark.gpu
BF16, BF16X3 = 1, 2


@pytest.fixture(scope="module")
def compressed():
    fa, tr = synth.fisp_train(200, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(100, 4000, 60), synth.log_grid(10, 500, 40))
    D = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    phi = dictionary.subspace(D, 10)
    Dc, n2, lut = as_f32_inputs(D @ phi, np.sum(np.abs(D) ** 2, axis=1), lut)
    return Dc, n2, lut


def _rows(Dc, n, seed):
    rng = np.random.default_rng(seed)
    X = Dc[rng.integers(0, len(Dc), n)] * rng.uniform(0.3, 2.0, (n, 1)) + 0.02 * rand_c(rng, n, Dc.shape[1])
    (X,) = as_f32_inputs(X)
    return X


def _sms():
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("prec", [BF16X3, BF16])
def test_results_do_not_depend_on_the_grouping_of_rows(compressed, prec):
    m = mrf()
    Dc, n2, lut = compressed
    n = (2 * _sms() + 9) * 128 + 77                 # more row blocks than two waves, ragged tail
    X = _rows(Dc, n, 5)
    Xd, Dd, Ld, Nd = c64(X), c64(Dc), f32(lut), f32(n2)
    idx, pd, _ = m.match(Xd, Dd, Ld, atom_norm2=Nd, precision=prec)
    idx, pd = np_(idx), np_(pd)
    for a, b in ((0, 128), (77, 3001), (1000, 1000 + 128 * _sms() + 5), (n - 300, n), (5, n - 5)):
        i2, p2, _ = m.match(Xd[a:b].contiguous(), Dd, Ld, atom_norm2=Nd, precision=prec)
        np.testing.assert_array_equal(np_(i2), idx[a:b])
        np.testing.assert_array_equal(np_(p2), pd[a:b])


def test_many_row_blocks_agree_with_fp32_and_oracle(compressed):
    m = mrf()
    Dc, n2, lut = compressed
    n = (2 * _sms() + 9) * 128 + 77
    X = _rows(Dc, n, 6)
    X[:3] = 0.0
    gb, pb, _ = m.match(c64(X), c64(Dc), f32(lut), atom_norm2=f32(n2), precision=BF16X3)
    gf, _, _ = m.match(c64(X), c64(Dc), f32(lut), atom_norm2=f32(n2), precision=0)
    gb, gf = np_(gb), np_(gf)
    assert (gb == gf).mean() >= 0.995
    assert np.all(gb[:3] == 0) and np.all(np_(pb)[:3] == 0)
    # the oracle on every 7th row (scores of all atoms in FP64)
    rows = np.arange(3, n, 7)
    oi, _, _, _ = omatch.match(X[rows], Dc, lut, atom_norm2=n2)
    sc = omatch.scores(X[rows], Dc, n2)
    r = np.arange(len(rows))
    ok = (gb[rows] == oi) | (sc[r, gb[rows]] >= sc[r, oi] * (1 - 1e-5))
    assert ok.mean() >= 0.995


@pytest.mark.parametrize("n", [300, 128 * 313 + 1])
def test_single_tile_dictionary(compressed, n):
    # 50 atoms: a single (ragged) atom tile
    m = mrf()
    Dc, n2, lut = compressed
    sel = np.linspace(0, len(Dc) - 1, 50).astype(int)
    D50, N50, L50 = Dc[sel], n2[sel], lut[sel]
    X = _rows(D50, n, 7)
    gb, _, _ = m.match(c64(X), c64(D50), f32(L50), atom_norm2=f32(N50), precision=BF16X3)
    gf, _, _ = m.match(c64(X), c64(D50), f32(L50), atom_norm2=f32(N50), precision=0)
    assert (np_(gb) == np_(gf)).mean() >= 0.999


def test_seeded_matching_of_many_row_blocks_equals_unseeded(compressed):
    m = mrf()
    Dc, n2, lut = compressed
    n = (2 * _sms() + 9) * 128 + 77
    X = c64(_rows(Dc, n, 8))
    Dd, Ld, Nd = c64(Dc), f32(lut), f32(n2)
    ref = m.match(X, Dd, Ld, atom_norm2=Nd, precision=BF16X3)
    Xp = (X + 0.05 * X.abs().mean() * torch.complex(torch.randn_like(X.real), torch.randn_like(X.real))).contiguous()
    cand = torch.full((n, 8), -1, dtype=torch.int32, device=X.device)
    m.match_seeded(Xp, Dd, Ld, cand, atom_norm2=Nd, precision=BF16X3)
    got = m.match_seeded(X, Dd, Ld, cand, atom_norm2=Nd, precision=BF16X3)
    for u, v in zip(got, ref):
        assert torch.equal(u, v)
