"""Seeded tensor-core matching (mrf_match_seeded) gives exactly the result
of the unseeded matcher, whatever the seeds.

A row's seeds only set the starting threshold of its candidate list: the
smallest FP32 score among TOPK distinct seed atoms, less a margin above the
tensor-core score error.  Every atom of the final top TOPK scores above
that, so the list -- and the FP32 re-rank of it -- must come out identical,
element by element, to an unseeded call: for seeds that are the row's own
candidates, the candidates of a perturbed fingerprint (the loop's case),
random distinct atoms, and invalid seeds (-1, repeats, out of range: the
row is then unseeded).  Checked for the split-BF16 (top 4) and BF16 (top 8)
forms on a ragged row count and at the full workload's size (65536
fingerprints x 5441 atoms, K = 10) in the loop's launch configuration."""
import numpy as np
import pytest
import torch

import synth
from oracle import dictionary, epg
from gpu_util import as_f32_inputs, c64, dev, f32, mrf, np_, rand_c

pytestmark = pytest.mark.gpu
BF16, BF16X3 = 1, 2
TOPK = {BF16: 8, BF16X3: 4}


@pytest.fixture(scope="module")
def compressed():
    fa, tr = synth.fisp_train(200, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(100, 4000, 60), synth.log_grid(10, 500, 40))
    D = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    phi = dictionary.subspace(D, 10)
    Dc, n2, lut = as_f32_inputs(D @ phi, np.sum(np.abs(D) ** 2, axis=1), lut)
    return c64(Dc), f32(n2), f32(lut)


def _cand(n, fill=-1):
    return torch.full((n, 8), fill, dtype=torch.int32, device=dev())


def _same(a, b):
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def _check_all_seeds(X, Dc, n2, lut, prec, rng):
    m = mrf()
    n, M, k = X.shape[0], Dc.shape[0], TOPK[prec]
    ref = m.match(X, Dc, lut, atom_norm2=n2, precision=prec)
    c0 = _cand(n)
    _same(m.match_seeded(X, Dc, lut, c0, atom_norm2=n2, precision=prec), ref)
    assert torch.all((c0[:, :k] >= 0) & (c0[:, :k] < M)) and torch.all(c0[:, k:] == -1)
    # seeds: the row's own candidates
    c = c0.clone()
    _same(m.match_seeded(X, Dc, lut, c, atom_norm2=n2, precision=prec), ref)
    assert torch.equal(c, c0)
    # seeds: candidates of a perturbed fingerprint
    Xp = X + 0.05 * X.abs().mean() * torch.complex(torch.randn_like(X.real), torch.randn_like(X.real))
    c = _cand(n)
    m.match_seeded(Xp, Dc, lut, c, atom_norm2=n2, precision=prec)
    _same(m.match_seeded(X, Dc, lut, c, atom_norm2=n2, precision=prec), ref)
    assert torch.equal(c, c0)
    # seeds: random distinct atoms
    r = np.stack([rng.choice(M, k, replace=False) for _ in range(n)])
    c = _cand(n)
    c[:, :k] = torch.tensor(r, dtype=torch.int32, device=dev())
    _same(m.match_seeded(X, Dc, lut, c, atom_norm2=n2, precision=prec), ref)
    assert torch.equal(c, c0)
    # invalid seeds: repeats, out of range, negative (rows left unseeded)
    c = c0.clone()
    c[0::3, 1] = c[0::3, 0]
    c[1::3, 0] = M
    c[2::3, k - 1] = -5
    _same(m.match_seeded(X, Dc, lut, c, atom_norm2=n2, precision=prec), ref)
    assert torch.equal(c, c0)


@pytest.mark.parametrize("prec", [BF16X3, BF16])
def test_seeded_matching_is_exact_ragged(compressed, prec):
    Dc, n2, lut = compressed
    rng = np.random.default_rng(prec)
    n = 3001                                          # 24 blocks of 128 rows, ragged tail
    Dh = np_(Dc)
    X = Dh[rng.integers(0, len(Dh), n)] * rng.uniform(0.3, 2.0, (n, 1)) + 0.02 * rand_c(rng, n, Dh.shape[1])
    X[5] = 0                                          # an all-zero fingerprint stays unseeded
    _check_all_seeds(c64(X.astype(np.complex64)), Dc, n2, lut, prec, rng)


def test_seeded_matching_is_exact_full_size():
    m = mrf()
    W = synth.WORKLOADS["mrf256_t1000"]
    fa, tr = synth.fisp_train(W.frames, seed=W.tr_seed)
    lut = f32(synth.workload_grid(W))
    D = m.epg_fisp(lut, f32(fa), f32(tr))
    phi, comp, n2 = m.dict_subspace(D, W.rank)
    N = W.n * W.n
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    pick = torch.randint(0, comp.shape[0], (N,), device="cuda", generator=gen)
    X = comp[pick] * (torch.rand(N, 1, device="cuda", generator=gen) + 0.2) + 0.02 * torch.complex(
        torch.randn(N, W.rank, device="cuda", generator=gen), torch.randn(N, W.rank, device="cuda", generator=gen))
    _check_all_seeds(X.contiguous(), comp, n2, lut, BF16X3, np.random.default_rng(12))


def test_seeded_matching_rejects_other_precisions(compressed):
    m = mrf()
    Dc, n2, lut = compressed
    X = Dc[:10].contiguous()
    for prec in (0, 3):
        with pytest.raises(m.MRFError):
            m.match_seeded(X, Dc, lut, _cand(10), atom_norm2=n2, precision=prec)
