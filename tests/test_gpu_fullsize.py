"""Parity at the full 256^2 x 1000-frame workload, in the launch configuration
bench.py times (48 shared interleaves, 2048 samples, grid 512, W = 4,
5441-atom dictionary compressed to K = 10).

The oracle cannot run the whole workload, so it checks sampled outputs it can
compute one by one (a few frames of the NUFFT, a few hundred voxels of the
matching, a few patches of the SVT input) and properties that hold at any
size (adjointness, frame form == grouped form, iterates stay finite)."""
import numpy as np
import pytest
import torch

import synth
from oracle import match as omatch, nufft as onufft
from gpu_util import c64, f32, mrf, np_, rand_c, rel

pytestmark = pytest.mark.gpu

W = synth.WORKLOADS["mrf256_t1000"]


@pytest.fixture(scope="module")
def full():
    m = mrf()
    k = synth.spiral_trajectory(W.n, W.frames, W.ns, W.interleaves).astype(np.float32)
    plan = m.nufft_plan(W.n, W.n, f32(k), os=W.os, kb_width=W.kb_width)
    return m, plan, k.astype(np.float64)


def test_full_size_forward_adjoint_sampled_frames(full):
    m, plan, k = full
    rng = np.random.default_rng(0)
    x = torch.complex(torch.randn(W.frames, W.n, W.n, device="cuda"), torch.randn(W.frames, W.n, W.n, device="cuda"))
    y = m.nufft_forward(plan, x)
    r = torch.complex(torch.randn(W.frames, W.ns, device="cuda"), torch.randn(W.frames, W.ns, device="cuda"))
    xa = m.nufft_adjoint(plan, r)
    grid = onufft.KBGrid(W.n, W.n, W.os, W.kb_width)
    for t in rng.choice(W.frames, 3, replace=False):
        xt = np_(x[t])[None].astype(np.complex128)
        assert rel(np_(y[t]), onufft.kb_forward(xt, k[t:t + 1], grid)[0]) < 1e-4
        rt = np_(r[t])[None].astype(np.complex128)
        assert rel(np_(xa[t]), onufft.kb_adjoint(rt, k[t:t + 1], grid)[0]) < 1e-4
    # adjointness over all 1000 frames (FP32 sums of 65M terms)
    lhs = torch.vdot(y.flatten().to(torch.complex128), r.flatten().to(torch.complex128))
    rhs = torch.vdot(x.flatten().to(torch.complex128), xa.flatten().to(torch.complex128))
    assert abs(complex(lhs - rhs)) / abs(complex(lhs)) < 1e-5


def test_full_size_frame_and_grouped_subspace_forms_agree(full):
    m, plan, k = full
    rng = np.random.default_rng(1)
    phi, _ = np.linalg.qr(rand_c(rng, W.frames, W.rank))
    phi_d = c64(phi)
    alpha = torch.complex(torch.randn(W.n, W.n, W.rank, device="cuda"), torch.randn(W.n, W.n, W.rank, device="cuda"))
    b = torch.complex(torch.randn(W.frames, W.ns, device="cuda"), torch.randn(W.frames, W.ns, device="cuda"))
    y0 = m.nufft_forward_subspace(plan, alpha, phi_d, 0.5, b, mode=0)
    y1 = m.nufft_forward_subspace(plan, alpha, phi_d, 0.5, b, mode=1)
    assert rel(np_(y1), np_(y0)) < 1e-4
    a0 = m.nufft_adjoint_subspace(plan, b, phi_d, 0.5, mode=0)
    a1 = m.nufft_adjoint_subspace(plan, b, phi_d, 0.5, mode=1)
    assert rel(np_(a1), np_(a0)) < 1e-4
    # one sampled frame against the oracle
    t = 417
    grid = onufft.KBGrid(W.n, W.n, W.os, W.kb_width)
    al = np_(alpha).astype(np.complex128)
    xt = (al @ phi.astype(np.complex64).astype(np.complex128)[t].conj())[None]
    yt = 0.5 * onufft.kb_forward(xt, k[t:t + 1], grid)[0] - np_(b[t])
    assert rel(np_(y1[t]), yt) < 1e-4


def test_full_size_dictionary_and_matching_sampled_voxels(full):
    m, plan, k = full
    fa, tr = synth.fisp_train(W.frames, seed=W.tr_seed)
    lut = synth.workload_grid(W)
    D = m.epg_fisp(f32(lut), f32(fa), f32(tr))
    phi, comp, n2 = m.dict_subspace(D, W.rank)
    rng = np.random.default_rng(2)
    N = W.n * W.n
    pick = torch.tensor(rng.integers(0, len(lut), N), device="cuda")
    alpha = comp[pick] * torch.rand(N, 1, device="cuda") + 0.05 * torch.complex(
        torch.randn(N, W.rank, device="cuda"), torch.randn(N, W.rank, device="cuda"))
    lut_d = f32(lut)
    gi32, pd32, _ = m.match(alpha, comp, lut_d, atom_norm2=n2, precision=0)
    gi3, pd3, _ = m.match(alpha, comp, lut_d, atom_norm2=n2, precision=2)
    assert (np_(gi3) == np_(gi32)).mean() > 0.995
    sample = rng.choice(N, 400, replace=False)
    X = np_(alpha[sample]).astype(np.complex128)
    Dc = np_(comp).astype(np.complex128)
    nn = np_(n2).astype(np.float64)
    oi, _, _, opd = omatch.match(X, Dc, lut, atom_norm2=nn)
    sc = omatch.scores(X, Dc, nn)
    rows = np.arange(len(sample))
    for gi in (np_(gi32)[sample], np_(gi3)[sample]):
        ok = (gi == oi) | (sc[rows, gi] >= sc[rows, oi] * (1 - 1e-5))
        assert ok.mean() >= 0.995


def test_full_size_recon_iterations_stay_finite_and_modes_agree(full):
    m, plan, k = full
    fa, tr = synth.fisp_train(W.frames, seed=W.tr_seed)
    lut = synth.workload_grid(W)
    D = m.epg_fisp(f32(lut), f32(fa), f32(tr))
    phi, comp, n2 = m.dict_subspace(D, W.rank)
    t1, t2, pd, mask, label = synth.phantom(W.n, seed=0)
    pairs = np.stack([np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0)], -1)
    S = m.epg_fisp(f32(pairs), f32(fa), f32(tr))
    X = (S * c64((pd * mask).ravel())[:, None]).T.contiguous().view(W.frames, W.n, W.n)
    b = m.nufft_forward(plan, X)
    del X, S
    costs = {}
    alphas = {}
    for flags, prec in ((0, 0), (8, 2)):
        p = m.ReconParams(patch=W.patch, stride=W.stride, knn=W.knn, flags=flags, match_precision=prec,
                          a_norm=0.0)
        r = m.Recon(plan, p, phi, comp, n2, f32(lut), b)
        c = r.iterate(2, costs=True)
        assert all(np.isfinite(c))
        costs[flags] = c
        alphas[flags] = np_(r.alpha())
    assert costs[8][0] == pytest.approx(costs[0][0], rel=1e-3)
    assert rel(alphas[8], alphas[0]) < 1e-2
