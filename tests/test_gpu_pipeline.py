"""GPU parity of the whole-path entry points.

* mrf_gridding_match, the plain reconstruction of the 64^2 x 100-frame
  workload (X = A^H b frame by frame, then exhaustive matching of the full
  100-frame fingerprints against 1500 EPG atoms): fingerprints within the
  NUFFT bound (1e-4) of the oracle's KB adjoint, indices equal to the
  oracle's matching of its own fingerprints except at near-ties (score within
  1e-4 of the best: the two sides' fingerprints differ by ~1e-5), PD to 1e-3.
* mrf_recon_run_host (host k-space in, host maps out) gives the maps of the
  device-pointer loop (mrf_recon_create + mrf_recon_iter + mrf_recon_maps)."""
import numpy as np
import pytest
import torch

import synth
from oracle import epg, match as omatch, nufft as onufft
from gpu_util import as_f32_inputs, c64, f32, mrf, np_, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1():
    w = synth.WORKLOADS["mrf64_t100"]
    t1, t2, pd, mask, _ = synth.phantom(w.n, seed=w.phantom_seed)
    fa, tr = synth.fisp_train(w.frames, seed=w.tr_seed)
    lut = synth.workload_grid(w)
    D = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    X = pd.reshape(-1, 1) * epg.fisp(np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0), fa, tr)
    X *= mask.reshape(-1, 1)
    k = synth.spiral_trajectory(w.n, w.frames, w.ns, w.interleaves)
    grid = onufft.KBGrid(w.n, w.n, w.os, w.kb_width)
    b = onufft.kb_forward(X.reshape(w.n, w.n, w.frames).transpose(2, 0, 1), k, grid)
    sig = np.sqrt(np.mean(np.abs(b) ** 2) * 10 ** (-w.snr_db / 10))
    b = b + sig * synth.complex_normal(b.shape, seed=w.noise_seed)
    k, b, D, lut = as_f32_inputs(k, b, D, lut)
    return dict(w=w, k=k, b=b, D=D, lut=lut, grid=grid, mask=mask)


def test_gridding_match_follows_oracle(c1):
    m = mrf()
    w = c1["w"]
    plan = m.nufft_plan(w.n, w.n, f32(c1["k"]))
    idx, pd, t1t2, rows = m.gridding_match(plan, c64(c1["b"]), c64(c1["D"]), f32(c1["lut"]), keep_rows=True)
    xa = onufft.kb_adjoint(c1["b"], c1["k"], c1["grid"])                  # [T, n, n]
    Xo = xa.reshape(w.frames, -1).T                                       # [n^2, T]
    assert rel(np_(rows), Xo) < 1e-4
    oi, ot1, ot2, opd = omatch.match(Xo, c1["D"], c1["lut"])
    gi = np_(idx)
    sc = omatch.scores(Xo, c1["D"])
    r = np.arange(len(gi))
    assert np.all(sc[r, gi] >= sc[r, oi] * (1 - 1e-4))
    same = gi == oi
    assert same.mean() > 0.99
    np.testing.assert_allclose(np_(pd)[same], opd[same], rtol=1e-3, atol=1e-6 * np.abs(opd).max())
    np.testing.assert_array_equal(np_(t1t2)[same], np.stack([ot1, ot2], -1)[same].astype(np.float32))


def test_gridding_match_rejects_mismatched_dictionary(c1):
    m = mrf()
    w = c1["w"]
    plan = m.nufft_plan(w.n, w.n, f32(c1["k"]))
    with pytest.raises(ValueError):
        m.gridding_match(plan, c64(c1["b"]), c64(c1["D"][:, :50]), f32(c1["lut"]))


def test_recon_run_host_gives_the_device_loop_maps():
    from test_gpu_recon import problem
    m = mrf()
    pr = problem(K=10)
    plan = m.nufft_plan(pr["n"], pr["n"], f32(pr["k"]))
    dc = c64(pr["D"] @ pr["phi"])
    n2 = f32(np.sum(np.abs(pr["D"]) ** 2, axis=1))
    phi, lut = c64(pr["phi"]), f32(pr["lut"])
    p = m.ReconParams(patch=8, stride=4, knn=10, flags=8 | 32, match_precision=2)   # grouped, serial
    rec = m.Recon(plan, p, phi, dc, n2, lut, c64(pr["b"]))
    c_dev = rec.iterate(3, costs=True)
    t1, t2, pdm, _ = [np_(t) for t in rec.maps()]
    del rec
    b_host = torch.tensor(np.ascontiguousarray(pr["b"]), dtype=torch.complex64).pin_memory()
    (h1, h2, hp), c_host = m.recon_run_host(plan, p, phi, dc, n2, lut, b_host, 3, costs=True)
    same = h1.numpy() == t1
    assert same.mean() > 0.99 and (h2.numpy() == t2).mean() > 0.99
    np.testing.assert_allclose(hp.numpy()[same], pdm[same], rtol=1e-3, atol=1e-6 * np.abs(pdm).max())
    np.testing.assert_allclose(c_host, c_dev, rtol=5e-3)
    # pageable host memory is accepted too
    pageable = torch.tensor(np.ascontiguousarray(pr["b"]), dtype=torch.complex64)
    (g1, _, _) = m.recon_run_host(plan, p, phi, dc, n2, lut, pageable, 1)
    assert np.isfinite(g1.numpy()).all()
