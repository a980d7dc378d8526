"""GPU parity of the learned matcher against the FP64 oracle (oracle/mlp.py):
gradient of the loss (with the BF16 weights the products use and the FP32
biases), one Adam step, the training-set transform, and inference; then
training on a small synthetic set and the learned matcher inside the loop.

Tolerances: FP32 accumulation over at most 1024-term sums, relative 1e-4
on whole vectors (5e-4 on the largest layer's gradient)."""
import numpy as np
import pytest
import torch

import synth
from oracle import epg, mlp as omlp
from gpu_util import c64, dev, f32, mrf, np_, rand_c, rel

pytestmark = pytest.mark.gpu

RANGES = (100.0, 4000.0, 10.0, 500.0, 0.05)


def _weight_mask():
    mask, at = np.zeros(omlp.n_params(), bool), 0
    for i, o in zip(omlp.SIZES[:-1], omlp.SIZES[1:]):
        mask[at:at + o * i] = True
        at += o * i + o
    return mask


def _net(seed=0, batch=256):
    m = mrf()
    p = synth.mlp_init_params(seed)
    p[~_weight_mask()] = 0.05 * np.random.default_rng(seed + 1).standard_normal((~_weight_mask()).sum())
    return m.Mlp(p, RANGES, max_batch=batch)


def _used_params(net):
    master, bf = net.params()
    theta = master.astype(np.float64)
    w = _weight_mask()
    theta[w] = bf[w]
    return theta


def test_gradient_matches_oracle():
    net = _net(0)
    rng = np.random.default_rng(2)
    B = 200
    x = rng.standard_normal((B, 20)).astype(np.float32)
    t = rng.standard_normal((B, 3)).astype(np.float32)
    g, loss = net.grad(f32(x), f32(t))
    theta = _used_params(net)
    y, cache = omlp.forward(theta, x.astype(np.float64))
    go = omlp.backward(theta, cache, y, t.astype(np.float64))
    assert float(np_(loss)[0]) == pytest.approx(omlp.loss(y, t), rel=1e-5)
    gg = np_(g).astype(np.float64)
    assert rel(gg, go) < 1e-4
    at = 0
    for i, o in zip(omlp.SIZES[:-1], omlp.SIZES[1:]):
        sl = slice(at, at + o * i + o)
        assert rel(gg[sl], go[sl]) < 5e-4, (i, o)
        at += o * i + o


def test_adam_step_matches_oracle():
    net = _net(3)
    rng = np.random.default_rng(4)
    x, t = f32(rng.standard_normal((128, 20))), f32(rng.standard_normal((128, 3)))
    g, _ = net.grad(x, t)
    before, _ = net.params()
    net.train_step(x, t, 1e-3)
    after, bf = net.params()
    ref, m, v = omlp.adam_step(before.astype(np.float64), np_(g).astype(np.float64), 0.0, 0.0, 1, 1e-3)
    np.testing.assert_allclose(after, ref, rtol=1e-5, atol=1e-7)
    w = _weight_mask()
    np.testing.assert_allclose(bf[w], after[w], rtol=2 ** -8)     # the BF16 copy follows the master weights


def test_training_set_matches_oracle():
    m = mrf()
    T, K, n = 120, 10, 500
    fa, tr = synth.fisp_train(T, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(100, 4000, 30), synth.log_grid(10, 500, 20))
    D = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    from oracle import dictionary
    phi = dictionary.subspace(D, K)
    t1t2, rho, snr, noise = synth.mlp_training_draws(n, K, seed=5)
    sig = m.epg_fisp(f32(t1t2), f32(fa), f32(tr))
    x, y = m.mlp_training_set(sig, f32(t1t2), f32(rho), f32(snr), c64(noise), c64(phi), RANGES)
    xo, yo = omlp.training_set(np_(sig), t1t2.astype(np.float32), rho.astype(np.float32),
                               snr.astype(np.float32), noise.astype(np.complex64),
                               phi.astype(np.complex64), RANGES)
    assert rel(np_(x), xo) < 1e-5
    assert rel(np_(y), yo) < 1e-5


def test_tensor_core_and_simt_training_products_agree():
    """The training products run on tcgen05 (split BF16, FP32 accumulation)
    by default; the SIMT engine computes the same gradient to the split
    form's ~2^-16, on a batch whose 1000 rows are not a multiple of the
    128-row tile, and both match the oracle's backward pass."""
    net = _net(3, batch=1000)
    rng = np.random.default_rng(4)
    B = 1000
    x = rng.standard_normal((B, 20)).astype(np.float32)
    t = rng.standard_normal((B, 3)).astype(np.float32)
    g_tc, l_tc = net.grad(f32(x), f32(t))
    g_tc = np_(g_tc).astype(np.float64)
    net.check()
    net.set_engine(tensor_cores=False)
    g_si, l_si = net.grad(f32(x), f32(t))
    g_si = np_(g_si).astype(np.float64)
    net.set_engine(tensor_cores=True)
    assert rel(g_tc, g_si) < 2e-5
    assert float(np_(l_tc)[0]) == pytest.approx(float(np_(l_si)[0]), rel=1e-5)
    theta = _used_params(net)
    y, cache = omlp.forward(theta, x.astype(np.float64))
    assert rel(g_tc, omlp.backward(theta, cache, y, t.astype(np.float64))) < 1e-4


def test_inference_matches_oracle_forward():
    """SIMT engine: FP32 activations.  Tensor-core engine: each layer's input
    rounded to BF16 (the oracle rounds the same way, from its FP64 values, so
    an activation can land one BF16 step apart: 2^-8 relative, rarely)."""
    net = _net(6)
    rng = np.random.default_rng(7)
    theta = _used_params(net)
    for n in (1000, 128 * 152 * 2 + 77):                      # ragged tails; more tiles than SMs
        x = rng.standard_normal((n, 20)).astype(np.float32)
        net.set_engine(tensor_cores=False)
        y = np_(net.infer(f32(x)))
        yo, _ = omlp.forward(theta, x.astype(np.float64))
        assert rel(y, yo) < 1e-4
        net.set_engine(tensor_cores=True)
        yt = np_(net.infer(f32(x)))
        net.check()
        yb, _ = omlp.forward(theta, x.astype(np.float64), act_bf16=True)
        assert rel(yt, yb) < 2e-3
        assert rel(yt, yo) < 2e-2


def _small_problem(T=200, K=10):
    m = mrf()
    fa, tr = synth.fisp_train(T, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(100, 4000, 60), synth.log_grid(10, 500, 40))
    D = m.epg_fisp(f32(lut), f32(fa), f32(tr))
    phi, comp, n2 = m.dict_subspace(D, K)
    return m, fa, tr, lut, phi, comp, n2


def test_training_learns_the_parameter_map():
    m, fa, tr, lut, phi, comp, n2 = _small_problem()
    pd_scale = float(1.0 / np.median(np.sqrt(np_(n2))))
    ranges = RANGES[:4] + (pd_scale,)
    draws = synth.mlp_training_draws(200_000, 10, seed=8)
    net, hist = m.train_matcher(synth.mlp_init_params(9), draws, f32(fa), f32(tr), phi, ranges, epochs=3,
                                batch=1024)
    assert hist[-1] < 0.25 * hist[0]
    # held-out noisy fingerprints: learned maps against the truth and against exhaustive matching
    test = synth.mlp_training_draws(4000, 10, seed=10, snr_db_range=(30.0, 30.0))
    tt = f32(test[0])
    sig = m.epg_fisp(tt, f32(fa), f32(tr))
    x, y = m.mlp_training_set(sig, tt, f32(test[1]), f32(test[2]), c64(test[3]), phi, ranges)
    u = np_(net.infer(x))
    t1 = np.exp(np.log(100) + 0.5 * (u[:, 0] + 1) * np.log(40.0))
    t2 = np.exp(np.log(10) + 0.5 * (u[:, 1] + 1) * np.log(50.0))
    e1 = np.linalg.norm(t1 - test[0][:, 0]) / np.linalg.norm(test[0][:, 0])
    e2 = np.linalg.norm(t2 - test[0][:, 1]) / np.linalg.norm(test[0][:, 1])
    assert e1 < 0.15 and e2 < 0.3, (e1, e2)


def test_learned_matcher_in_the_loop():
    """The loop runs with the learned matcher; its maps stay close to the
    exhaustive loop's, and fingerprints it maps off the dictionary's box go
    through the exhaustive fallback (idx >= 0 there, -1 elsewhere)."""
    m, fa, tr, lut, phi, comp, n2 = _small_problem(T=100)
    n = 64
    pd_scale = float(1.0 / np.median(np.sqrt(np_(n2))))
    ranges = RANGES[:4] + (pd_scale,)
    net, _ = m.train_matcher(synth.mlp_init_params(11), synth.mlp_training_draws(200_000, 10, seed=12),
                             f32(fa), f32(tr), phi, ranges, epochs=3, batch=1024)
    t1, t2, pd, mask, _ = synth.phantom(n, seed=0)
    pairs = np.stack([np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0)], -1)
    S = m.epg_fisp(f32(pairs), f32(fa), f32(tr))
    X = (S * c64((pd * mask).ravel())[:, None]).T.contiguous().view(100, n, n)
    k = f32(synth.spiral_trajectory(n, 100, 512, 10).astype(np.float32))
    plan = m.nufft_plan(n, n, k)
    b = m.nufft_forward(plan, X)
    maps = {}
    for name, flags, mlp in (("exhaustive", 8, None), ("learned", 8 | 16, net)):
        p = m.ReconParams(patch=8, stride=4, knn=4, flags=flags, match_precision=2, mlp=mlp)
        r = m.Recon(m.nufft_plan(n, n, k), p, phi, comp, n2, f32(lut), b)
        r.iterate(5)
        maps[name] = [np_(v) for v in r.maps()]
    mk = mask.astype(bool)
    for i in (0, 1):
        e = np.linalg.norm((maps["learned"][i] - maps["exhaustive"][i])[mk]) / np.linalg.norm(maps["exhaustive"][i][mk])
        assert e < 0.25, (i, e)
        assert np.all(np.isfinite(maps["learned"][i]))
    idx = maps["learned"][3]
    assert np.all((idx == -1) | ((idx >= 0) & (idx < len(lut))))


def test_learned_matcher_gain_over_exhaustive_matching():
    """What the trained network gains over the method without it, measured in
    the loop at K = 10 on the 256^2 image of the benchmark (100 frames, 2048
    samples from 48 interleaves) matched against its 5441-atom grid: per
    iteration, the device time of the matching step
    (features, network inference on the tensor cores, decoding and the
    exhaustive fallback) against the seeded split-BF16 exhaustive matcher,
    from the library's per-kernel CUDA events with the steps serialised;
    the learned maps stay within the error of the exhaustive loop's maps
    that the in-loop test allows."""
    m = mrf()
    w = synth.WORKLOADS["mrf256_t100"]
    fa, tr = synth.fisp_train(100, seed=w.tr_seed)
    lut = synth.workload_grid(w)
    D = m.epg_fisp(f32(lut), f32(fa), f32(tr))
    phi, comp, n2 = m.dict_subspace(D, 10)
    pd_scale = float(1.0 / np.median(np.sqrt(np_(n2))))
    ranges = (w.t1_range[0], w.t1_range[1], w.t2_range[0], w.t2_range[1], pd_scale)
    net, _ = m.train_matcher(synth.mlp_init_params(21), synth.mlp_training_draws(300_000, 10, seed=22,
                                                                                  t1_range=w.t1_range,
                                                                                  t2_range=w.t2_range),
                             f32(fa), f32(tr), phi, ranges, epochs=3, batch=1024)
    n = w.n
    t1, t2, pd, mask, _ = synth.phantom(n, seed=0)
    pairs = np.stack([np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0)], -1)
    S = m.epg_fisp(f32(pairs), f32(fa), f32(tr))
    X = (S * c64((pd * mask).ravel())[:, None]).T.contiguous().view(100, n, n)
    k = f32(synth.spiral_trajectory(n, 100, w.ns, w.interleaves).astype(np.float32))
    b = m.nufft_forward(m.nufft_plan(n, n, k), X)
    # the matching step's kernels: the exhaustive matcher's, and the network's
    # with its decoding and exhaustive fallback
    prefixes = {"exhaustive": ("k_match", "k_tc_prepare"),
                "learned": ("k_mlp", "k_learned", "k_fallback", "k_match", "k_tc_prepare")}
    ms, maps = {}, {}
    for name, flags, mlp in (("exhaustive", 8 | 32, None), ("learned", 8 | 16 | 32, net)):
        p = m.ReconParams(patch=8, stride=4, knn=10, flags=flags, match_precision=2, mlp=mlp)
        r = m.Recon(m.nufft_plan(n, n, k), p, phi, comp, n2, f32(lut), b)
        r.iterate(2)
        torch.cuda.synchronize()
        m.profile_enable(True)
        m.profile_mark()
        r.iterate(5)
        torch.cuda.synchronize()
        prof = m.profile_read()
        m.profile_enable(False)
        ms[name] = sum(v[0] for kn, v in prof.items() if kn.startswith(prefixes[name])) / 5
        maps[name] = [np_(v) for v in r.maps()]
    # measured on a GB300: 0.133 ms against 0.148 ms per iteration (the
    # network's inference is 0.092 ms; features, decoding and the fallback
    # launches take the rest)
    assert ms["learned"] < 0.95 * ms["exhaustive"], ms
    mk = mask.astype(bool)
    for i in (0, 1):
        e = np.linalg.norm((maps["learned"][i] - maps["exhaustive"][i])[mk]) / np.linalg.norm(maps["exhaustive"][i][mk])
        assert e < 0.25, (i, e)
