"""Pins of the oracle's Algorithm 1 (MS-LLR) on a tiny problem."""
import numpy as np
import pytest

import synth
from oracle import dictionary, graph, nufft, recon


def tiny_problem(n=16, T=24, ns=96, K=4, seed=0, snr_db=30.0):
    t1, t2, pd, mask, _ = synth.phantom(n, seed=seed)
    fa, tr = synth.fisp_train(T, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(250, 3000, 10), synth.log_grid(25, 350, 8))
    D = dictionary.simulate(lut, fa, tr)
    phi = dictionary.subspace(D, K)
    from oracle import epg
    X = (pd.reshape(-1, 1) * epg.fisp(np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0), fa, tr))
    X = X * mask.reshape(-1, 1)
    k = synth.spiral_trajectory(n, T, ns, interleaves=6)
    grid = nufft.KBGrid(n, n, 2, 4)
    b = nufft.kb_forward(X.reshape(n, n, T).transpose(2, 0, 1), k, grid)
    sig = np.sqrt(np.mean(np.abs(b) ** 2) * 10 ** (-snr_db / 10))
    b = b + sig * synth.complex_normal(b.shape, seed=1)
    return dict(b=b, k=k, grid=grid, phi=phi, D=D, lut=lut, t1=t1, t2=t2, pd=pd, mask=mask)


@pytest.fixture(scope="module")
def prob():
    return tiny_problem()


def test_opnorm_matches_dense_svd(prob):
    P = recon.Params(patch=8, stride=4, knn=4, power_iters=60)
    r = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P)
    n, K = 16, prob["phi"].shape[1]
    cols = []
    for j in range(n * n * K):
        e = np.zeros(n * n * K, complex)
        e[j] = 1.0
        cols.append(r.A_raw(e.reshape(n, n, K) @ prob["phi"].conj().T).ravel())
    smax = np.linalg.svd(np.stack(cols, 1), compute_uv=False)[0]
    est = r.opnorm()
    # power iteration approaches the largest singular value from below
    assert est <= smax * (1 + 1e-12) and est >= smax * (1 - 1e-3)


def test_iterates_stay_on_s_and_data_term_decreases(prob):
    P = recon.Params(patch=8, stride=4, knn=4)
    r = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P).init()
    assert r.gamma > 0 and r.a > 0
    data = []
    for _ in range(4):
        r.iterate()
        np.testing.assert_allclose(r.PS(r.X), r.X, atol=1e-10 * np.abs(r.X).max())
        data.append(0.5 * np.sum(np.abs(r.A(r.X) - r.bs) ** 2))
    c = np.array(r.cost)
    assert np.all(np.isfinite(c))
    assert np.all(np.diff(data) < 0)                      # checked, not assumed
    # L and lambda1 are re-estimated every pass, so the total cost may move a
    # little, but it must not oscillate the way the printed product does
    assert c[1:].max() <= 1.05 * c[1]
    assert len(r.lam1_hist) == 5 and all(l > 0 for l in r.lam1_hist)


def test_printed_lambda1_product_oscillates(prob):
    P = recon.Params(patch=8, stride=4, knn=4, literal_lam1=True)
    r = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P).init()
    for _ in range(3):
        r.iterate()
    assert max(r.cost[1:]) > 2.0 * r.cost[1]


def test_explicit_scales_reproduce_auto(prob):
    P = recon.Params(patch=8, stride=4, knn=4)
    r1 = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P).init()
    P2 = recon.Params(patch=8, stride=4, knn=4, a_norm=r1.a, x_scale=r1.gamma)
    r2 = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P2).init()
    r1.iterate()
    r2.iterate()
    np.testing.assert_allclose(r1.X, r2.X, atol=0)


def test_stop_rule_fires():
    prob = tiny_problem(snr_db=60.0)
    P = recon.Params(patch=8, stride=4, knn=4, tol=1.0)   # any decrease under 100 % stops
    r = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P).init()
    assert r.iterate() is True
    assert r.iterate() is False


def test_noiseless_fully_sampled_loop_recovers_the_true_maps():
    """A special case of Algorithm 1 with a known answer: every tissue value is
    a dictionary atom (times a PD), every frame samples the full Cartesian
    k-space, the data are noiseless, and the regularisation weights are small.
    Then matching must find the true atom of every voxel at the start and keep
    it through the iterations, and the PD must stay close to the truth (the
    K = 6 subspace and the regularisers perturb it by a few per cent)."""
    n, T, K = 16, 24, 6
    t1m, t2m, pdm, mask, label = synth.phantom(n, seed=0)
    fa, tr = synth.fisp_train(T, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(250, 3000, 10), synth.log_grid(25, 350, 8))
    D = dictionary.simulate(lut, fa, tr)
    phi = dictionary.subspace(D, K)
    rng = np.random.default_rng(0)
    pick = {r: int(rng.integers(0, len(lut))) for r in np.unique(label)}
    idx_true = np.vectorize(pick.get)(label)
    X = pdm.ravel()[:, None] * D[idx_true.ravel()] * mask.ravel()[:, None]
    ax = np.arange(-n // 2, n // 2) * 2 * np.pi / n
    ky, kx = np.meshgrid(ax, ax, indexing="ij")
    k = np.broadcast_to(np.stack([kx.ravel(), ky.ravel()], -1), (T, n * n, 2)).copy()
    grid = nufft.KBGrid(n, n, 2, 4)
    b = nufft.kb_forward(X.reshape(n, n, T).transpose(2, 0, 1), k, grid)
    P = recon.Params(patch=8, stride=4, knn=4, lam1_0=0.01, lam2=0.01, beta=0.2)
    r = recon.MSLLR(b, k, grid, phi, D, lut, P).init()
    assert np.all(r.maps[0][mask] == idx_true[mask])
    idx, t1, t2, pd = r.run(5)
    assert np.all(idx[mask] == idx_true[mask])
    np.testing.assert_array_equal(t1[mask], lut[idx_true[mask], 0])
    np.testing.assert_array_equal(t2[mask], lut[idx_true[mask], 1])
    assert np.max(np.abs(pd[mask] - pdm[mask]) / pdm[mask]) < 0.05


def _smooth(r, X):
    """The smooth part of the objective whose gradient the bracket of Eq. 12
    is: 1/2 ||A X - b||^2 + (lambda1 / 2) Tr(Q(X) L Q(X)^H).  For a real
    symmetric L the gradient 2 df/d(conj X) of the trace is 2 Q^*(Q(X) L), so
    Eq. 12's lambda1 Q^*(Q(X) L) belongs to the trace weighted lambda1 / 2."""
    res = r.A(X) - r.bs
    return 0.5 * float(np.sum(np.abs(res) ** 2)) + 0.5 * r.lam1 * graph.trace_term(X, r.L, r.pg)


def _directional(f, X, E):
    """Central difference of f along E.  f is quadratic, so the difference is
    exact up to rounding for any step; h is taken at the scale of X."""
    h = np.linalg.norm(X) / np.linalg.norm(E)
    return (f(X + h * E) - f(X - h * E)) / (2 * h)


@pytest.mark.parametrize("lam1", [None, 0.0, 3.0])
def test_eq12_gradient_is_the_gradient_of_the_smooth_part(prob, lam1):
    """Re <gradient(X), E> equals the directional derivative of the smooth part
    along E for random directions, with lambda1 as the loop sets it, zero
    (data term alone) and large (graph term dominant), so a wrong sign or
    weight of either term fails."""
    P = recon.Params(patch=8, stride=4, knn=4)
    r = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P).init()
    if lam1 is not None:
        r.lam1 = lam1
    rng = np.random.default_rng(5)
    X = r.X + 0.3 * np.abs(r.X).max() * (rng.standard_normal(r.X.shape) + 1j * rng.standard_normal(r.X.shape))
    g = r.gradient(X)
    f = lambda Y: _smooth(r, Y)
    for _ in range(3):
        E = rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)
        d = _directional(f, X, E)
        assert float(np.real(np.vdot(g, E))) == pytest.approx(d, rel=1e-8)
    if lam1 == 3.0:
        # the graph part carries a real share of the derivative here
        ft = lambda Y: 0.5 * r.lam1 * graph.trace_term(Y, r.L, r.pg)
        assert abs(_directional(ft, X, E)) > 1e-2 * abs(_directional(f, X, E))


@pytest.mark.parametrize("mu", [1.0, 0.37])
def test_eq12_z_step_is_the_projected_gradient_step(prob, mu):
    """Z = P_S(X - mu grad): Z lies on S, and for directions E on S the step
    (X - Z) / mu has Re <(X - Z)/mu, E> equal to the smooth part's directional
    derivative along E (the iterate X is on S, so only the projected gradient
    is seen there); a wrong mu, sign or lambda1 weight fails."""
    P = recon.Params(patch=8, stride=4, knn=4, mu=mu)
    r = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P).init()
    r.lam1 = 2.0
    X = r.X
    Z = r.z_step(X)
    np.testing.assert_allclose(r.PS(Z), Z, atol=1e-10 * np.abs(Z).max())
    step = (X - Z) / mu
    f = lambda Y: _smooth(r, Y)
    rng = np.random.default_rng(9)
    for _ in range(3):
        E = r.PS(rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape))
        assert float(np.real(np.vdot(step, E))) == pytest.approx(_directional(f, X, E), rel=1e-8)
    # iterate() takes this step: with lambda2 = 0 the X update returns Z itself
    P0 = recon.Params(patch=8, stride=4, knn=4, mu=mu, lam2=0.0)
    r0 = recon.MSLLR(prob["b"], prob["k"], prob["grid"], prob["phi"], prob["D"], prob["lut"], P0).init()
    Z0 = r0.z_step(r0.X)
    r0.iterate()
    np.testing.assert_allclose(r0.X, Z0, rtol=0, atol=1e-12 * np.abs(Z0).max())
