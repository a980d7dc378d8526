"""Pins of the oracle's patch operators, graph weights and Laplacian (Eq. 6-10)."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import graph, patches


def test_three_node_laplacian_layout():
    w12, w13, w23 = 0.3, 0.7, 0.2
    W = np.array([[0, w12, w13], [w12, 0, w23], [w13, w23, 0]])
    expect = np.array([[w12 + w13, -w12, -w13],
                       [-w12, w12 + w23, -w23],
                       [-w13, -w23, w13 + w23]])
    np.testing.assert_allclose(graph.laplacian(W), expect, rtol=0, atol=0)


def test_patch_origins_and_coverage():
    np.testing.assert_array_equal(patches.origins(128, 11, 5)[-2:], [115, 117])
    pg = patches.PatchGrid(256, 256, 8, 4)
    assert pg.count == 63 * 63
    cnt = pg.coverage()
    assert cnt[0, 0] == 1 and cnt[5, 5] == 4 and cnt[0, 5] == 2 and cnt.min() >= 1


def test_patch_adjoint():
    rng = np.random.default_rng(0)
    pg = patches.PatchGrid(20, 17, 6, 3)
    x = rng.standard_normal((20, 17, 3)) + 1j * rng.standard_normal((20, 17, 3))
    y = rng.standard_normal((pg.count, 36, 3)) + 1j * rng.standard_normal((pg.count, 36, 3))
    assert np.vdot(pg.extract(x), y) == pytest.approx(np.vdot(x, pg.adjoint(y)), rel=1e-12)


def test_knn_matches_kdtree():
    rng = np.random.default_rng(1)
    F = rng.standard_normal((200, 7))
    nbr, d2 = graph.knn(F, 5)
    dist, _ = cKDTree(F).query(F, k=6)
    np.testing.assert_allclose(np.sqrt(d2), dist[:, 1:], rtol=1e-12)
    assert not np.any(nbr == np.arange(200)[:, None])


def test_knn_ties_take_lower_index():
    F = np.zeros((6, 2))
    F[5] = 1.0
    nbr, d2 = graph.knn(F, 3)
    np.testing.assert_array_equal(nbr[0], [1, 2, 3])
    np.testing.assert_array_equal(nbr[4], [0, 1, 2])
    assert graph.sigma2(d2) == pytest.approx(2.0)         # only the non-zero distances
    assert graph.sigma2(np.zeros((3, 2))) == 1.0


def test_sigma2_is_the_median_of_the_nonzero_distances_brute_force():
    """sigma^2 against a pure-Python median (sorted list; the mean of the two
    middle values for an even count) of the non-zero entries, on small integer
    sets with zeros, ties, odd and even counts."""
    rng = np.random.default_rng(11)
    for trial in range(200):
        d = rng.integers(0, 6, int(rng.integers(1, 15))).astype(float)
        nz = sorted(v for v in d.tolist() if v > 0)
        if not nz:
            want = 1.0
        elif len(nz) % 2:
            want = nz[len(nz) // 2]
        else:
            want = 0.5 * (nz[len(nz) // 2 - 1] + nz[len(nz) // 2])
        assert graph.sigma2(d) == want, (trial, d)


def test_laplacian_properties():
    rng = np.random.default_rng(2)
    F = rng.standard_normal((40, 4))
    nbr, d2 = graph.knn(F, 6)
    W = graph.adjacency(nbr, d2, graph.sigma2(d2))
    L = graph.laplacian(W)
    np.testing.assert_allclose(L, L.T, atol=0)
    np.testing.assert_allclose(L.sum(axis=1), 0, atol=1e-12)
    assert np.linalg.eigvalsh(L).min() > -1e-12
    assert L.max() == pytest.approx(np.diag(L).max())


def test_trace_form_equals_pairwise_form():
    # Eq. 8 <-> Eq. 9: Tr(Q L Q^H) = 1/2 sum_ij W_ij ||Q_i - Q_j||^2
    rng = np.random.default_rng(3)
    pg = patches.PatchGrid(12, 12, 4, 4)
    X = rng.standard_normal((12, 12, 3)) + 1j * rng.standard_normal((12, 12, 3))
    W = rng.uniform(0, 1, (pg.count, pg.count))
    W = 0.5 * (W + W.T)
    np.fill_diagonal(W, 0)
    L = graph.laplacian(W)
    Q = pg.extract(X)
    pair = sum(W[i, j] * np.sum(np.abs(Q[i] - Q[j]) ** 2)
               for i in range(pg.count) for j in range(pg.count))
    assert graph.trace_term(X, L, pg) == pytest.approx(0.5 * pair, rel=1e-12)


def test_trace_from_forward_knn_lists_alone():
    """With W = (K + K^T)/2 of a kNN graph, Tr(Q L Q^H) = sum_j deg_j |Q_j|^2 -
    sum_j sum_{i in N(j)} w_ji Re <Q_j, Q_i>: the reverse half of W adds the
    same sum as the forward half (the form the device's cost trace uses)."""
    rng = np.random.default_rng(9)
    pg = patches.PatchGrid(20, 20, 4, 2)
    X = rng.standard_normal((20, 20, 3)) + 1j * rng.standard_normal((20, 20, 3))
    F = rng.integers(0, 50, (pg.count, 6))
    nbr, d2 = graph.knn(F, 5)
    w = np.exp(-d2 / graph.sigma2(d2.astype(np.float64)))
    L = graph.laplacian(graph.adjacency(nbr, d2, graph.sigma2(d2.astype(np.float64))))
    deg = np.diag(L)
    Q = pg.extract(X).reshape(pg.count, -1)
    fwd = sum(deg[j] * np.vdot(Q[j], Q[j]).real for j in range(pg.count)) - sum(
        w[j, q] * np.vdot(Q[j], Q[nbr[j, q]]).real for j in range(pg.count) for q in range(nbr.shape[1]))
    assert graph.trace_term(X, L, pg) == pytest.approx(fwd, rel=1e-12)


def test_graph_term_is_gradient_of_trace():
    # d/de Tr(Q(X+eE) L Q(X+eE)^H) at e=0 equals 2 Re <E, Q^*(Q(X) L)>
    rng = np.random.default_rng(4)
    pg = patches.PatchGrid(10, 10, 4, 2)
    X = rng.standard_normal((10, 10, 2)) + 1j * rng.standard_normal((10, 10, 2))
    E = rng.standard_normal((10, 10, 2)) + 1j * rng.standard_normal((10, 10, 2))
    W = rng.uniform(0, 1, (pg.count, pg.count))
    W = 0.5 * (W + W.T)
    np.fill_diagonal(W, 0)
    L = graph.laplacian(W)
    h = 1e-6
    fd = (graph.trace_term(X + h * E, L, pg) - graph.trace_term(X - h * E, L, pg)) / (2 * h)
    an = 2 * np.real(np.vdot(E, graph.graph_term(X, L, pg)))
    assert fd == pytest.approx(an, rel=1e-6)


def test_features_scale_and_fixed_point():
    pg = patches.PatchGrid(8, 8, 4, 4)
    t1 = np.full((8, 8), 1000.0)
    t2 = np.full((8, 8), 50.0)
    t2[0, 0] = 100.0 * 3 / 8192                 # exactly half an LSB: rounds to even (0)
    t2[0, 1] = 100.0 * 5 / 8192                 # 2.5 LSB -> 2
    F = graph.features(t1, t2, pg, 2000.0, 100.0)
    assert F.shape == (4, 32) and F.dtype == np.int64
    assert F[0, 0] == 2048 and F[0, 2] == 2048
    assert F[0, 1] == 2 and F[0, 3] == 2
    assert F[1, 1] == 2048


def test_integer_distances_are_exact_ties():
    # two candidates at the same distance through different voxels tie exactly
    F = np.array([[0, 0, 0], [3, 0, 0], [0, 3, 0], [0, 0, 2]], dtype=np.int64)
    nbr, d2 = graph.knn(F, 3)
    np.testing.assert_array_equal(nbr[0], [3, 1, 2])
    np.testing.assert_array_equal(d2[0], [4, 9, 9])


def test_kth_distance_is_bounded_by_any_k_other_rows():
    """Any k distinct rows other than i are candidates for row i, so the
    k-th smallest distance of the exact kNN is at most the largest distance
    from row i to them: the bound with which a previous graph seeds the
    search.  Checked against the graph of other features (a stale graph),
    random rows and the exact lists themselves (where it is attained),
    and brute force on the same rows."""
    rng = np.random.default_rng(4)
    k = 6
    F = rng.integers(0, 40, (300, 5))
    F[100:160] = F[100]                               # a flat block: exact ties
    nbr, d2 = graph.knn(F, k)
    brute = np.sort(((F[:, None, :] - F[None, :, :]) ** 2).sum(-1) + np.diag(np.full(len(F), 10**9)), axis=1)
    np.testing.assert_array_equal(d2, brute[:, :k])
    stale, _ = graph.knn(rng.integers(0, 40, (300, 5)), k)
    rand = np.stack([rng.choice(np.delete(np.arange(300), i), k, replace=False) for i in range(300)])
    for seeds in (stale, rand, nbr):
        assert all(len(set(r)) == k and i not in r for i, r in enumerate(seeds))
        bound = ((F[:, None, :] - F[seeds]) ** 2).sum(-1).max(axis=1)
        assert np.all(d2[:, k - 1] <= bound)
    np.testing.assert_array_equal(((F[:, None, :] - F[nbr]) ** 2).sum(-1).max(axis=1), d2[:, k - 1])
