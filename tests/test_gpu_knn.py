"""GPU parity of the exact patch kNN (the sparse graph of Eq. 7) against the
oracle's brute force: neighbour indices and squared distances bit-exact.

Integer features make every distance an exact integer, so the lists are
unique (ties to the lower index) and must agree element by element: on
patch vectors of piecewise-constant maps (many exact ties), on random
vectors with repeated rows (distance-0 ties), at the extremes of the 12-bit
range, for vector lengths of the tensor-core path (fd <= 128) and of the
SIMT path (fd > 128), ragged counts, knn from 1 to 32."""
import numpy as np
import pytest
import torch

import synth
from oracle import graph as ograph, patches as opatches
from gpu_util import dev, mrf, np_

pytestmark = pytest.mark.gpu


def _padded(F):
    """int32 device tensor [np, ld] with ld a multiple of 4, zero padding."""
    n, fd = F.shape
    ld = (fd + 3) // 4 * 4
    P = np.zeros((n, ld), np.int32)
    P[:, :fd] = F
    return torch.tensor(P, device=dev()), fd


def _check(F, knn):
    m = mrf()
    Fd, fd = _padded(F)
    nbr, d2 = m.patch_knn(Fd, knn, fd=fd)
    onbr, od2 = ograph.knn(F.astype(np.int64), knn)
    gn = np_(nbr).astype(np.int64)
    gd = np_(d2).view(np.uint32).astype(np.int64)
    np.testing.assert_array_equal(gd, od2)
    np.testing.assert_array_equal(gn, onbr)


def _map_features(n, p, stride, seed):
    t1, t2, pd, mask, label = synth.phantom(n, seed=seed)
    grid = opatches.PatchGrid(n, n, p, stride)
    return ograph.features(t1, t2, grid, 4000.0, 500.0)


@pytest.mark.parametrize("n,p,stride,knn", [(64, 8, 4, 10), (96, 4, 2, 16), (48, 5, 3, 8), (40, 1, 1, 1)])
def test_knn_phantom_patches_exact(n, p, stride, knn):
    _check(_map_features(n, p, stride, seed=n), knn)


def test_knn_full_size_patch_grid_exact():
    # 256 x 256 maps, 8 x 8 patches at stride 4: 3969 patches of 128 entries
    _check(_map_features(256, 8, 4, seed=3), 10)


@pytest.mark.parametrize("npatch,fd,knn", [(1037, 50, 16), (777, 32, 32), (300, 2, 1), (129, 128, 10),
                                           (500, 162, 10), (333, 242, 12)])
def test_knn_random_vectors_with_repeats_exact(npatch, fd, knn):
    rng = np.random.default_rng(npatch + fd)
    base = rng.integers(0, 4097, (npatch // 3 + 1, fd))
    F = base[rng.integers(0, len(base), npatch)]          # repeated rows: distance-0 ties
    F[::7] = rng.integers(0, 4097, (len(F[::7]), fd))
    _check(F, knn)


def test_knn_extreme_values_exact():
    rng = np.random.default_rng(5)
    F = np.where(rng.random((260, 128)) < 0.5, 0, 4096)    # distances up to 128 x 4096^2 = 2^31
    _check(F, 10)


def test_knn_rejects_out_of_range_and_too_few():
    m = mrf()
    F = np.zeros((200, 128), np.int64)
    F[17, 3] = 4097
    Fd, fd = _padded(F)
    with pytest.raises(m.MRFError):
        m.patch_knn(Fd, 10, fd=fd)
    Fd, fd = _padded(np.zeros((10, 8), np.int64))
    with pytest.raises(m.MRFError):
        m.patch_knn(Fd, 10, fd=fd)


def _sigma2_case(vals):
    """GPU sigma^2 of the uint32 distances vals against the oracle's median,
    bit-exact: the median of integers / 4096^2 is exact in fp64, and both
    sides round it once to float32.  The cases cover odd and even counts,
    middle values tied or not, a median bin larger than the kernel's
    shared-memory list (then read from global memory), and inputs with no
    non-zero entry."""
    v = np.asarray(vals, np.uint64).astype(np.uint32)
    d = torch.tensor(v.view(np.int32), device=dev())
    got = np_(mrf().graph_sigma2(d))[0]
    want = np.float32(ograph.sigma2(v.astype(np.float64) / float(ograph.QSCALE ** 2)))
    assert got == want, (v.size, got, want)


_SIGMA2_CASES = ["empty", "zeros", "one", "odd", "even_split", "even_tied", "all_equal", "low_bits",
                 "few_distinct", "top_bit", "large", "wide_bin", "tied_bin", "small_values"]


@pytest.mark.parametrize("case", _SIGMA2_CASES)
def test_graph_sigma2_matches_oracle_median(case):
    rng = np.random.default_rng(_SIGMA2_CASES.index(case))
    if case == "empty":
        vals = []
    elif case == "zeros":
        vals = np.zeros(1000)
    elif case == "one":
        vals = np.zeros(777); vals[500] = 123456
    elif case == "odd":
        vals = rng.integers(1, 2**31, 4001)
    elif case == "even_split":                       # the two middle values differ
        vals = np.concatenate([rng.integers(1, 1000, 3000), rng.integers(5000, 9000, 3000), np.zeros(17)])
        rng.shuffle(vals)
    elif case == "even_tied":                        # the two middle values are equal
        vals = np.concatenate([np.full(2000, 40), np.full(11, 41), np.full(1989, 7), np.zeros(50)])
        rng.shuffle(vals)
    elif case == "all_equal":
        vals = np.concatenate([np.full(3000, 98765), np.zeros(3)])
    elif case == "low_bits":                          # values that differ in the lowest bits only
        vals = 1_000_000 + rng.integers(0, 5, 10001)
    elif case == "few_distinct":                      # the tie structure of piecewise-constant maps
        vals = rng.choice(np.array([0, 4096, 8192, 16384 * 9, 2**24]), 39690, p=[0.3, 0.3, 0.2, 0.15, 0.05])
    elif case == "top_bit":                           # the full 32-bit range
        vals = rng.integers(2**31 - 10, 2**32, 5000)
    elif case == "large":
        vals = np.where(rng.random(200003) < 0.1, 0, rng.integers(1, 2**28, 200003))
    elif case == "wide_bin":                          # 10^4 distinct values in one log-scale bin
        vals = 2**20 + rng.integers(0, 2**14, 10000)
    elif case == "tied_bin":                          # more copies of the median than the list holds
        vals = np.concatenate([np.full(9000, 12345), rng.integers(1, 12345, 4000), rng.integers(12346, 10**6, 4000)])
    else:                                             # values below 128 (one value per bin)
        vals = rng.integers(0, 128, 3001)
    _sigma2_case(vals)


def test_graph_sigma2_of_workload_distances():
    """sigma^2 of the kNN distances of the full-size workload's patch graph
    (63 x 63 patches of 8 x 8, k = 10) against the oracle."""
    F = _map_features(256, 8, 4, seed=3)
    nbr, d2 = mrf().patch_knn(_padded(F)[0], 10, fd=F.shape[1])
    _sigma2_case(np_(d2).view(np.uint32).ravel())


def _seeds(kind, F, knn, rng):
    n = F.shape[0]
    if kind == "exact":
        return ograph.knn(F.astype(np.int64), knn)[0]
    if kind == "previous_maps":                     # the loop's case: the graph of other maps
        return ograph.knn(_map_features(128, 8, 4, seed=11).astype(np.int64), knn)[0]
    rows = np.stack([rng.choice(np.delete(np.arange(n), i), knn, replace=False) for i in range(n)])
    if kind == "invalid":                           # lists that give no bound, beside valid ones
        rows[0, 3] = 0                              # the row itself
        rows[1, 5] = rows[1, 2]                     # a repeated row
        rows[2, 0] = -1
        rows[3, 9] = n
        rows[4:40] = rng.integers(0, n, (36, knn))  # arbitrary values
    return rows


@pytest.mark.parametrize("kind", ["exact", "previous_maps", "random", "invalid"])
def test_seeded_knn_matches_oracle(kind):
    """A seed list (in the loop: the previous iteration's graph) only bounds
    each row's search by the largest distance to its knn distinct seeds; the
    neighbours and distances stay the oracle's whatever the seeds, including
    lists that give no bound (the row itself, a repeated row, out-of-range
    or arbitrary values).  961 patch vectors of piecewise-constant maps
    (many exact ties), k = 10."""
    F = _map_features(128, 8, 4, seed=3)
    knn = 10
    seed = _seeds(kind, F, knn, np.random.default_rng(7))
    Fd, fd = _padded(F)
    sd = torch.tensor(np.ascontiguousarray(seed, np.int32), device=dev())
    nbr, d2 = mrf().patch_knn(Fd, knn, fd=fd, seed=sd)
    onbr, od2 = ograph.knn(F.astype(np.int64), knn)
    np.testing.assert_array_equal(np_(d2).view(np.uint32).astype(np.int64), od2)
    np.testing.assert_array_equal(np_(nbr).astype(np.int64), onbr)
