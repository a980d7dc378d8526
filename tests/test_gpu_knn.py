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
