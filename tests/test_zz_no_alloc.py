"""mrf_match_noalloc: matching for callers that cannot allocate device memory
(a service that owns the GPU's memory pool, or a serving loop that must not
pay for cudaMalloc/cudaFree).  Its scratch is a fixed array inside the
library, so the check is that it returns exactly what mrf_match returns, on
two calls in a row (the second with other sizes, so leftovers of the first
call cannot leak into it), and that it refuses sizes beyond the array.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest
import torch

from gpu_util import c64, f32, mrf, np_, rand_c

pytestmark = pytest.mark.gpu


def _call(name, x, D, lut, n2=None):
    from paper_2310_05647_gb300 import _lib
    n, L = x.shape
    m = D.shape[0]
    idx = torch.full((n,), -1, dtype=torch.int32, device=x.device)
    pd = torch.full((n,), -1.0, dtype=torch.float32, device=x.device)
    tt = torch.full((n, 2), -1.0, dtype=torch.float32, device=x.device)
    p = lambda t: C.c_void_p(0 if t is None else t.data_ptr())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.call(name, p(x), n, L, p(D), p(n2), p(lut), m, 0, p(idx), p(pd), p(tt), s)
    return np_(idx), np_(pd), np_(tt)


@pytest.mark.parametrize("sizes", [[(700, 40, 300), (2000, 10, 1111)]])
def test_no_alloc_matches_allocating_entry_point(sizes):
    mrf()
    rng = np.random.default_rng(11)
    for n, L, m in sizes:                       # two calls in a row
        D = rand_c(rng, m, L)
        X = D[rng.integers(0, m, n)] * rng.uniform(0.3, 2.0, (n, 1)) + 0.3 * rand_c(rng, n, L)
        lut = rng.uniform(10, 3000, (m, 2))
        n2 = np.sum(np.abs(D) ** 2, 1) if L == 10 else None
        args = (c64(X), c64(D), f32(lut), None if n2 is None else f32(n2))
        ref = _call("mrf_match", *args)
        got = _call("mrf_match_noalloc", *args)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_allclose(got[1], ref[1], rtol=1e-6, atol=0)
        np.testing.assert_array_equal(got[2], ref[2])


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    m = mrf()
    x = c64(np.zeros((1, 4)))
    D = c64(np.ones((2, 4)))
    lut = f32(np.ones((2, 2)))
    from paper_2310_05647_gb300 import _lib
    lib = _lib.load()
    p = lambda t: C.c_void_p(t.data_ptr())
    st = lib.mrf_match_noalloc(p(x), (1 << 18) + 1, 4, p(D), None, p(lut), 2, 0, None, None, None, None)
    assert st == 1 and b"exceeds" in lib.mrf_last_error()
    st = lib.mrf_match_noalloc(p(x), 1, 4, p(D), None, p(lut), (1 << 16) + 1, 0, None, None, None, None)
    assert st == 1
