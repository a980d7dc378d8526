"""GPU parity of the multi-frame NUFFT (Eq. 1) against the FP64 oracle.

Tolerance: relative L2 <= 1e-4 in FP32 against the oracle's KB gridding with
the same kernel width and oversampling (FP32 rounding of the FFT and the
kernel weights is ~1e-6; the bound leaves headroom for 512-point FFTs)."""
import numpy as np
import pytest

import synth
from oracle import nufft as onufft
from gpu_util import as_f32_inputs, c64, dev, f32, mrf, np_, rand_c, rel

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _case(n, T, ns, interleaves, width=4, seed=0):
    rng = np.random.default_rng(seed)
    if interleaves < 0:
        k = rng.uniform(-np.pi, np.pi, (T, ns, 2))
    else:
        k = synth.spiral_trajectory(n, T, ns, interleaves)
    x = rand_c(rng, T, n, n)
    y = rand_c(rng, T, ns)
    k, x, y = as_f32_inputs(k, x, y)
    return k, x, y, onufft.KBGrid(n, n, 2, width)


@pytest.mark.parametrize("n,T,ns,il,w", [
    (32, 5, 300, -1, 4),      # G = 64, random samples, every frame distinct
    (32, 7, 257, 3, 6),       # W = 6, ragged sample count, shared trajectories
    (64, 9, 512, 0, 4),       # G = 128, golden-angle spiral
    (128, 4, 1024, 2, 4),     # G = 256
    (256, 3, 2048, 48, 4),    # G = 512, the 256^2 spiral arm of 2048 samples
    (192, 4, 1536, 3, 4),     # G = 384 = 3 x 128: the mixed-radix FFT (192^2 serving slices)
    (48, 5, 400, -1, 6),      # G = 96 = 3 x 32 is not a supported grid: checked below
    (32, 600, 2048, -1, 4),   # 600 distinct frames x 2048 samples x 16 taps: beyond the sorted
                              # spread table's 2^24 entries, so the adjoint takes the atomic spread
])
def test_forward_adjoint_match_oracle(n, T, ns, il, w):
    m = mrf()
    k, x, y, grid = _case(n, T, ns, il, w)
    if 2 * n == 96:
        with pytest.raises(m.MRFError):
            m.nufft_plan(n, n, f32(k), kb_width=w)
        return
    plan = m.nufft_plan(n, n, f32(k), kb_width=w)
    yg = np_(m.nufft_forward(plan, c64(x)))
    assert rel(yg, onufft.kb_forward(x, k, grid)) < TOL
    xg = np_(m.nufft_adjoint(plan, c64(y)))
    assert rel(xg, onufft.kb_adjoint(y, k, grid)) < TOL


def test_adjointness_on_gpu():
    m = mrf()
    k, x, y, _ = _case(64, 6, 700, 0)
    plan = m.nufft_plan(64, 64, f32(k))
    ax = np_(m.nufft_forward(plan, c64(x)))
    ahy = np_(m.nufft_adjoint(plan, c64(y)))
    lhs, rhs = np.vdot(ax, y), np.vdot(x, ahy)
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_w6_against_exact_nudft():
    m = mrf()
    k, x, y, _ = _case(32, 3, 400, -1)
    plan = m.nufft_plan(32, 32, f32(k), kb_width=6)
    assert rel(np_(m.nufft_forward(plan, c64(x))), onufft.nudft_forward(x, k)) < 1e-4
    assert rel(np_(m.nufft_adjoint(plan, c64(y))), onufft.nudft_adjoint(y, k, 32, 32)) < 1e-4


def test_edge_samples_and_single_sample():
    m = mrf()
    n = 32
    k = np.array([[[-np.pi, -np.pi], [-np.pi, 0.0], [0.0, 0.0], [np.pi * 0.999, -np.pi],
                   [2 * np.pi * 3 / 64, 2 * np.pi * 5 / 64]]])
    rng = np.random.default_rng(3)
    k, x = as_f32_inputs(k, rand_c(rng, 1, n, n))
    grid = onufft.KBGrid(n, n, 2, 4)
    plan = m.nufft_plan(n, n, f32(k))
    assert rel(np_(m.nufft_forward(plan, c64(x))), onufft.kb_forward(x, k, grid)) < TOL
    k1 = k[:, 2:3]
    plan1 = m.nufft_plan(n, n, f32(k1))
    y1 = np.array([[1.0 + 2.0j]])
    assert rel(np_(m.nufft_adjoint(plan1, c64(y1))), onufft.kb_adjoint(y1, k1, grid)) < TOL


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,T,ns,il,K", [(32, 24, 200, 4, 4), (64, 40, 512, 0, 10), (128, 30, 1024, 6, 16)])
def test_subspace_forms_match_oracle(mode, n, T, ns, il, K):
    m = mrf()
    rng = np.random.default_rng(5)
    k = synth.spiral_trajectory(n, T, ns, il)
    phi, _ = np.linalg.qr(rand_c(rng, T, K))
    alpha = rand_c(rng, n, n, K)
    b = rand_c(rng, T, ns)
    r = rand_c(rng, T, ns)
    k, phi, alpha, b, r = as_f32_inputs(k, phi, alpha, b, r)
    grid = onufft.KBGrid(n, n, 2, 4)
    scale = 0.37
    X = alpha @ phi.conj().T                                   # [n, n, T]
    y0 = scale * onufft.kb_forward(np.moveaxis(X, -1, 0), k, grid) - b
    a0 = scale * np.moveaxis(onufft.kb_adjoint(r, k, grid), 0, -1) @ phi
    plan = m.nufft_plan(n, n, f32(k))
    yg = np_(m.nufft_forward_subspace(plan, c64(alpha), c64(phi), scale, c64(b), mode=mode))
    assert rel(yg, y0) < TOL
    ag = np_(m.nufft_adjoint_subspace(plan, c64(r), c64(phi), scale, mode=mode))
    assert rel(ag, a0) < TOL


def test_bad_arguments_raise():
    m = mrf()
    k = f32(np.zeros((2, 4, 2)))
    with pytest.raises(m.MRFError):
        m.nufft_plan(48, 48, k)                                # grid 96 unsupported
    with pytest.raises(m.MRFError):
        m.nufft_plan(32, 32, f32(np.full((2, 4, 2), 4.0)))     # outside [-pi, pi]


@pytest.mark.parametrize("mode", [0, 1])
def test_subspace_forms_on_the_384_grid(mode):
    """Both operator forms on a 192^2 image (G = 384, mixed radix 3 x 2^7)
    against the oracle applied to the expanded frames."""
    m = mrf()
    n, T, ns, K = 192, 12, 1536, 4
    rng = np.random.default_rng(3)
    k = synth.spiral_trajectory(n, T, ns, 4)
    phi, _ = np.linalg.qr(rand_c(rng, T, K))
    alpha = rand_c(rng, n, n, K)
    y = rand_c(rng, T, ns)
    k, phi, alpha, y = as_f32_inputs(k, phi, alpha, y)
    grid = onufft.KBGrid(n, n, 2, 4)
    plan = m.nufft_plan(n, n, f32(k))
    yg = np_(m.nufft_forward_subspace(plan, c64(alpha), c64(phi), 1.0, mode=mode))
    frames = np.einsum("yxk,tk->tyx", alpha, phi.conj())
    assert rel(yg, onufft.kb_forward(frames, k, grid)) < TOL
    ag = np_(m.nufft_adjoint_subspace(plan, c64(y), c64(phi), 1.0, mode=mode))
    ao = np.einsum("tyx,tk->yxk", onufft.kb_adjoint(y, k, grid), phi)
    assert rel(ag, ao) < TOL
