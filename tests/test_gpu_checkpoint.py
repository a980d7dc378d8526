"""Checkpoint / resume of the loop: iterations resumed from a checkpoint in a
fresh object must follow the uninterrupted run (same coefficient images,
costs and maps up to the atomic-accumulation order of the grouped adjoint),
and a checkpoint must be refused by an object with other scales or shape."""
import numpy as np
import pytest

from gpu_util import mrf, np_, rel
from test_gpu_recon import gpu_recon, problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [0, 1])
def test_resume_matches_uninterrupted_run(mode):
    m = mrf()
    pr = problem()
    a = gpu_recon(pr, mode=mode)
    a.iterate(3)
    buf = a.checkpoint()
    info = a.info()
    ca = a.iterate(2, costs=True)
    b = gpu_recon(pr, mode=mode, a_norm=info["a_norm"], x_scale=info["x_scale"])
    b.restore(buf)
    cb = b.iterate(2, costs=True)
    tol = 1e-5
    assert rel(np_(b.alpha()), np_(a.alpha())) < tol
    np.testing.assert_allclose(cb, ca, rtol=tol)
    assert (np_(b.maps()[3]) == np_(a.maps()[3])).mean() > 0.999


def test_restore_rejects_other_scales_and_shapes():
    m = mrf()
    pr = problem()
    a = gpu_recon(pr, mode=1)
    a.iterate(1)
    buf = a.checkpoint()
    info = a.info()
    b = gpu_recon(pr, mode=1, a_norm=2 * info["a_norm"], x_scale=info["x_scale"])
    with pytest.raises(m.MRFError):
        b.restore(buf)
    c = gpu_recon(problem(K=6), mode=1, a_norm=info["a_norm"], x_scale=info["x_scale"])
    with pytest.raises(m.MRFError):
        c.restore(buf)
    with pytest.raises(m.MRFError):
        a.restore(buf[:100])
