"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import numpy as np
import pytest
import torch

_built = False


def mrf():
    """The package with libmrf.so built; fails (does not skip) when it cannot load."""
    global _built
    if not _built:
        from paper_2310_05647_gb300 import build
        build.build()
        _built = True
    import paper_2310_05647_gb300 as m
    return m


def dev():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    return torch.device("cuda:0")


def c64(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.complex64, device=dev())


def f32(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev())


def np_(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def as_f32_inputs(*arrs):
    """Round inputs to the precision the GPU receives, so both sides see the same values."""
    out = []
    for a in arrs:
        a = np.asarray(a)
        out.append(a.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(a)
                   else a.astype(np.float32).astype(np.float64))
    return out
