"""PyTorch-facing wrappers with the same names as the C ABI (marshalling only).

Every function takes CUDA tensors, checks dtype/shape/contiguity, allocates
outputs with torch (device memory plumbing) and calls the matching ``mrf_*``
entry point on the current CUDA stream.  No arithmetic of the method happens
here.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, fields

import torch

from . import _lib
from ._lib import MRFError

__all__ = ["MRFError", "NufftPlan", "Recon", "ReconParams", "dict_subspace", "epg_fisp", "gridding_match", "match",
           "nufft_adjoint", "nufft_adjoint_subspace", "nufft_forward", "nufft_forward_subspace",
           "nufft_plan", "recon_run_host"]

MATCH_FP32, MATCH_BF16, MATCH_BF16X3, MATCH_FP8, MATCH_LITERAL_NORM2 = 0, 1, 2, 3, 0x100
RECON_LITERAL_XUPDATE, RECON_LITERAL_LAMBDA1, RECON_NO_COST, RECON_GROUPED, RECON_LEARNED, RECON_SERIAL = (
    1, 2, 4, 8, 16, 32)
RECON_EAGER = 64


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _check(t, name, dtype, shape=None):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


# ---------------------------------------------------------------------------
# NUFFT
# ---------------------------------------------------------------------------
class NufftPlan:
    """Owner of an mrf_plan (KB gridding NUFFT for T frames of ny x nx)."""

    def __init__(self, nx, ny, traj, os=2, kb_width=4):
        traj = _check(traj, "traj", torch.float32)
        if traj.dim() != 3 or traj.shape[2] != 2:
            raise ValueError("traj must be [T, ns, 2]")
        self.nx, self.ny, self.T, self.ns = nx, ny, traj.shape[0], traj.shape[1]
        self.device = traj.device
        h = C.c_void_p()
        _lib.call("mrf_nufft_plan", C.byref(h), nx, ny, self.T, self.ns, _ptr(traj), os, kb_width, _stream())
        self.handle = h

    def gather_tuning(self):
        """(entries per thread, threads per block) the spread autotuner chose; (0, 0) before tuning."""
        run, thr = C.c_int(0), C.c_int(0)
        _lib.call("mrf_nufft_gather_tuning", self.handle, C.byref(run), C.byref(thr))
        return run.value, thr.value

    def tuning(self):
        """The grouped operator's tuned choices: {"gather_run", "gather_threads",
        "strip_width"} (0 before the first grouped transform)."""
        v = [C.c_int(0) for _ in range(3)]
        _lib.call("mrf_nufft_tuning", self.handle, *[C.byref(x) for x in v])
        return dict(zip(("gather_run", "gather_threads", "strip_width"), (x.value for x in v)))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.call("mrf_nufft_destroy", h)
            except Exception:
                pass
            self.handle = None


def nufft_plan(nx, ny, traj, os=2, kb_width=4):
    return NufftPlan(nx, ny, traj, os, kb_width)


def nufft_forward(plan: NufftPlan, x, out=None):
    _check(x, "x", torch.complex64, (plan.T, plan.ny, plan.nx))
    y = out if out is not None else torch.empty((plan.T, plan.ns), dtype=torch.complex64, device=x.device)
    _check(y, "y", torch.complex64, (plan.T, plan.ns))
    _lib.call("mrf_nufft_forward", plan.handle, _ptr(x), _ptr(y), _stream())
    return y


def nufft_adjoint(plan: NufftPlan, y, out=None):
    _check(y, "y", torch.complex64, (plan.T, plan.ns))
    x = out if out is not None else torch.empty((plan.T, plan.ny, plan.nx), dtype=torch.complex64, device=y.device)
    _check(x, "x", torch.complex64, (plan.T, plan.ny, plan.nx))
    _lib.call("mrf_nufft_adjoint", plan.handle, _ptr(y), _ptr(x), _stream())
    return x


def nufft_forward_subspace(plan: NufftPlan, alpha, phi, scale=1.0, b=None, mode=0, out=None):
    K = phi.shape[1]
    _check(alpha, "alpha", torch.complex64, (plan.ny, plan.nx, K))
    _check(phi, "phi", torch.complex64, (plan.T, K))
    if b is not None:
        _check(b, "b", torch.complex64, (plan.T, plan.ns))
    y = out if out is not None else torch.empty((plan.T, plan.ns), dtype=torch.complex64, device=alpha.device)
    _lib.call("mrf_nufft_forward_subspace", plan.handle, _ptr(alpha), _ptr(phi), K, float(scale), _ptr(b),
              _ptr(y), mode, _stream())
    return y


def nufft_adjoint_subspace(plan: NufftPlan, y, phi, scale=1.0, mode=0, out=None):
    K = phi.shape[1]
    _check(y, "y", torch.complex64, (plan.T, plan.ns))
    _check(phi, "phi", torch.complex64, (plan.T, K))
    a = out if out is not None else torch.empty((plan.ny, plan.nx, K), dtype=torch.complex64, device=y.device)
    _lib.call("mrf_nufft_adjoint_subspace", plan.handle, _ptr(y), _ptr(phi), K, float(scale), _ptr(a), mode,
              _stream())
    return a


# ---------------------------------------------------------------------------
# Dictionary
# ---------------------------------------------------------------------------
def epg_fisp(t1t2, fa_deg, tr_ms, te_ms=2.94, ti_ms=20.0, inversion=True):
    _check(t1t2, "t1t2", torch.float32)
    _check(fa_deg, "fa_deg", torch.float32)
    _check(tr_ms, "tr_ms", torch.float32, fa_deg.shape)
    m, T = t1t2.shape[0], fa_deg.shape[0]
    out = torch.empty((m, T), dtype=torch.complex64, device=t1t2.device)
    _lib.call("mrf_epg_fisp", _ptr(t1t2), m, _ptr(fa_deg), _ptr(tr_ms), T, float(te_ms), float(ti_ms),
              1 if inversion else 0, _ptr(out), _stream())
    return out


def dict_subspace(D, K):
    """(phi [T, K], compressed atoms [m, K], ||d||^2 [m]) of dictionary D [m, T]."""
    _check(D, "D", torch.complex64)
    m, T = D.shape
    phi = torch.empty((T, K), dtype=torch.complex64, device=D.device)
    comp = torch.empty((m, K), dtype=torch.complex64, device=D.device)
    n2 = torch.empty((m,), dtype=torch.float32, device=D.device)
    _lib.call("mrf_dict_subspace", _ptr(D), m, T, K, _ptr(phi), _ptr(comp), _ptr(n2), _stream())
    return phi, comp, n2


def match(x, D, lut, atom_norm2=None, precision=MATCH_FP32):
    """(idx [n] int32, pd [n], t1t2 [n, 2]) of fingerprints x [n, L] against D [m, L]."""
    _check(x, "x", torch.complex64)
    _check(D, "D", torch.complex64)
    n, L = x.shape
    m = D.shape[0]
    if D.shape[1] != L:
        raise ValueError("x and D lengths differ")
    _check(lut, "lut", torch.float32, (m, 2))
    if atom_norm2 is not None:
        _check(atom_norm2, "atom_norm2", torch.float32, (m,))
    idx = torch.empty((n,), dtype=torch.int32, device=x.device)
    pd = torch.empty((n,), dtype=torch.float32, device=x.device)
    t1t2 = torch.empty((n, 2), dtype=torch.float32, device=x.device)
    _lib.call("mrf_match", _ptr(x), n, L, _ptr(D), _ptr(atom_norm2), _ptr(lut), m, int(precision), _ptr(idx),
              _ptr(pd), _ptr(t1t2), _stream())
    return idx, pd, t1t2


def gridding_match(plan, y, D, lut, atom_norm2=None, precision=MATCH_FP32, keep_rows=False):
    """The plain reconstruction: X = A^H y frame by frame, then matching of every
    voxel's T-frame fingerprint against D [m, T].  Returns (idx, pd, t1t2) as
    match() for the ny*nx voxels, plus the fingerprint rows [ny*nx, T] when
    keep_rows."""
    _check(y, "y", torch.complex64, (plan.T, plan.ns))
    _check(D, "D", torch.complex64)
    m, T = D.shape
    if T != plan.T:
        raise ValueError("D must have one column per frame")
    _check(lut, "lut", torch.float32, (m, 2))
    if atom_norm2 is not None:
        _check(atom_norm2, "atom_norm2", torch.float32, (m,))
    n = plan.nx * plan.ny
    idx = torch.empty((n,), dtype=torch.int32, device=y.device)
    pd = torch.empty((n,), dtype=torch.float32, device=y.device)
    t1t2 = torch.empty((n, 2), dtype=torch.float32, device=y.device)
    rows = torch.empty((n, T), dtype=torch.complex64, device=y.device) if keep_rows else None
    _lib.call("mrf_gridding_match", plan.handle, _ptr(y), _ptr(D), _ptr(atom_norm2), _ptr(lut), m, int(precision),
              _ptr(idx), _ptr(pd), _ptr(t1t2), _ptr(rows), _stream())
    return (idx, pd, t1t2, rows) if keep_rows else (idx, pd, t1t2)


def match_seeded(x, D, lut, cand, atom_norm2=None, precision=MATCH_BF16X3):
    """match() for repeated matching of the same rows: cand [n, 8] int32 on the
    device holds each row's seed atoms on entry (-1: none) and its tensor-core
    candidates on return; the winners are those of match() for any seeds."""
    _check(x, "x", torch.complex64)
    _check(D, "D", torch.complex64)
    n, L = x.shape
    m = D.shape[0]
    if D.shape[1] != L:
        raise ValueError("x and D lengths differ")
    _check(lut, "lut", torch.float32, (m, 2))
    _check(cand, "cand", torch.int32, (n, 8))
    if atom_norm2 is not None:
        _check(atom_norm2, "atom_norm2", torch.float32, (m,))
    idx = torch.empty((n,), dtype=torch.int32, device=x.device)
    pd = torch.empty((n,), dtype=torch.float32, device=x.device)
    t1t2 = torch.empty((n, 2), dtype=torch.float32, device=x.device)
    _lib.call("mrf_match_seeded", _ptr(x), n, L, _ptr(D), _ptr(atom_norm2), _ptr(lut), m, int(precision),
              _ptr(cand), _ptr(idx), _ptr(pd), _ptr(t1t2), _stream())
    return idx, pd, t1t2


def patch_knn(F, knn, fd=None, seed=None):
    """(nbr [np, knn] int32, d2 [np, knn] int32 holding uint32 bits) of the
    integer patch vectors F [np, ld] (entries past fd zero, ld % 4 == 0).
    seed (int32 [np, knn], optional): a previous neighbour list that bounds
    the search; the result does not depend on it."""
    _check(F, "F", torch.int32)
    npatch, ld = F.shape
    fd = ld if fd is None else int(fd)
    nbr = torch.empty((npatch, knn), dtype=torch.int32, device=F.device)
    d2 = torch.empty((npatch, knn), dtype=torch.int32, device=F.device)
    if seed is None:
        _lib.call("mrf_patch_knn", _ptr(F), npatch, fd, ld, int(knn), _ptr(nbr), _ptr(d2), _stream())
    else:
        _check(seed, "seed", torch.int32)
        if tuple(seed.shape) != (npatch, knn):
            raise ValueError(f"seed must be [{npatch}, {knn}] (got {tuple(seed.shape)})")
        _lib.call("mrf_patch_knn_seeded", _ptr(F), npatch, fd, ld, int(knn), _ptr(seed), _ptr(nbr), _ptr(d2),
                  _stream())
    return nbr, d2


def graph_sigma2(d2):
    """sigma^2 [1] float32 on the device: the median of the non-zero entries of
    the squared patch distances d2 (int32 holding uint32 bits) / 4096^2, 1 if
    none (the weight scale of the patch graph, Eq. 7)."""
    _check(d2, "d2", torch.int32)
    out = torch.empty((1,), dtype=torch.float32, device=d2.device)
    _lib.call("mrf_graph_sigma2", _ptr(d2), d2.numel(), _ptr(out), _stream())
    return out


# ---------------------------------------------------------------------------
# Algorithm 1
# ---------------------------------------------------------------------------
@dataclass
class ReconParams:
    mu: float = 1.0
    lam1_0: float = 0.1
    lam2: float = 0.1
    beta: float = 0.2
    patch: int = 8
    stride: int = 4
    knn: int = 10
    power_iters: int = 20
    pd_target: float = 100.0
    a_norm: float = 0.0
    x_scale: float = 0.0
    flags: int = 0
    match_precision: int = MATCH_FP32
    mlp: object = None          # Mlp for RECON_LEARNED (kept alive by the Recon)

    def as_c(self):
        vals = [getattr(self, f.name) for f in fields(self) if f.name != "mlp"]
        return _lib.ReconParams(*vals, self.mlp.handle.value if self.mlp is not None else None)


class Mlp:
    """Owner of an mrf_mlp: the learned matcher's 20-256-256-256-3 GELU network."""

    N_PARAMS = 137731

    def __init__(self, params, decode, max_batch=1024):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.N_PARAMS:
            raise ValueError(f"expected {self.N_PARAMS} parameters")
        d = np.ascontiguousarray(decode, dtype=np.float32)
        self.decode = tuple(float(v) for v in d)
        self.max_batch = int(max_batch)
        h = C.c_void_p()
        _lib.call("mrf_mlp_create", C.byref(h), p.ctypes.data, p.size, d.ctypes.data, self.max_batch)
        self.handle = h

    def params(self):
        """(FP32 master parameters, BF16 values used in the products) as NumPy arrays."""
        import numpy as np
        a = np.empty(self.N_PARAMS, np.float32)
        b = np.empty(self.N_PARAMS, np.float32)
        _lib.call("mrf_mlp_get_params", self.handle, a.ctypes.data, b.ctypes.data)
        return a, b

    def grad(self, x, t):
        _check(x, "x", torch.float32)
        _check(t, "t", torch.float32, (x.shape[0], 3))
        g = torch.empty(self.N_PARAMS, dtype=torch.float32, device=x.device)
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        _lib.call("mrf_mlp_grad", self.handle, _ptr(x), _ptr(t), x.shape[0], _ptr(g), _ptr(loss), _stream())
        return g, loss

    def train_step(self, x, t, lr, loss=None):
        _lib.call("mrf_mlp_train_step", self.handle, _ptr(x), _ptr(t), x.shape[0], float(lr), _ptr(loss),
                  _stream())

    def set_engine(self, tensor_cores=True):
        _lib.call("mrf_mlp_set_engine", self.handle, 1 if tensor_cores else 0)

    def check(self):
        _lib.call("mrf_mlp_check", self.handle, _stream())

    def infer(self, x):
        _check(x, "x", torch.float32)
        y = torch.empty((x.shape[0], 3), dtype=torch.float32, device=x.device)
        _lib.call("mrf_mlp_infer", self.handle, _ptr(x), x.shape[0], _ptr(y), _stream())
        return y

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.call("mrf_mlp_destroy", h)
            except Exception:
                pass
            self.handle = None


def mlp_training_set(sig, t1t2, rho, snr_db, noise, phi, ranges):
    """(x [n, 2K], y [n, 3]) training fingerprints from noiseless signals sig [n, T]."""
    import numpy as np
    n, T = sig.shape
    K = phi.shape[1]
    _check(sig, "sig", torch.complex64)
    _check(t1t2, "t1t2", torch.float32, (n, 2))
    _check(rho, "rho", torch.float32, (n,))
    _check(snr_db, "snr_db", torch.float32, (n,))
    _check(noise, "noise", torch.complex64, (n, K))
    _check(phi, "phi", torch.complex64, (T, K))
    r = np.ascontiguousarray(ranges, dtype=np.float32)
    x = torch.empty((n, 2 * K), dtype=torch.float32, device=sig.device)
    y = torch.empty((n, 3), dtype=torch.float32, device=sig.device)
    _lib.call("mrf_mlp_training_set", _ptr(sig), _ptr(t1t2), _ptr(rho), _ptr(snr_db), _ptr(noise), n, T, _ptr(phi),
              K, r.ctypes.data, _ptr(x), _ptr(y), _stream())
    return x, y


def train_matcher(params0, draws, fa_deg, tr_ms, phi, ranges, epochs=3, batch=1024, lr=(1e-3, 1e-5), chunk=65536,
                  perm_seed=0):
    """Train the learned matcher on fingerprints synthesised on the GPU.

    draws = (t1t2 [n, 2], rho [n], snr_db [n], noise [n, K] complex) as NumPy
    arrays (the caller's random draws); params0: initial packed parameters.
    The set is simulated chunk by chunk (EPG signals, subspace projection,
    noise, normalisation) and kept on the device; training runs `epochs`
    passes of Adam over shuffled batches with a cosine decay from lr[0] to
    lr[1].  Returns (Mlp, per-epoch mean batch losses)."""
    import math
    import numpy as np
    t1t2, rho, snr, noise = draws
    n = t1t2.shape[0]
    dev = phi.device
    xs, ys = [], []
    for c0 in range(0, n, chunk):
        c1 = min(n, c0 + chunk)
        tt = torch.tensor(np.ascontiguousarray(t1t2[c0:c1]), dtype=torch.float32, device=dev)
        sig = epg_fisp(tt, fa_deg, tr_ms)
        x, y = mlp_training_set(sig, tt, torch.tensor(rho[c0:c1], dtype=torch.float32, device=dev),
                                torch.tensor(snr[c0:c1], dtype=torch.float32, device=dev),
                                torch.tensor(np.ascontiguousarray(noise[c0:c1]), dtype=torch.complex64, device=dev),
                                phi, ranges)
        xs.append(x)
        ys.append(y)
        del sig
    X, Y = torch.cat(xs), torch.cat(ys)
    net = Mlp(params0, ranges, max_batch=batch)
    gen = torch.Generator(device=dev)
    gen.manual_seed(perm_seed)
    steps = epochs * (n // batch)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    acc = torch.zeros(1, dtype=torch.float64, device=dev)
    history, step = [], 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen, device=dev)
        acc.zero_()
        for b0 in range(0, n - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            rate = lr[1] + 0.5 * (lr[0] - lr[1]) * (1.0 + math.cos(math.pi * step / max(steps - 1, 1)))
            net.train_step(xb, yb, rate, loss)
            acc += loss
            step += 1
        history.append(float(acc) / (n // batch))
    return net, history


class Recon:
    """Owner of an mrf_recon: Algorithm 1 state on the GPU."""

    def __init__(self, plan: NufftPlan, params: ReconParams, phi, dict_c, atom_norm2, lut, b):
        K = phi.shape[1]
        m = dict_c.shape[0]
        _check(phi, "phi", torch.complex64, (plan.T, K))
        _check(dict_c, "dict_c", torch.complex64, (m, K))
        _check(atom_norm2, "atom_norm2", torch.float32, (m,))
        _check(lut, "lut", torch.float32, (m, 2))
        _check(b, "b", torch.complex64, (plan.T, plan.ns))
        self.plan, self.K = plan, K
        self._keep = (phi, dict_c, atom_norm2, lut, b, params.mlp)      # the C object borrows these
        self._params = params.as_c()
        h = C.c_void_p()
        _lib.call("mrf_recon_create", C.byref(h), plan.handle, C.byref(self._params), _ptr(phi), K, _ptr(dict_c),
                  _ptr(atom_norm2), _ptr(lut), m, _ptr(b), _stream())
        self.handle = h

    def iterate(self, n=1, costs=False):
        buf = (C.c_double * n)() if costs else None
        _lib.call("mrf_recon_iter", self.handle, n, buf if costs else None, _stream())
        return list(buf) if costs else None

    def maps(self):
        p = self.plan
        dev = self._keep[0].device
        t1 = torch.empty((p.ny, p.nx), dtype=torch.float32, device=dev)
        t2 = torch.empty_like(t1)
        pd = torch.empty_like(t1)
        idx = torch.empty((p.ny, p.nx), dtype=torch.int32, device=dev)
        _lib.call("mrf_recon_maps", self.handle, _ptr(t1), _ptr(t2), _ptr(pd), _ptr(idx), _stream())
        return t1, t2, pd, idx

    def alpha(self):
        p = self.plan
        a = torch.empty((p.ny, p.nx, self.K), dtype=torch.complex64, device=self._keep[0].device)
        _lib.call("mrf_recon_alpha", self.handle, _ptr(a), _stream())
        return a

    def checkpoint(self):
        """The loop state as a NumPy uint8 array (see mrf_recon_checkpoint)."""
        import numpy as np
        n = C.c_size_t(0)
        _lib.call("mrf_recon_checkpoint_size", self.handle, C.byref(n))
        buf = np.empty(n.value, np.uint8)
        _lib.call("mrf_recon_checkpoint", self.handle, buf.ctypes.data, n.value, _stream())
        return buf

    def restore(self, buf):
        import numpy as np
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _lib.call("mrf_recon_restore", self.handle, buf.ctypes.data, buf.size, _stream())

    def svt_stats(self):
        """(sweeps, rotations, patch_svts): Jacobi sweeps and column-pair rotations
        the SVT step executed since create, summed over patches, and patches x
        SVT launches."""
        vals = [C.c_double() for _ in range(3)]
        _lib.call("mrf_recon_svt_stats", self.handle, *[C.byref(v) for v in vals], _stream())
        return tuple(v.value for v in vals)

    def info(self):
        vals = [C.c_double() for _ in range(4)]
        _lib.call("mrf_recon_info", self.handle, *[C.byref(v) for v in vals], _stream())
        return dict(zip(["a_norm", "x_scale", "lam1", "sigma2"], [v.value for v in vals]))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.call("mrf_recon_destroy", h)
            except Exception:
                pass
            self.handle = None


def recon_run_host(plan, params, phi, dict_c, atom_norm2, lut, b_host, iters, costs=False):
    """One reconstruction from host k-space to host maps through
    mrf_recon_run_host: b_host is a CPU complex64 tensor [T, ns] (pinned for an
    asynchronous copy); returns CPU float32 maps (t1, t2, pd) [ny, nx] (and the
    per-iteration costs)."""
    K = phi.shape[1]
    m = dict_c.shape[0]
    _check(phi, "phi", torch.complex64, (plan.T, K))
    _check(dict_c, "dict_c", torch.complex64, (m, K))
    _check(atom_norm2, "atom_norm2", torch.float32, (m,))
    _check(lut, "lut", torch.float32, (m, 2))
    if not isinstance(b_host, torch.Tensor) or b_host.is_cuda or b_host.dtype != torch.complex64 \
            or not b_host.is_contiguous() or tuple(b_host.shape) != (plan.T, plan.ns):
        raise ValueError(f"b_host must be a contiguous CPU complex64 tensor of shape {(plan.T, plan.ns)}")
    pin = b_host.is_pinned()
    maps = [torch.empty((plan.ny, plan.nx), dtype=torch.float32, pin_memory=pin) for _ in range(3)]
    cost = (C.c_double * max(iters, 1))() if costs else None
    prm = params.as_c()
    _lib.call("mrf_recon_run_host", plan.handle, C.byref(prm), _ptr(phi), K, _ptr(dict_c), _ptr(atom_norm2),
              _ptr(lut), m, _ptr(b_host), int(iters), _ptr(maps[0]), _ptr(maps[1]), _ptr(maps[2]), cost,
              _stream())
    return (tuple(maps), list(cost)[:iters]) if costs else tuple(maps)


class Batch:
    """Owner of an mrf_batch: slices (Recon objects with their own plans and one
    shared dictionary) advanced together; every iteration after the first is
    one CUDA graph launch.  Keeps the Recon objects alive."""

    def __init__(self, recons):
        recons = list(recons)
        if not recons:
            raise ValueError("a batch needs at least one slice")
        self.recons = recons
        arr = (C.c_void_p * len(recons))(*[r.handle.value for r in recons])
        h = C.c_void_p()
        _lib.call("mrf_batch_create", C.byref(h), arr, len(recons), _stream())
        self.handle = h

    def iterate(self, n=1):
        _lib.call("mrf_batch_iter", self.handle, int(n), _stream())

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                _lib.call("mrf_batch_destroy", h)
            except Exception:
                pass
            self.handle = None


def wait_selftest(polls=1000):
    """Run the bounded-wait self-test; raises MRFError (status MRF_ETIMEOUT) as designed."""
    _lib.call("mrf_wait_selftest", int(polls), _stream())


# ---------------------------------------------------------------------------
# Tracing
# ---------------------------------------------------------------------------
def launch_count():
    """Kernels launched by libmrf.so since it was loaded."""
    return int(_lib.load().mrf_launch_count())


def profile_enable(on=True):
    _lib.call("mrf_profile_enable", 1 if on else 0)


def profile_mark():
    """Boundary on the current stream: the next kernel's interval starts here."""
    _lib.call("mrf_profile_mark", _stream())


def profile_read():
    """{kernel name: (total ms, timed launches)} of the marks recorded so far."""
    lib = _lib.load()
    n = lib.mrf_profile_collect()
    if n < 0:
        raise MRFError("mrf_profile_collect", 3, lib.mrf_last_error().decode())
    out = {}
    buf = C.create_string_buffer(128)
    ms = C.c_double()
    cnt = C.c_longlong()
    for i in range(n):
        _lib.call("mrf_profile_entry", i, buf, 128, C.byref(ms), C.byref(cnt))
        out[buf.value.decode()] = (ms.value, cnt.value)
    return out
