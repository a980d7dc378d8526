"""Seeded synthetic inputs for MR fingerprinting reconstruction.

This module holds only input generation: tissue maps, the flip-angle /
repetition-time train, k-space trajectories, unit-variance complex noise and
the (T1, T2) grids a dictionary is simulated on.  It contains none of the
reconstruction arithmetic (no Bloch/EPG simulation, no NUFFT, no matching), so
both the CPU oracle and the GPU path can draw the same inputs from it.

The paper's simulation data (ground-truth maps from prior work, Sec. IV-A) and
its in-vivo scan are not available; these generators stand in for them with
the same structure: a piecewise-constant numerical phantom, a FISP train with
TE = 2.94 ms (Sec. IV), one variable-density spiral interleaf per frame, and a
log-spaced (T1, T2) dictionary grid that omits T1 < T2 (the rule of Sec. IV's
dictionary discretisation).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

GOLDEN_ANGLE = 2.0 * math.pi * (1.0 - 2.0 / (1.0 + math.sqrt(5.0)))  # 137.508 deg
TE_MS = 2.94   # echo time of the FISP sequence (Sec. IV)
TI_MS = 20.0   # inversion delay before the train (not given by the paper)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    n: int                 # image is n x n
    frames: int            # T (the paper's L)
    ns: int                # samples per frame
    interleaves: int       # distinct spiral interleaves (0 = golden-angle per frame)
    os: int = 2            # grid oversampling
    kb_width: int = 4      # Kaiser-Bessel width W
    t1_range: tuple = (300.0, 2500.0)
    t2_range: tuple = (30.0, 300.0)
    n_t1: int = 50
    n_t2: int = 30
    rank: int = 0          # temporal subspace rank K (0 = full T)
    snr_db: float = 30.0
    phantom_seed: int = 0
    noise_seed: int = 1
    tr_seed: int = 2
    patch: int = 8
    stride: int = 4
    knn: int = 10
    iters: int = 10
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    # 64x64 phantom, T=100, one golden-angle-rotated spiral of 512 samples per
    # frame, 50 x 30 log-spaced atoms; A^H gridding then exhaustive matching.
    "mrf64_t100": Workload("mrf64_t100", n=64, frames=100, ns=512, interleaves=0,
                           t1_range=(300.0, 2500.0), t2_range=(30.0, 300.0),
                           n_t1=50, n_t2=30, rank=0),
    # 256x256 phantom, T=1000, 1 of 48 spiral interleaves per frame (2048
    # samples), 2x grid, KB width 4, ~6000 atoms compressed to K=10; 10
    # iterations with 8x8 patches (stride 4) and a k=10 nearest-patch graph.
    "mrf256_t1000": Workload("mrf256_t1000", n=256, frames=1000, ns=2048, interleaves=48,
                             t1_range=(100.0, 4000.0), t2_range=(10.0, 500.0),
                             n_t1=100, n_t2=60, rank=10),
    # The same image, patch grid, dictionary and interleaf pattern with 100
    # frames: the per-image kernels (matching, kNN, SVT, graph term) have the
    # shapes of the 1000-frame workload at a tenth of the device memory, for
    # small profiling captures.
    "mrf256_t100": Workload("mrf256_t100", n=256, frames=100, ns=2048, interleaves=48,
                            t1_range=(100.0, 4000.0), t2_range=(10.0, 500.0),
                            n_t1=100, n_t2=60, rank=10),
}


# ----------------------------------------------------------------------------
# Phantom
# ----------------------------------------------------------------------------
def phantom(n: int, seed: int = 0, regions: int = 8):
    """Piecewise-constant tissue maps on an n x n grid.

    A disk of radius 0.45 n (the background tissue) holds ``regions - 1``
    seeded ellipses; outside the disk is air (PD = T1 = T2 = 0).  Each region
    draws T1 log-uniform in [300, 2500] ms, T2 log-uniform in [30, 300] ms and
    PD uniform in [0.5, 1.0].

    Returns (t1, t2, pd, mask, label) as float64 / bool / int arrays [n, n]
    indexed [y, x].
    """
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    cx = cy = (n - 1) / 2.0
    mask = (x - cx) ** 2 + (y - cy) ** 2 <= (0.45 * n) ** 2
    label = np.where(mask, 0, -1)
    for r in range(1, regions):
        rad = 0.30 * n * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * math.pi)
        ex, ey = cx + rad * math.cos(ang), cy + rad * math.sin(ang)
        a = rng.uniform(0.06, 0.16) * n
        b = rng.uniform(0.06, 0.16) * n
        th = rng.uniform(0, math.pi)
        c, s = math.cos(th), math.sin(th)
        u = (x - ex) * c + (y - ey) * s
        v = -(x - ex) * s + (y - ey) * c
        inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
        label = np.where(inside & mask, r, label)
    t1v = np.exp(rng.uniform(math.log(300.0), math.log(2500.0), regions))
    t2v = np.exp(rng.uniform(math.log(30.0), math.log(300.0), regions))
    pdv = rng.uniform(0.5, 1.0, regions)
    t1 = np.where(mask, t1v[np.clip(label, 0, None)], 0.0)
    t2 = np.where(mask, t2v[np.clip(label, 0, None)], 0.0)
    pd = np.where(mask, pdv[np.clip(label, 0, None)], 0.0)
    return t1, t2, pd, mask, label


# ----------------------------------------------------------------------------
# Sequence
# ----------------------------------------------------------------------------
def fisp_train(frames: int, seed: int = 2):
    """Flip angles (degrees) and repetition times (ms) of a FISP train.

    FA_t = 5 + 55 |sin(pi t / 200)| (sinusoidal lobes between 5 and 60 deg),
    TR_t uniform in [12, 15] ms (seeded).  The paper shows its own train only in
    a figure (Fig. 3a,b), which is not available.
    """
    t = np.arange(frames, dtype=np.float64)
    fa = 5.0 + 55.0 * np.abs(np.sin(np.pi * t / 200.0))
    tr = np.random.default_rng(seed).uniform(12.0, 15.0, frames)
    return fa, tr


# ----------------------------------------------------------------------------
# Trajectory
# ----------------------------------------------------------------------------
def spiral_interleaf(n: int, ns: int, n_interleaves: int = 48):
    """One variable-density spiral arm, k(tau) = pi tau^2 exp(i 2 pi n_turns tau).

    k is in radians per voxel; |k| reaches pi at the end of the arm.  The
    quadratic radius makes the sampling density highest at the centre.
    Returns complex128 [ns].
    """
    tau = np.arange(ns, dtype=np.float64) / max(ns - 1, 1)
    n_turns = math.ceil(2 * n / (2 * n_interleaves))
    return np.pi * tau ** 2 * np.exp(1j * 2 * np.pi * n_turns * tau)


def spiral_trajectory(n: int, frames: int, ns: int, interleaves: int, per_frame: int = 1):
    """k-space sample positions [frames, per_frame * ns, 2] as (kx, ky) in radians/voxel.

    interleaves == 0: frame t is the base arm rotated by t golden angles.
    interleaves == P: frame t uses arms (t per_frame + j) mod P, j < per_frame,
    arm a rotated by 2 pi a / P, concatenated.
    Coordinates are wrapped into [-pi, pi).
    """
    arm = spiral_interleaf(n, ns, 48 if interleaves == 0 else interleaves)
    t = np.arange(frames)
    if interleaves == 0:
        if per_frame != 1:
            raise ValueError("golden-angle frames carry one arm each")
        rot = t * GOLDEN_ANGLE
        k = arm[None, :] * np.exp(1j * rot)[:, None]
    else:
        arms = (t[:, None] * per_frame + np.arange(per_frame)[None, :]) % interleaves     # [frames, per_frame]
        rot = 2 * np.pi * arms / interleaves
        k = (arm[None, None, :] * np.exp(1j * rot)[:, :, None]).reshape(frames, per_frame * ns)
    out = np.stack([k.real, k.imag], axis=-1)
    out = np.mod(out + np.pi, 2 * np.pi) - np.pi
    return out


def interleaf_of_frame(frames: int, interleaves: int):
    """Arm index of each frame (frames sharing an arm share sample positions)."""
    if interleaves == 0:
        return np.arange(frames)
    return np.arange(frames) % interleaves


# ----------------------------------------------------------------------------
# Noise
# ----------------------------------------------------------------------------
def complex_normal(shape, seed: int):
    """Circular complex Gaussian draws with E|z|^2 = 1 (real, imag each var 1/2)."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal(shape)
    im = rng.standard_normal(shape)
    return (re + 1j * im) / math.sqrt(2.0)


def real_normal(shape, seed: int):
    return np.random.default_rng(seed).standard_normal(shape)


# ----------------------------------------------------------------------------
# Dictionary grids
# ----------------------------------------------------------------------------
def log_grid(lo: float, hi: float, n: int):
    return np.exp(np.linspace(math.log(lo), math.log(hi), n))


def keep_t1_ge_t2(t1s, t2s):
    """All (T1, T2) pairs of two axes with T1 >= T2 (pairs with T1 < T2 are omitted)."""
    T1, T2 = np.meshgrid(t1s, t2s, indexing="ij")
    keep = T1 >= T2
    return np.stack([T1[keep], T2[keep]], axis=-1)


def workload_grid(w: Workload):
    """(T1, T2) lookup table [M, 2] of the workload's dictionary."""
    return keep_t1_ge_t2(log_grid(*w.t1_range, w.n_t1), log_grid(*w.t2_range, w.n_t2))


def paper_grid():
    """The (T1, T2) axes of the paper's dictionary discretisation (Sec. IV).

    T1: 100..2000 step 20, then 2300..5000 step 300.  T2: 20..100 step 5,
    110..200 step 10, 300..1900 step 200.
    """
    t1 = np.concatenate([np.arange(100, 2001, 20), np.arange(2300, 5001, 300)]).astype(np.float64)
    t2 = np.concatenate([np.arange(20, 101, 5), np.arange(110, 201, 10),
                         np.arange(300, 1901, 200)]).astype(np.float64)
    return t1, t2


# ----------------------------------------------------------------------------
# Draws of the learned matcher's training set (random numbers only; the
# arithmetic that turns them into fingerprints runs in the library)
# ----------------------------------------------------------------------------
def mlp_training_draws(n: int, K: int, seed: int, t1_range=(100.0, 4000.0), t2_range=(10.0, 500.0),
                       pd_range=(0.2, 1.2), snr_db_range=(20.0, 40.0)):
    """(t1t2 [n, 2], rho [n], snr_db [n], noise [n, K] complex): T1 and T2
    log-uniform over their ranges with T1 >= T2 (rejection), PD and SNR
    uniform, complex Gaussian noise of unit variance per coefficient."""
    rng = np.random.default_rng(seed)
    out = np.empty((0, 2))
    while len(out) < n:
        m = 2 * (n - len(out)) + 16
        t1 = np.exp(rng.uniform(np.log(t1_range[0]), np.log(t1_range[1]), m))
        t2 = np.exp(rng.uniform(np.log(t2_range[0]), np.log(t2_range[1]), m))
        keep = t1 >= t2
        out = np.concatenate([out, np.stack([t1[keep], t2[keep]], -1)])[:n]
    rho = rng.uniform(pd_range[0], pd_range[1], n)
    snr = rng.uniform(snr_db_range[0], snr_db_range[1], n)
    noise = (rng.standard_normal((n, K)) + 1j * rng.standard_normal((n, K))) / np.sqrt(2.0)
    return out, rho, snr, noise


def mlp_init_params(seed: int, sizes=(20, 256, 256, 256, 3)):
    """Initial packed parameters of the learned matcher (per layer W [out][in],
    then b [out]): W uniform in +-sqrt(6 / in), b = 0."""
    rng = np.random.default_rng(seed)
    out = []
    for i, o in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / i)
        out += [rng.uniform(-lim, lim, o * i), np.zeros(o)]
    return np.concatenate(out)
