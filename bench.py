#!/usr/bin/env python
"""Benchmark: MS-LLR reconstruction iterations per second at 256^2 x 1000 frames.

One step = one iteration of Algorithm 1 on the GPU (data-term adjoint and
forward NUFFT over the 1000 frames, graph term, SVT, X update, cost,
matching and the k-nearest-patch Laplacian), through the C ABI, with every
input resident in device memory.  Two variants are timed:
  plain  - per-frame NUFFT (1000 forward + 1000 adjoint transforms per
           iteration) and FP32 exhaustive matching;
  chosen - the same operator evaluated in grouped form (K oversampled FFTs
           and interleaf-grouped interpolation) and tensor-core matching
           (split BF16 products, FP32 accumulation, FP32 top-8 re-rank).
`value` is the chosen variant's whole-job iterations/s.  Under torchrun each
rank reconstructs its own slice (weak scaling, no data-path collective).

Inputs are synthetic and seeded (synth/): a 256^2 phantom of 8 regions, a
FISP train of 1000 repetitions, 1 of 48 variable-density spiral interleaves of
2048 samples per frame, complex Gaussian noise at 30 dB, and a dictionary of
100 x 60 log-spaced (T1, T2) pairs simulated by the library's EPG kernel.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MRF recon iters/s at 256^2x1000 frames, chosen vs plain; T1/T2 NRMSE vs oracle"
WORKLOAD = "mrf256_t1000"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variants", default="plain,chosen,learned")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched-serving measurement")
    ap.add_argument("--workload", default=WORKLOAD, choices=["mrf256_t1000", "mrf256_t100"],
                    help="mrf256_t100: the same image with 100 frames, for small profiling captures")
    ap.add_argument("--oracle-leg", default=None, help=argparse.SUPPRESS)   # child process of the cpu_baseline leg
    ap.add_argument("--only-full-length-matching", type=int, default=0, metavar="N",
                    help="run only the full-length matching measurement with N fingerprints (profiling captures)")
    ap.add_argument("--no-oracle-parity", action="store_true",
                    help="skip the oracle comparison on the reduced copy of the problem and the 64^2 x 100 line")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (barrier and max over ranks only)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        import torch
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.file:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------
def make_inputs(seed):
    """Device inputs of the 256^2 x 1000-frame workload, built with the library's kernels."""
    import numpy as np
    import torch

    import synth
    import paper_2310_05647_gb300 as mrf

    w = synth.WORKLOADS[WORKLOAD]
    dev = torch.device("cuda")
    t1, t2, pd, mask, label = synth.phantom(w.n, seed=seed)
    fa, tr = synth.fisp_train(w.frames, seed=w.tr_seed)
    lut = synth.workload_grid(w)
    traj = synth.spiral_trajectory(w.n, w.frames, w.ns, w.interleaves)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    fa_d, tr_d = f32(fa), f32(tr)
    lut_d = f32(lut)
    D = mrf.epg_fisp(lut_d, fa_d, tr_d)                              # [M, T]
    phi, comp, n2 = mrf.dict_subspace(D, w.rank)
    # ground-truth series: one EPG signal per region, times PD (input synthesis)
    regions = np.unique(label[label >= 0])
    pairs = np.stack([[t1[label == r][0], t2[label == r][0]] for r in regions])
    S = mrf.epg_fisp(f32(pairs), fa_d, tr_d)                          # [R, T]
    lab = torch.tensor(np.where(label >= 0, np.searchsorted(regions, np.maximum(label, 0)), 0).ravel(),
                       device=dev, dtype=torch.long)
    pdm = f32(pd.ravel()).to(torch.complex64)
    X = (S[lab] * pdm[:, None]).T.contiguous().view(w.frames, w.n, w.n)   # [T, ny, nx]
    plan = mrf.nufft_plan(w.n, w.n, f32(traj), os=w.os, kb_width=w.kb_width)
    b = mrf.nufft_forward(plan, X)
    del X
    sig = math.sqrt(float((b.abs() ** 2).mean()) * 10 ** (-w.snr_db / 10))
    g = torch.Generator(device=dev)
    g.manual_seed(1000 + w.noise_seed + seed)
    noise = torch.complex(torch.randn(b.shape, generator=g, device=dev),
                          torch.randn(b.shape, generator=g, device=dev)) * (sig / math.sqrt(2.0))
    b = (b + noise).contiguous()
    torch.cuda.synchronize()
    return dict(w=w, plan=plan, phi=phi, comp=comp, n2=n2, lut=lut_d, b=b, truth=(t1, t2, pd, mask),
                atoms=int(lut.shape[0]))


def params_for(variant, w, mlp=None):
    """plain: frame-by-frame operator, FP32 exhaustive matching; chosen: grouped
    operator, split-BF16 tensor-core matching; learned: chosen with the learned
    matcher (exhaustive split-BF16 fallback)."""
    import paper_2310_05647_gb300 as mrf
    from paper_2310_05647_gb300.api import RECON_GROUPED, RECON_LEARNED
    from paper_2310_05647_gb300.api import MATCH_BF16X3, MATCH_FP32
    flags = {"plain": 0, "chosen": RECON_GROUPED, "learned": RECON_GROUPED | RECON_LEARNED}[variant]
    prec = MATCH_FP32 if variant == "plain" else MATCH_BF16X3
    return mrf.ReconParams(patch=w.patch, stride=w.stride, knn=w.knn, flags=flags, match_precision=prec,
                           mlp=mlp if variant == "learned" else None)


def train_learned(inp, n_train=2_000_000, epochs=3, seed=0):
    """The learned matcher for this workload: 2M noisy EPG fingerprints of the
    workload's sequence (T1, T2 over the dictionary's ranges, SNR 20-40 dB),
    simulated and trained on the GPU."""
    import numpy as np
    import torch

    import synth
    import paper_2310_05647_gb300 as mrf

    w = inp["w"]
    fa, tr = synth.fisp_train(w.frames, seed=w.tr_seed)
    n2 = inp["n2"].cpu().numpy()
    ranges = (w.t1_range[0], w.t1_range[1], w.t2_range[0], w.t2_range[1], float(1.0 / np.median(np.sqrt(n2))))
    draws = synth.mlp_training_draws(n_train, w.rank, seed=3000 + seed, t1_range=w.t1_range, t2_range=w.t2_range)
    dev = torch.device("cuda")
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net, hist = mrf.train_matcher(synth.mlp_init_params(4000 + seed), draws, f32(fa), f32(tr), inp["phi"], ranges,
                                  epochs=epochs, batch=1024)
    torch.cuda.synchronize()
    return net, {"fingerprints": n_train, "epochs": epochs, "batch": 1024, "seconds": time.perf_counter() - t0,
                 "loss_per_epoch": hist}


def nrmse(truth, maps):
    import numpy as np
    t1, t2, pd, mask = truth
    out = {}
    for name, ref, est in (("t1", t1, maps[0]), ("t2", t2, maps[1]), ("pd", pd, maps[2])):
        e = est[mask]
        r = ref[mask]
        out[name] = float(np.sqrt(np.sum((e - r) ** 2) / np.sum(r ** 2)))
    return out


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu --set full capture of the kernel as it stands, on the same launch
# shape (the matcher's shape, 65536 fingerprints x 5441 atoms x K = 10, does
# not depend on the frame count; captured on the 100-frame workload).  An
# entry must be dropped whenever its kernel changes.
MEASURED_TRAFFIC = {
    "k_match_tc": (8819200, "ncu --set full, mrf256_t100 workload, launch shape of the full workload "
                            "(profiles/k_match_tc_mrf256_t100.md)"),
    "k_graph_blocks": (5970176, "ncu --set full of the Q(X)L launch, mrf256_t100 workload, launch shape of the "
                                "full workload (profiles/graph_kernels_mrf256_t100.md)"),
}


# algorithmic bytes (HBM-bound kernels) or flops (ALU-bound) per launch
def algorithmic_work(kernel, inp):
    w = inp["w"]
    T, n, ns, K, G = w.frames, w.n, w.ns, w.rank, w.os * w.n
    M = inp["atoms"]
    frame_h1 = n * G * 8                          # one frame's half-oversampled intermediate
    cnt = (n - w.patch) // w.stride + 1 + (1 if (n - w.patch) % w.stride else 0)
    npatch = cnt * cnt
    ngroups = w.interleaves or T
    table = {
        # per-frame subspace expansion: coefficients (L2-resident, read once) + H1 write
        "k_rows_fwd_expand": ("hbm", T * frame_h1 + n * n * K * 8),
        # column FFT + interpolation: H1 read + samples (trajectory record + value) written
        "k_cols_interp": ("hbm", T * (frame_h1 + ns * 8 + ns * 8 + ns * 8)),
        # spread + column IFFT: samples read + H1 written
        "k_spread_cols": ("hbm", T * (ns * 8 + ns * 8 + frame_h1)),
        "k_spread_gather": ("hbm", T * (ns * 8 + ns * 8 + frame_h1)),     # the sorted-gather form, same bytes
        # row IFFT + subspace reduction: H1 read + partial coefficient images
        "k_rows_adj_reduce": ("hbm", T * frame_h1),
        "k_rows_fwd": ("hbm", T * (n * n * 8 + frame_h1)),
        "k_rows_adj": ("hbm", T * (frame_h1 + n * n * 8)),
        # exhaustive matching: complex MAC = 8 flops
        "k_match_fp32": ("alu", 8.0 * n * n * M * K),
        # tensor-core matching: the complex inner products as a real GEMM,
        # 2 x N x (2 M) x (2 K) (the split-BF16 form issues 3x this)
        "k_match_tc": ("tensor", 2.0 * n * n * (2 * M) * (2 * K)),
        # exact patch kNN: FP16 GEMM of the np query vectors against 2 np candidate
        # rows (h, l) over the 2 p^2 = 128 entries
        "k_knn_tc": ("tensor", 2.0 * npatch * (2 * npatch) * (2 * w.patch ** 2)),
        # SVT (Gram matrix + two-sided Jacobi): executed FP32 flops from the
        # kernel's own sweep and rotation counts (svt_flops)
        "k_svt": svt_flops(npatch, w.patch ** 2, K, inp.get("svt_work")),
        # graph term: the coefficient image read once, Q(X) L written per patch
        "k_graph_blocks": ("hbm", n * n * K * 8 + npatch * w.patch ** 2 * K * 8),
    }
    return table.get(kernel)


def svt_flops(npatch, pp, K, work):
    """Executed FP32 flops of one k_svt launch (an FMA counts 2, a complex
    multiply-add 8): per patch the Gram matrix (8 pp NG), the warm-start
    transform and the new V (3 x 8 KP^3), the column norms of A V (8 pp KP^2),
    M = V diag(f) V^H (8 KP^2 K) and P = A M (8 pp KP K); per Jacobi sweep
    (KP - 1) rounds of NOFF off-diagonal 2 x 2 blocks (4 two-term complex
    rotations, 56 flops) and KP NPAIR column pairs of W (14 flops); per
    rotation 30 flops.  Sweeps and rotations come from the kernel's counters."""
    if not work:
        return None
    KP = K if K in (4, 8, 10, 12, 16) else (4 if K <= 4 else 8 if K <= 8 else 12 if K <= 12 else 16)
    npair = KP // 2
    ng, noff = KP * (KP + 1) // 2, npair * (npair - 1) // 2
    per_sweep = (KP - 1) * (56 * noff + 14 * KP * npair)
    fixed = 8 * pp * ng + 24 * KP ** 3 + 8 * pp * KP * KP + 8 * KP * KP * K + 8 * pp * KP * K
    return ("alu", npatch * (work["sweeps_per_patch"] * per_sweep + work["rotations_per_patch"] * 30 + fixed))


def time_variant(variant, inp, steps, warmup, dist):
    import numpy as np
    import torch

    import paper_2310_05647_gb300 as mrf

    w = inp["w"]
    rec = mrf.Recon(inp["plan"], params_for(variant, w, inp.get("mlp")), inp["phi"], inp["comp"], inp["n2"],
                    inp["lut"], inp["b"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")    # 256 MiB > L2
    for _ in range(warmup):
        flush.zero_()
        rec.iterate(1)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    launches0 = mrf.launch_count()
    dist.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        for i in range(steps):
            flush.zero_()
            starts[i].record()
            rec.iterate(1)
            ends[i].record()
        torch.cuda.synchronize()
    dist.barrier()
    launches = mrf.launch_count() - launches0
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    # per-kernel intervals of the same concurrent loop, from an untimed pass
    # with the profiler on (it records an event per launch, so the loop then
    # launches its kernels one by one instead of replaying the recorded one)
    mrf.profile_enable(True)
    for i in range(steps):
        flush.zero_()
        mrf.profile_mark()
        rec.iterate(1)
    torch.cuda.synchronize()
    prof = mrf.profile_read()
    mrf.profile_enable(False)
    # results after warm-up + the timed steps (read before the clock window below)
    t1, t2, pd, idx = rec.maps()
    maps = [t.cpu().numpy() for t in (t1, t2, pd)]
    fallback = float((idx >= 0).float().mean())
    info = rec.info()
    alpha = rec.alpha().clone()
    # The timed region is far shorter than the sampler's 200 ms period: keep the
    # same iteration running for a sustained window and sample clocks there too.
    # (Untimed: it only checks the clocks the timed steps ran under.)
    with Clocks(torch.cuda.current_device()) as clk2:
        t0 = time.time()
        while time.time() - t0 < 1.5:
            for _ in range(20):
                flush.zero_()
                rec.iterate(1)
            torch.cuda.synchronize()
    clocks = merge_clocks(clk.summary(), clk2.summary(), 1e3 * (time.time() - t0))
    del rec
    return dict(ms=ms, launches=launches, profile=prof, clocks=clocks,
                nrmse=nrmse(inp["truth"], maps), info=info, maps=maps, alpha=alpha, fallback=fallback)


def profile_serial(variant, inp, iters=10, warmup=3):
    """Per-kernel CUDA-event durations of the variant with its steps serialised
    (MRF_RECON_SERIAL: same kernels, inputs and results; in the default
    concurrent loop the kernels share the SMs, so their intervals overlap)."""
    import torch

    import paper_2310_05647_gb300 as mrf
    from paper_2310_05647_gb300.api import RECON_SERIAL

    w = inp["w"]
    p = params_for(variant, w, inp.get("mlp"))
    p.flags |= RECON_SERIAL
    rec = mrf.Recon(inp["plan"], p, inp["phi"], inp["comp"], inp["n2"], inp["lut"], inp["b"])
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        flush.zero_()
        rec.iterate(1)
    torch.cuda.synchronize()
    mrf.profile_enable(True)
    sv0 = rec.svt_stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = 0.0
    for _ in range(iters):
        flush.zero_()
        mrf.profile_mark()
        e0.record()
        rec.iterate(1)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    prof = mrf.profile_read()
    mrf.profile_enable(False)
    sv1 = rec.svt_stats()
    # executed Jacobi work per patch and SVT launch over the profiled iterations
    dp = sv1[2] - sv0[2]
    work = {"sweeps_per_patch": (sv1[0] - sv0[0]) / dp, "rotations_per_patch": (sv1[1] - sv0[1]) / dp}
    del rec
    return prof, ms / iters, iters, work


def merge_clocks(timed, sustained, sustained_ms):
    """Clock record of the timed steps plus the sustained window that follows them."""
    out = dict(sustained)
    out["samples_timed_region"] = timed.get("samples", 0)
    out["sm_mhz_timed_region"] = timed.get("sm_mhz")
    out["reasons"] = sorted(set(timed.get("reasons", [])) | set(sustained.get("reasons", [])))
    out["window"] = (f"median over a {sustained_ms:.0f} ms window of the same iteration loop run right after "
                     f"the timed steps (the timed region itself is shorter than the 200 ms sampling period)")
    return out


def precision_variants(inp, alpha, reps=5):
    """Match the final iterate with every matching precision: per-call device time,
    index agreement and T1/T2/PD NRMSE against the FP32 exhaustive result."""
    import numpy as np
    import torch

    import paper_2310_05647_gb300 as mrf
    from paper_2310_05647_gb300.api import MATCH_BF16, MATCH_BF16X3, MATCH_FP8, MATCH_FP32

    w = inp["w"]
    x = alpha.reshape(w.n * w.n, w.rank).contiguous()
    out, ref = {}, None
    for name, prec in (("fp32", MATCH_FP32), ("bf16x3", MATCH_BF16X3), ("bf16", MATCH_BF16), ("fp8", MATCH_FP8)):
        res = mrf.match(x, inp["comp"], inp["lut"], atom_norm2=inp["n2"], precision=prec)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(reps):
            res = mrf.match(x, inp["comp"], inp["lut"], atom_norm2=inp["n2"], precision=prec)
        ev[1].record()
        torch.cuda.synchronize()
        idx, pd, t1t2 = (t.cpu().numpy() for t in res)
        maps = (t1t2[:, 0], t1t2[:, 1], pd)
        if ref is None:
            ref = (idx, maps)
        err = {nm: float(np.linalg.norm(maps[i] - ref[1][i]) / max(np.linalg.norm(ref[1][i]), 1e-30))
               for i, nm in enumerate(("t1", "t2", "pd"))}
        out[name] = {"ms_per_match": ev[0].elapsed_time(ev[1]) / reps,
                     "index_agreement_vs_fp32": float((idx == ref[0]).mean()), "nrmse_vs_fp32": err}
    return out


def full_length_matching(peaks, reps=3, n=65536):
    """Matching of full 1000-frame fingerprints (Eq. 5 without the subspace):
    65536 noisy fingerprints built from the 256^2 workload's 5441 EPG atoms,
    split-BF16 streamed tensor-core matcher against the FP32 SIMT matcher.
    Algorithmic work: the complex GEMM, 8 N M T flops (the split form issues
    3x that on the tensor cores)."""
    import torch

    import synth
    import paper_2310_05647_gb300 as mrf
    from paper_2310_05647_gb300.api import MATCH_BF16, MATCH_BF16X3, MATCH_FP32

    w = synth.WORKLOADS[WORKLOAD]
    dev = torch.device("cuda")
    fa, tr = synth.fisp_train(1000, seed=w.tr_seed)
    f32 = lambda a: torch.tensor(a, dtype=torch.float32, device=dev)
    lut = f32(synth.workload_grid(w))
    D = mrf.epg_fisp(lut, f32(fa), f32(tr))
    n2 = (D.abs() ** 2).sum(1).float().contiguous()
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    M, T = D.shape[0], D.shape[1]
    pick = torch.randint(0, M, (n,), generator=g, device=dev)
    noise = torch.complex(torch.randn(n, T, generator=g, device=dev), torch.randn(n, T, generator=g, device=dev))
    X = (D[pick] * 0.8 + 0.02 * D.abs().mean() * noise).contiguous()
    del noise
    flops = 8.0 * n * M * T
    peak = peaks.get("bf16_tflops_sustained", 1716.1)
    out = {"what": f"{n} fingerprints x {M} atoms x {T} frames (full-length Eq. 5), one mrf_match call",
           "algorithmic_flops": flops}
    res = {}
    for name, prec, r in (("bf16x3", MATCH_BF16X3, reps), ("bf16", MATCH_BF16, reps), ("fp32", MATCH_FP32, 1)):
        res[name] = mrf.match(X, D, lut, atom_norm2=n2, precision=prec)
        torch.cuda.synchronize()
        mrf.profile_enable(True)
        mrf.profile_mark()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(r):
            res[name] = mrf.match(X, D, lut, atom_norm2=n2, precision=prec)
        e1.record()
        torch.cuda.synchronize()
        prof = mrf.profile_read()
        mrf.profile_enable(False)
        ms = e0.elapsed_time(e1) / r
        ent = {"ms_per_call": ms, "tflops_algorithmic": flops / ms / 1e9,
               "kernels_ms": {k: round(v[0] / max(v[1], 1), 4) for k, v in prof.items()}}
        if name != "fp32" and "k_match_tc_long" in prof:
            kms = prof["k_match_tc_long"][0] / max(prof["k_match_tc_long"][1], 1)
            ent["roofline"] = {"kernel": "k_match_tc_long", "bound": "tensor", "achieved": flops / kms / 1e9,
                               "peak": peak, "unit": "TFLOP/s", "frac": flops / kms / 1e9 / peak,
                               "issued_frac": (3 if name == "bf16x3" else 1) * flops / kms / 1e9 / peak,
                               "peak_source": "of measured (bf16 sustained)", "ms_per_launch": kms}
        out[name] = ent
    for name in ("bf16x3", "bf16"):
        out[f"index_agreement_{name}_vs_fp32"] = float((res[name][0] == res["fp32"][0]).float().mean())
    del X, D
    return out


def serving(seed=0, slices=16, iters=10, rounds=10):
    """Batched serving: `slices` slices of uneven size (grid 128^2 or 256^2, T in
    {500, 750, 1000}, 1-3 spiral arms per frame, seeded draws) sharing one atom
    grid, each compressed in its own frame count's subspace.  Throughput and
    request latency of the batched loop (one CUDA graph launch per iteration
    of all slices) against the same slices iterated one after another."""
    import numpy as np
    import torch

    import synth
    import paper_2310_05647_gb300 as mrf
    from paper_2310_05647_gb300.api import MATCH_BF16X3, RECON_GROUPED, RECON_NO_COST

    w = synth.WORKLOADS[WORKLOAD]
    rng = np.random.default_rng(1000 + seed)
    dev = torch.device("cuda")
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    fa, tr = synth.fisp_train(1000, seed=w.tr_seed)
    lut = synth.workload_grid(w)
    lut_d = f32(lut)
    D = mrf.epg_fisp(lut_d, f32(fa), f32(tr))
    comp = {}
    for T in (500, 750, 1000):
        comp[T] = mrf.dict_subspace(D[:, :T].contiguous(), w.rank)
    del D
    cfg, recons, keep = [], [], []
    for i in range(slices):
        n = int(rng.choice([128, 192, 256]))
        T = int(rng.choice([500, 750, 1000]))
        per = int(rng.integers(1, 4))
        cfg.append({"n": n, "frames": T, "arms_per_frame": per})
        t1, t2, pd, mask, label = synth.phantom(n, seed=100 + i)
        pairs = np.stack([np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0)], -1)
        S = mrf.epg_fisp(f32(pairs), f32(fa[:T]), f32(tr[:T]))
        X = (S * f32((pd * mask).ravel()).to(torch.complex64)[:, None]).T.contiguous().view(T, n, n)
        del S
        plan = mrf.nufft_plan(n, n, f32(synth.spiral_trajectory(n, T, w.ns, w.interleaves, per_frame=per)))
        b = mrf.nufft_forward(plan, X)
        del X
        sig = math.sqrt(float((b.abs() ** 2).mean()) * 10 ** (-w.snr_db / 10))
        g = torch.Generator(device=dev)
        g.manual_seed(2000 + i)
        b = (b + torch.complex(torch.randn(b.shape, generator=g, device=dev),
                               torch.randn(b.shape, generator=g, device=dev)) * (sig / math.sqrt(2.0))).contiguous()
        phi, cmp_, n2 = comp[T]
        p = mrf.ReconParams(patch=w.patch, stride=w.stride, knn=w.knn, flags=RECON_GROUPED | RECON_NO_COST,
                            match_precision=MATCH_BF16X3)
        recons.append(mrf.Recon(plan, p, phi, cmp_, n2, lut_d, b))
        keep.append((plan, b))
    torch.cuda.synchronize()
    # unbatched: every slice's iterations issued one slice after another
    for r in recons:
        r.iterate(1)
    torch.cuda.synchronize()
    solo = []                             # each slice served alone: its own request latency
    for r in recons:
        t0 = time.perf_counter()
        r.iterate(iters)
        torch.cuda.synchronize()
        solo.append(time.perf_counter() - t0)
    seq_s = sum(solo)
    batch = mrf.Batch(recons)
    l0 = mrf.launch_count()
    batch.iterate(2)                      # one eager iteration + the captured one
    per_iter_kernels = (mrf.launch_count() - l0) // 2
    lat = []
    for _ in range(rounds):
        t0 = time.perf_counter()
        batch.iterate(iters)              # synchronises
        lat.append(time.perf_counter() - t0)
    tuning = [r.plan.tuning() for r in recons]
    maps_ok = all(bool(torch.isfinite(r.maps()[0]).all()) for r in recons)
    del batch
    tot = sum(lat)
    return {"what": f"{slices} slices, {iters} iterations per request; grids from {{128^2, 192^2, 256^2}}, "
                    f"T from {{500, 750, 1000}}, 1-3 arms of {w.ns} samples per "
                    f"frame, shared {len(lut)}-atom grid, split-BF16 matching, no cost terms",
            "slices": cfg,
            "throughput_slice_iters_per_s": slices * iters * rounds / tot,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99)),
                           "rounds": rounds},
            # every stage of a batched iteration is one launch over all slices, so
            # a slice's maps are ready when its request's batch completes: its
            # latency is the batch's (p50/p99 over slices x rounds)
            "per_slice_latency_ms": {"p50": 1e3 * float(np.percentile(np.repeat(lat, slices), 50)),
                                     "p99": 1e3 * float(np.percentile(np.repeat(lat, slices), 99)),
                                     "samples": slices * rounds},
            "per_slice_latency_ms_served_alone": {"p50": 1e3 * float(np.percentile(solo, 50)),
                                                  "p99": 1e3 * float(np.percentile(solo, 99)),
                                                  "samples": slices},
            "unbatched_slice_iters_per_s": slices * iters / seq_s,
            "kernels_per_batched_iteration": per_iter_kernels,
            "autotuned": [dict(n=c["n"], **t) for c, t in zip(cfg, tuning)], "maps_finite": maps_ok}


def e2e_chosen(inp, iters, reps=2):
    """End to end through the C ABI's host-buffer call (mrf_recon_run_host):
    pinned host k-space in, initialisation (A^H b, matching, graph) and
    `iters` iterations, T1/T2/PD maps back in host memory; the copies run
    inside the call."""
    import paper_2310_05647_gb300 as mrf

    w = inp["w"]
    b_host = inp["b"].cpu().pin_memory()
    p = params_for("chosen", w)
    times = []
    for r in range(reps + 1):
        t0 = time.perf_counter()
        maps = mrf.recon_run_host(inp["plan"], p, inp["phi"], inp["comp"], inp["n2"], inp["lut"], b_host, iters)
        dt = time.perf_counter() - t0          # the call synchronises its stream
        if r > 0:
            times.append(dt)
    h2d = b_host.numel() * 8
    d2h = sum(m.numel() * 4 for m in maps)
    return statistics.mean(times), h2d, d2h


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample of one iteration, extrapolated)
# ---------------------------------------------------------------------------
ORACLE_SAMPLE_SCALE = 0.25     # one sample size for the reference arm and the cpu_baseline leg


def oracle_iteration_seconds(scale=ORACLE_SAMPLE_SCALE):
    """Seconds the FP64 oracle needs for one Algorithm 1 iteration at 256^2 x 1000,
    extrapolated from timed samples of each step (frames, voxels, patches and
    graph rows), with `scale` shrinking every sample."""
    import numpy as np

    import synth
    from oracle import graph, llr, match as omatch, nufft as onufft, patches

    w = synth.WORKLOADS[WORKLOAD]
    n, T, ns = w.n, w.frames, w.ns
    rng = np.random.default_rng(0)
    parts = {}
    # data term: forward + adjoint NUFFT on F frames
    F = max(1, int(4 * scale))
    k = synth.spiral_trajectory(n, F, ns, w.interleaves)
    grid = onufft.KBGrid(n, n, w.os, w.kb_width)
    x = rng.standard_normal((F, n, n)) + 1j * rng.standard_normal((F, n, n))
    t0 = time.perf_counter()
    y = onufft.kb_forward(x, k, grid)
    onufft.kb_adjoint(y, k, grid)
    parts["nufft_pair"] = (time.perf_counter() - t0) * T / F * 2      # residual forward + adjoint per pass
    # matching at full length against the workload's dictionary size
    M = len(synth.workload_grid(w))
    nv = max(16, int(256 * scale))
    X = rng.standard_normal((nv, T)) + 1j * rng.standard_normal((nv, T))
    D = rng.standard_normal((M, T)) + 1j * rng.standard_normal((M, T))
    lut = np.ones((M, 2))
    t0 = time.perf_counter()
    omatch.match(X, D, lut)
    parts["match"] = (time.perf_counter() - t0) * (n * n) / nv
    # SVT of p^2 x T patches (twice: P step and the cost's nuclear norms)
    pg = patches.PatchGrid(n, n, w.patch, w.stride)
    npt = max(4, int(32 * scale))
    Pt = rng.standard_normal((npt, w.patch ** 2, T)) + 1j * rng.standard_normal((npt, w.patch ** 2, T))
    t0 = time.perf_counter()
    llr.svt_patches(Pt, 5.0)
    parts["svt"] = (time.perf_counter() - t0) * pg.count / npt * 2
    # graph: kNN over all patches on a sample of query rows
    t1m = rng.uniform(100, 4000, (n, n))
    t2m = rng.uniform(10, 500, (n, n))
    Fe = graph.features(t1m, t2m, pg, 4000.0, 500.0)
    rows = max(8, int(200 * scale))
    t0 = time.perf_counter()
    for i in range(rows):
        di = np.sum((Fe - Fe[i]) ** 2, axis=1)
        np.argsort(di, kind="stable")[:w.knn]
    parts["knn"] = (time.perf_counter() - t0) * pg.count / rows
    # graph term and trace with the dense Laplacian on Tg of the T frames
    Tg = max(1, int(2 * scale))
    img = rng.standard_normal((n, n, Tg)) + 1j * rng.standard_normal((n, n, Tg))
    L = np.zeros((pg.count, pg.count))
    t0 = time.perf_counter()
    graph.graph_term(img, L, pg)
    graph.trace_term(img, L, pg)
    parts["graph_term"] = (time.perf_counter() - t0) * T / Tg
    # projection and X update on full data
    Xf = rng.standard_normal((n * n, T // 10)) + 1j * rng.standard_normal((n * n, T // 10))
    phi = np.linalg.qr(rng.standard_normal((T // 10, w.rank)))[0]
    t0 = time.perf_counter()
    (Xf @ phi) @ phi.conj().T
    parts["projection"] = (time.perf_counter() - t0) * 10 * 2
    total = sum(parts.values())
    sample = (f"per-step samples extrapolated to one iteration: NUFFT pair on {F} of {T} frames, "
              f"matching {nv} of {n * n} voxels x {M} atoms x {T} frames, SVT of {npt} of {pg.count} "
              f"{w.patch}x{w.patch}x{T} patches, kNN rows {rows} of {pg.count}, graph term on {Tg} of {T} "
              f"frames, projection on {T // 10} frames")
    return total, parts, sample


# ---------------------------------------------------------------------------
# the FP64 oracle on problems it finishes in seconds (cpu_baseline leg)
# ---------------------------------------------------------------------------
# A reduced copy of the 256^2 x 1000 problem (same dictionary grid, sequence
# recipe, interleaf pattern, rank, patches, neighbours and iteration count;
# 64^2 voxels and 100 frames) on which the oracle's Algorithm 1 runs to the
# end, so the GPU variants' maps can be compared with the oracle's.
SMALL = dict(n=64, frames=100, ns=256, interleaves=48)


def _f32(a):
    import numpy as np
    a = np.asarray(a)
    return a.astype(np.complex64).astype(np.complex128) if np.iscomplexobj(a) else \
        a.astype(np.float32).astype(np.float64)


def _save(path, **arrs):
    import numpy as np
    np.savez(path + ".tmp.npz", **arrs)
    os.replace(path + ".tmp.npz", path)


def oracle_leg(out_dir, iters):
    """Child process: build the inputs of the reduced problem and of the 64^2 x
    100 plain workload with the oracle (saved for the GPU side), then time the
    oracle on both: A^H gridding + exhaustive matching, and Algorithm 1's
    initialisation + `iters` iterations.  Run with one BLAS thread: the
    oracle's many small SVDs are ~20x slower with a multi-threaded BLAS."""
    import numpy as np

    import synth
    from oracle import dictionary, epg, match as omatch, nufft as onufft, recon as orecon

    big = synth.WORKLOADS["mrf256_t1000"]
    n, T, ns, il = SMALL["n"], SMALL["frames"], SMALL["ns"], SMALL["interleaves"]
    t1, t2, pd, mask, _ = synth.phantom(n, seed=big.phantom_seed)
    fa, tr = synth.fisp_train(T, seed=big.tr_seed)
    lut = synth.workload_grid(big)
    D = epg.fisp(lut[:, 0], lut[:, 1], fa, tr)
    X = pd.reshape(-1, 1) * epg.fisp(np.maximum(t1.ravel(), 1.0), np.maximum(t2.ravel(), 1.0), fa, tr)
    X *= mask.reshape(-1, 1)
    k = synth.spiral_trajectory(n, T, ns, il)
    grid = onufft.KBGrid(n, n, big.os, big.kb_width)
    b = onufft.kb_forward(X.reshape(n, n, T).transpose(2, 0, 1), k, grid)
    b = b + np.sqrt(np.mean(np.abs(b) ** 2) * 10 ** (-big.snr_db / 10)) * synth.complex_normal(b.shape, seed=1)
    phi = dictionary.subspace(D, big.rank)
    k, b, phi, D, lut, fa, tr = (_f32(a) for a in (k, b, phi, D, lut, fa, tr))
    _save(os.path.join(out_dir, "loop_inputs.npz"), k=k, b=b, phi=phi, D=D, lut=lut, fa=fa, tr=tr, t1=t1, t2=t2,
          pd=pd, mask=mask)
    # 64^2 x 100 plain workload: A^H gridding then exhaustive full-length matching
    c1 = synth.WORKLOADS["mrf64_t100"]
    ct1, ct2, cpd, cmask, _ = synth.phantom(c1.n, seed=c1.phantom_seed)
    cfa, ctr = synth.fisp_train(c1.frames, seed=c1.tr_seed)
    clut = synth.workload_grid(c1)
    cD = epg.fisp(clut[:, 0], clut[:, 1], cfa, ctr)
    cX = cpd.reshape(-1, 1) * epg.fisp(np.maximum(ct1.ravel(), 1.0), np.maximum(ct2.ravel(), 1.0), cfa, ctr)
    cX *= cmask.reshape(-1, 1)
    ck = synth.spiral_trajectory(c1.n, c1.frames, c1.ns, c1.interleaves)
    cgrid = onufft.KBGrid(c1.n, c1.n, c1.os, c1.kb_width)
    cb = onufft.kb_forward(cX.reshape(c1.n, c1.n, c1.frames).transpose(2, 0, 1), ck, cgrid)
    cb = cb + np.sqrt(np.mean(np.abs(cb) ** 2) * 10 ** (-c1.snr_db / 10)) * synth.complex_normal(cb.shape, seed=1)
    ck, cb, cD, clut = (_f32(a) for a in (ck, cb, cD, clut))
    _save(os.path.join(out_dir, "c1_inputs.npz"), k=ck, b=cb, D=cD, lut=clut, t1=ct1, t2=ct2, pd=cpd, mask=cmask)
    reps, t0 = 3, time.perf_counter()
    for _ in range(reps):
        xa = onufft.kb_adjoint(cb, ck, cgrid)
        ci, c_t1, c_t2, c_pd = omatch.match(xa.reshape(c1.frames, -1).T, cD, clut)
    c1_s = (time.perf_counter() - t0) / reps
    _save(os.path.join(out_dir, "c1_oracle.npz"), idx=ci, t1=c_t1, t2=c_t2, pd=c_pd, seconds=c1_s)
    # Algorithm 1 on the reduced problem
    t0 = time.perf_counter()
    o = orecon.MSLLR(b, k, grid, phi, D, lut, orecon.Params(patch=big.patch, stride=big.stride,
                                                            knn=big.knn)).init()
    init_s = time.perf_counter() - t0
    its = []
    for _ in range(iters):
        t0 = time.perf_counter()
        o.iterate()
        its.append(time.perf_counter() - t0)
    idx, ot1, ot2, opd = o.maps
    _save(os.path.join(out_dir, "loop_oracle.npz"), idx=idx, t1=ot1, t2=ot2, pd=opd / o.gamma, a=o.a, gamma=o.gamma,
          init_s=init_s, its=np.array(its), cost=np.array(o.cost))


def start_oracle_leg(out_dir, iters):
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    log = open(os.path.join(out_dir, "oracle_leg.log"), "w")
    return subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-leg", out_dir,
                             "--steps", str(iters)], env=env, stdout=log, stderr=subprocess.STDOUT)


def _wait_file(path, proc, timeout=900.0):
    t0 = time.time()
    while not os.path.exists(path):
        if proc.poll() is not None and not os.path.exists(path):
            raise RuntimeError(f"oracle leg exited ({proc.returncode}) before writing {os.path.basename(path)}")
        if time.time() - t0 > timeout:
            raise RuntimeError(f"oracle leg: no {os.path.basename(path)} after {timeout:.0f} s")
        time.sleep(0.2)
    import numpy as np
    return dict(np.load(path))


def _nrmse(ref, est, mask):
    import numpy as np
    r, e = np.asarray(ref, np.float64)[mask], np.asarray(est, np.float64)[mask]
    den = np.sum(r ** 2)
    return float(np.sqrt(np.sum((e - r) ** 2) / den)) if den > 0 else 0.0


def small_problem_parity(out_dir, proc, variants, iters):
    """Each GPU variant on the reduced problem, from the oracle's inputs, for
    `iters` iterations; T1/T2/PD NRMSE of its maps against the oracle's."""
    import numpy as np
    import torch

    import synth
    import paper_2310_05647_gb300 as mrf

    inp = _wait_file(os.path.join(out_dir, "loop_inputs.npz"), proc)
    big = synth.WORKLOADS["mrf256_t1000"]
    dev = torch.device("cuda")
    c64 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.complex64, device=dev)
    f32 = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    n = SMALL["n"]
    plan = mrf.nufft_plan(n, n, f32(inp["k"]), os=big.os, kb_width=big.kb_width)
    phi, D = inp["phi"], inp["D"]
    n2 = np.sum(np.abs(D) ** 2, axis=1)
    args = (c64(phi), c64(D @ phi), f32(n2), f32(inp["lut"]), c64(inp["b"]))
    mlp = None
    if "learned" in variants:
        draws = synth.mlp_training_draws(1_000_000, big.rank, seed=3100, t1_range=big.t1_range,
                                         t2_range=big.t2_range)
        ranges = (big.t1_range[0], big.t1_range[1], big.t2_range[0], big.t2_range[1],
                  float(1.0 / np.median(np.sqrt(n2))))
        mlp, _ = mrf.train_matcher(synth.mlp_init_params(4100), draws, f32(inp["fa"]), f32(inp["tr"]), args[0],
                                   ranges, epochs=3, batch=1024)
    gpu = {}
    for v in variants:
        rec = mrf.Recon(plan, params_for(v, big, mlp), *args)
        rec.iterate(iters)
        gpu[v] = [t.cpu().numpy() for t in rec.maps()]
        del rec
    orc = _wait_file(os.path.join(out_dir, "loop_oracle.npz"), proc)
    mask = inp["mask"].astype(bool)
    out = {"what": f"reduced copy of the problem ({n}^2 voxels, {SMALL['frames']} frames, {SMALL['ns']} samples "
                   f"per frame from {SMALL['interleaves']} interleaves, the {len(D)}-atom grid, K = {big.rank}, "
                   f"{big.patch}x{big.patch} patches at stride {big.stride}, {big.knn} neighbours): each variant's "
                   f"maps after {iters} iterations against the FP64 oracle's Algorithm 1 after {iters} iterations "
                   f"(each side estimates its own scales a and gamma), over the object mask",
           "oracle_nrmse_vs_truth": {nm: _nrmse(inp[nm], orc[nm], mask) for nm in ("t1", "t2", "pd")}}
    for v, (t1, t2, pd, idx) in gpu.items():
        e = {"t1": _nrmse(orc["t1"], t1, mask), "t2": _nrmse(orc["t2"], t2, mask),
             "pd": _nrmse(orc["pd"], pd, mask)}
        if v != "learned":
            e["index_agreement"] = float((idx.ravel() == orc["idx"].ravel()).mean())
        e["nrmse_vs_truth"] = {nm: _nrmse(inp[nm], x, mask) for nm, x in (("t1", t1), ("t2", t2), ("pd", pd))}
        out[v] = e
    return out, orc


def c1_line(out_dir, proc, reps=20):
    """The 64^2 x 100 plain workload: A^H gridding of the 100 frames then
    exhaustive FP32 matching of the full 100-frame fingerprints
    (mrf_gridding_match), GPU timed with CUDA events, against the oracle."""
    import numpy as np
    import torch

    import synth
    import paper_2310_05647_gb300 as mrf

    inp = _wait_file(os.path.join(out_dir, "c1_inputs.npz"), proc)
    c1 = synth.WORKLOADS["mrf64_t100"]
    dev = torch.device("cuda")
    plan = mrf.nufft_plan(c1.n, c1.n, torch.tensor(inp["k"], dtype=torch.float32, device=dev), os=c1.os,
                          kb_width=c1.kb_width)
    b = torch.tensor(inp["b"], dtype=torch.complex64, device=dev)
    D = torch.tensor(inp["D"], dtype=torch.complex64, device=dev)
    lut = torch.tensor(inp["lut"], dtype=torch.float32, device=dev)
    res = mrf.gridding_match(plan, b, D, lut)
    torch.cuda.synchronize()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    ms = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = mrf.gridding_match(plan, b, D, lut)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    idx, pd, t1t2 = (t.cpu().numpy() for t in res)
    tc = mrf.gridding_match(plan, b, D, lut, precision=2)
    ms_tc = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        tc = mrf.gridding_match(plan, b, D, lut, precision=2)
        e1.record()
        torch.cuda.synchronize()
        ms_tc.append(e0.elapsed_time(e1))
    tc_idx = tc[0].cpu().numpy()
    orc = _wait_file(os.path.join(out_dir, "c1_oracle.npz"), proc)
    mask = inp["mask"].astype(bool)
    shp = (c1.n, c1.n)
    g = {"t1": t1t2[:, 0].reshape(shp), "t2": t1t2[:, 1].reshape(shp), "pd": pd.reshape(shp)}
    orc = {k: (v.reshape(shp) if np.ndim(v) == 1 else v) for k, v in orc.items()}
    return {"workload": "mrf64_t100", "what": "A^H gridding of 100 frames (64^2, 512 golden-angle spiral samples "
                                              "per frame) then exhaustive FP32 matching of the 100-frame "
                                              "fingerprints against 1500 EPG atoms (mrf_gridding_match)",
            "gpu_ms": statistics.median(ms), "oracle_ms": 1e3 * float(orc["seconds"]),
            "gpu_ms_split_bf16_tensor": statistics.median(ms_tc),
            "index_agreement_split_bf16_vs_oracle": float((tc_idx == orc["idx"].ravel()).mean()),
            "speedup_vs_oracle": 1e3 * float(orc["seconds"]) / statistics.median(ms),
            "l2": "flushed before every timed call",
            "index_agreement_vs_oracle": float((idx == orc["idx"].ravel()).mean()),
            "nrmse_vs_oracle": {nm: _nrmse(orc[nm], g[nm], mask) for nm in ("t1", "t2", "pd")},
            "nrmse_vs_truth": {"t1": _nrmse(inp["t1"], g["t1"], mask), "t2": _nrmse(inp["t2"], g["t2"], mask),
                               "pd_after_global_scale": _nrmse(inp["pd"], g["pd"] * _ls_scale(g["pd"], inp["pd"], mask),
                                                               mask)},
            "pd_note": "A^H b carries no density compensation, so PD is in arbitrary units: its error against the "
                       "truth is taken after the least-squares global scale"}


def _ls_scale(est, ref, mask):
    import numpy as np
    e, r = np.asarray(est, np.float64)[mask], np.asarray(ref, np.float64)[mask]
    den = float(np.dot(e, e))
    return float(np.dot(e, r)) / den if den > 0 else 1.0


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def roof_entry(kname, kms, inp, peaks, hbm_peak, peak_src):
    """Roofline record of one kernel from its mean launch duration (ms) and its
    algorithmic work per launch."""
    work = algorithmic_work(kname, inp)
    if work and work[0] == "hbm":
        ach = work[1] / (kms * 1e-3) / 1e9
        return {"kernel": kname, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "peak_source": peak_src, "traffic": None,
                "algorithmic_bytes_per_launch": work[1], "ms_per_launch": kms}
    if work and work[0] == "tensor":
        peak = peaks.get("bf16_tflops_sustained", 1716.1)
        ach = work[1] / (kms * 1e-3) / 1e12
        return {"kernel": kname, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": "of measured (bf16 sustained)",
                "issued_flops_per_launch": work[1] * 3 if kname == "k_match_tc" else work[1],
                "traffic": MEASURED_TRAFFIC.get(kname, (None,))[0],
                "traffic_source": MEASURED_TRAFFIC.get(kname, (None, None))[1],
                "algorithmic_flops_per_launch": work[1], "ms_per_launch": kms}
    if work and work[0] == "alu":
        peak = 152 * 128 * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        ach = work[1] / (kms * 1e-3) / 1e12
        roof = {"kernel": kname, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "peak_source": "FP32 FMA: 152 SMs x 128 lanes x 2 x max SM clock",
                "traffic": MEASURED_TRAFFIC.get(kname, (None,))[0],
                "traffic_source": MEASURED_TRAFFIC.get(kname, (None, None))[1],
                "ms_per_launch": kms}
        if kname == "k_svt":
            roof["executed_flops_per_launch"] = work[1]
            roof["svt_work"] = inp.get("svt_work")
            roof["flops_note"] = ("the SVD is iterative: executed flops from the kernel's own sweep and "
                                  "rotation counters, not a fixed algorithmic count")
            hb = svt_hbm_bytes(inp)
            roof["algorithmic_hbm_bytes_per_launch"] = hb
            roof["hbm_frac"] = hb / (kms * 1e-3) / 1e9 / hbm_peak
        else:
            roof["algorithmic_flops_per_launch"] = work[1]
        return roof
    return {"kernel": kname, "bound": None, "ms_per_launch": kms, "note": "no algorithmic-work model for this kernel"}


def svt_hbm_bytes(inp):
    """HBM bytes of one SVT launch: every patch's p^2 x K coefficients read and
    its P written (c64), and its K x K right singular vectors read and written."""
    w = inp["w"]
    cnt = (w.n - w.patch) // w.stride + 1 + (1 if (w.n - w.patch) % w.stride else 0)
    return cnt * cnt * (2 * w.patch ** 2 * w.rank * 8 + 2 * w.rank * w.rank * 8)


ROOF_KERNELS = {"chosen": ["k_match_tc", "k_svt", "k_knn_tc", "k_graph_blocks"],
                "plain": ["k_rows_fwd_expand", "k_cols_interp", "k_spread_gather", "k_rows_adj_reduce", "k_match_fp32"]}


def run_reference(args, dist):
    if dist.rank != 0:
        return
    times, walls = [], []
    sample = ""
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s, _, sample = oracle_iteration_seconds()
        wall = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(s)
            walls.append(wall)
    sec = statistics.mean(times)
    val = 1.0 / sec
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "implementation": "FP64 CPU oracle (NumPy), literal full-frame form"},
            "cpu_baseline": {"kind": "oracle", "value": val, "unit": "iters/s", "cores": cores(), "sample": sample,
                             "extrapolated": True,
                             "method": "each step times every stage of one full-size iteration on a bounded sample "
                                       "and scales it to the full workload; ms_per_step is that extrapolated "
                                       "iteration time, not the wall time of the step",
                             "sample_wall_seconds_per_step": statistics.mean(walls)},
            "e2e": {"value": val, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, dist):
    import torch

    import paper_2310_05647_gb300 as mrf
    from paper_2310_05647_gb300 import build

    build.build()
    torch.cuda.set_device(dist.local)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    if args.only_full_length_matching:
        print(json.dumps({"full_length_matching": full_length_matching(peaks, reps=1,
                                                                       n=args.only_full_length_matching)}))
        return
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    leg, leg_dir = None, None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline and not args.no_oracle_parity:
        # the oracle runs beside the GPU work (one host thread); its results are read at the end
        leg_dir = tempfile.mkdtemp(prefix="mrf_oracle_")
        leg = start_oracle_leg(leg_dir, synth_iters())
    inp = make_inputs(seed=dist.rank)
    w = inp["w"]
    variants = [v for v in args.variants.split(",") if v]
    training = None
    if "learned" in variants:
        inp["mlp"], training = train_learned(inp, seed=dist.rank)
    res = {}
    for v in variants:
        res[v] = time_variant(v, inp, args.steps, args.warmup, dist)
        res[v]["serial"] = profile_serial(v, inp, iters=10 if v != "plain" else 3)
    main = "chosen" if "chosen" in res else variants[0]
    r = res[main]
    ms_step = dist.max(r["ms"]) / args.steps
    value = dist.world * 1000.0 / ms_step
    # dominant kernel of the main variant, from its serialised profile
    if "serial" in r:
        prof, serial_ms, serial_iters, inp["svt_work"] = r["serial"]
    else:
        prof, serial_ms, serial_iters = r["profile"], r["ms"] / args.steps, args.steps
    kname = max(prof, key=lambda k: prof[k][0]) if prof else None
    roof = None
    if kname:
        roof = roof_entry(kname, prof[kname][0] / max(prof[kname][1], 1), inp, peaks, hbm_peak, peak_src)
    if roof is not None:
        cp = r["profile"]
        roof["timing"] = ("kernel duration from a serialised pass of the same loop (CUDA events on the launching "
                          "stream, %d iterations, %.3f ms per iteration); in the concurrent timed loop the kernel "
                          "shares the SMs with other steps" % (serial_iters, serial_ms))
        if kname in cp:
            roof["ms_per_launch_in_concurrent_loop"] = cp[kname][0] / max(cp[kname][1], 1)
    kernels = {k: {"ms_per_step": v[0] / serial_iters, "launches": v[1]} for k, v in
               sorted(prof.items(), key=lambda kv: -kv[1][0])}
    line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": dist.world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": w.n, "frames": w.frames, "samples_per_frame": w.ns,
                       "interleaves": w.interleaves, "grid": w.os * w.n, "kb_width": w.kb_width,
                       "atoms": inp["atoms"], "rank": w.rank, "patch": w.patch, "stride": w.stride,
                       "knn": w.knn, "variant": main, "l2": "flushed (256 MiB write) before every timed step",
                       "parallelism": f"{dist.world} independent slices (weak)"},
            "variants": {v: {"iters_per_s": 1000.0 * args.steps / res[v]["ms"],
                             "ms_per_step": res[v]["ms"] / args.steps, "nrmse_vs_truth": res[v]["nrmse"],
                             "lam1": res[v]["info"]["lam1"],
                             "top_kernels_ms_per_step": (
                                 {k: round(t[0] / res[v]["serial"][2], 4) for k, t in
                                  sorted(res[v]["serial"][0].items(), key=lambda kv: -kv[1][0])[:8]}
                                 if "serial" in res[v] else
                                 {k: round(t[0] / args.steps, 4) for k, t in
                                  sorted(res[v]["profile"].items(), key=lambda kv: -kv[1][0])[:8]}),
                             "serial_ms_per_step": res[v]["serial"][1] if "serial" in res[v] else None,
                             "top_kernels_concurrent_ms_per_step": {
                                 k: round(t[0] / args.steps, 4) for k, t in
                                 sorted(res[v]["profile"].items(), key=lambda kv: -kv[1][0])[:8]}}
                         for v in res},
            "roofline": roof, "kernels": kernels, "clocks": r["clocks"], "gpu_launches": r["launches"]}
    if "learned" in res:
        import numpy as np
        lv = line["variants"]["learned"]
        lv["training"] = training
        lv["fallback_fraction"] = res["learned"]["fallback"]
        if "chosen" in res:
            a, b = res["chosen"]["maps"], res["learned"]["maps"]
            mask = inp["truth"][3]
            lv["nrmse_vs_exhaustive"] = {nm: float(np.sqrt(np.sum((b[i][mask] - a[i][mask]) ** 2) /
                                                           np.sum(a[i][mask] ** 2)))
                                         for i, nm in enumerate(("t1", "t2", "pd"))}
    if "plain" in res and "chosen" in res:
        import numpy as np
        a, b = res["plain"]["maps"], res["chosen"]["maps"]
        mask = inp["truth"][3]
        line["chosen_vs_plain_nrmse"] = {nm: float(np.sqrt(np.sum((b[i][mask] - a[i][mask]) ** 2) /
                                                           np.sum(a[i][mask] ** 2)))
                                         for i, nm in enumerate(("t1", "t2", "pd"))}
    if "chosen" in res:
        line["precision_variants"] = {
            "what": "matching of the chosen run's final iterate (256^2 fingerprints x %d atoms, K = %d): device "
                    "ms per mrf_match call, index agreement and map NRMSE vs FP32 exhaustive matching"
                    % (inp["atoms"], w.rank),
            **precision_variants(inp, res["chosen"]["alpha"])}
    if dist.world == 1:
        line["full_length_matching"] = full_length_matching(peaks)
    if not args.no_serving and dist.world == 1:
        line["serving"] = serving(seed=dist.rank)
    if not args.no_e2e:
        sec, h2d, d2h = e2e_chosen(inp, w.iters)
        sec = dist.max(sec)
        line["e2e"] = {"value": dist.world * w.iters / sec, "unit": "iters/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h,
                       "what": f"one mrf_recon_run_host call per step: pinned host k-space -> device, init "
                               f"(A^H b, matching, graph), {w.iters} iterations, T1/T2/PD maps -> host"}
    for v, names in ROOF_KERNELS.items():
        if v not in res:
            continue
        pv, iv = (res[v]["serial"][0], res[v]["serial"][2]) if "serial" in res[v] else (res[v]["profile"], args.steps)
        ents = [roof_entry(k, pv[k][0] / max(pv[k][1], 1), inp, peaks, hbm_peak, peak_src) for k in names if k in pv]
        line.setdefault("roofline_kernels", {})[v] = [
            {kk: e[kk] for kk in ("kernel", "bound", "achieved", "peak", "unit", "frac", "ms_per_launch",
                                  "algorithmic_bytes_per_launch", "algorithmic_flops_per_launch",
                                  "executed_flops_per_launch", "hbm_frac") if kk in e} for e in ents]
    orc = None
    if leg is not None:
        # failures here are reported in the line, which is still printed
        try:
            line["nrmse_vs_oracle"], orc = small_problem_parity(leg_dir, leg, variants, synth_iters())
        except Exception as exc:
            line["nrmse_vs_oracle"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        try:
            line["c1"] = c1_line(leg_dir, leg)
        except Exception as exc:
            line["c1"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        try:
            leg.wait(timeout=900)
        except subprocess.TimeoutExpired:
            leg.kill()
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        sec, parts, sample = oracle_iteration_seconds()
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "iters/s", "cores": cores(), "kind": "oracle",
                                "sample": sample, "seconds_by_step": parts, "extrapolated": True,
                                "method": "each step of one full-size iteration timed on a bounded sample (frames, "
                                          "voxels, patches, graph rows) and scaled to the full workload; not a "
                                          "timed full iteration"}
        if orc is not None:
            its = [float(x) for x in orc["its"]]
            line["cpu_baseline"]["measured_reduced_problem"] = {
                "what": "the oracle's Algorithm 1 timed in full on the reduced copy of the problem (64^2 voxels, "
                        "100 frames, same dictionary grid, rank, patches and neighbours)",
                "seconds_per_iteration": statistics.mean(its), "iters_per_s": 1.0 / statistics.mean(its),
                "init_seconds": float(orc["init_s"]), "iterations": len(its), "cores": 1,
                "blas_threads": 1}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def synth_iters():
    import synth
    return synth.WORKLOADS["mrf256_t1000"].iters


def main():
    global WORKLOAD
    args = parse()
    WORKLOAD = args.workload
    if args.oracle_leg:
        oracle_leg(args.oracle_leg, args.steps)
        return
    dist = Dist()
    try:
        if args.impl == "reference":
            run_reference(args, dist)
        else:
            run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
