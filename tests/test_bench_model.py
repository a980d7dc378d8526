"""The work model behind bench.py's roofline object, on CPU: the per-launch
flops and bytes it reports for the benchmark workload (256^2, 5441 atoms,
K = 10, 3969 patches of 8 x 8) follow the formulas stated beside them."""
import pytest

import bench
import synth


def _inp():
    return {"w": synth.WORKLOADS["mrf256_t1000"], "atoms": 5441}


def test_tensor_matcher_flops():
    kind, flops = bench.algorithmic_work("k_match_tc", _inp())
    assert kind == "tensor"
    assert flops == 2.0 * 65536 * (2 * 5441) * (2 * 10)           # 28.5 GFLOP
    assert flops == pytest.approx(28.53e9, rel=1e-3)


def test_svt_executed_flops():
    work = {"sweeps_per_patch": 5.409, "rotations_per_patch": 164.89}
    inp = dict(_inp(), svt_work=work)
    kind, flops = bench.algorithmic_work("k_svt", inp)
    assert kind == "alu"
    pp, KP, K, npatch = 64, 10, 10, 63 * 63
    per_sweep = 4 * pp * KP + 8 * pp * (KP // 2) * (KP - 1)
    per_rot = 18 * (pp + KP)
    fixed = 8 * pp * KP * KP + 4 * pp * KP + 10 * pp * K * KP
    assert flops == pytest.approx(npatch * (5.409 * per_sweep + 164.89 * per_rot + fixed), rel=1e-12)
    assert flops == pytest.approx(1.887e9, rel=2e-3)
    # without counters there is no SVT model
    assert bench.algorithmic_work("k_svt", _inp()) is None
