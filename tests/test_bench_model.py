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
    """Gram matrix + two-sided Jacobi on the K x K matrix: fixed work per patch
    (Gram 8 pp NG, V transforms 24 KP^3, column norms 8 pp KP^2, M 8 KP^2 K,
    P 8 pp KP K) plus per-sweep and per-rotation work, for KP = K = 10, 8 x 8
    patches, 3969 patches."""
    work = {"sweeps_per_patch": 3.0, "rotations_per_patch": 40.0}
    inp = dict(_inp(), svt_work=work)
    kind, flops = bench.algorithmic_work("k_svt", inp)
    assert kind == "alu"
    fixed = 8 * 64 * 55 + 24 * 1000 + 8 * 64 * 100 + 8 * 100 * 10 + 8 * 64 * 100      # 162560
    per_sweep = 9 * (56 * 10 + 14 * 10 * 5)                                            # 11340
    assert fixed == 162560 and per_sweep == 11340
    assert flops == pytest.approx(3969 * (3.0 * per_sweep + 40.0 * 30 + fixed), rel=1e-12)
    assert flops == pytest.approx(0.785e9, rel=2e-3)
    # without counters there is no SVT model
    assert bench.algorithmic_work("k_svt", _inp()) is None
