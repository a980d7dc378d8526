"""Pins of the oracle's dictionary, subspace and matching (Eq. 3, 5, 14)."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import dictionary, match

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_paper_dictionary_size():
    t1, t2 = synth.paper_grid()
    assert len(t1) == GOLDEN["dictionary_t1_count"]["value"]
    assert len(t2) == GOLDEN["dictionary_t2_count"]["value"]
    assert len(synth.keep_t1_ge_t2(t1, t2)) == GOLDEN["dictionary_size"]["value"]


@pytest.fixture(scope="module")
def small_dict():
    fa, tr = synth.fisp_train(60, seed=2)
    lut = synth.keep_t1_ge_t2(synth.log_grid(200, 3000, 12), synth.log_grid(20, 400, 9))
    return lut, dictionary.simulate(lut, fa, tr)


def _brute(x, D):
    best, bi = -1.0, -1
    for m in range(D.shape[0]):
        num = abs(sum(np.conj(D[m, t]) * x[t] for t in range(D.shape[1])))
        sc = num / np.sqrt(sum(abs(D[m, t]) ** 2 for t in range(D.shape[1])))
        if sc > best:
            best, bi = sc, m
    return bi


def test_noiseless_atoms_match_themselves(small_dict):
    lut, D = small_dict
    rng = np.random.default_rng(0)
    pd = rng.uniform(0.2, 3.0, D.shape[0])
    idx, t1, t2, pdh = match.match(D * pd[:, None], D, lut)
    np.testing.assert_array_equal(idx, np.arange(D.shape[0]))
    np.testing.assert_allclose(pdh, pd, rtol=1e-12)
    np.testing.assert_array_equal(t1, lut[:, 0])
    np.testing.assert_array_equal(t2, lut[:, 1])


def test_matches_brute_force(small_dict):
    lut, D = small_dict
    rng = np.random.default_rng(1)
    X = D[rng.integers(0, D.shape[0], 6)] + 0.05 * (rng.standard_normal((6, D.shape[1]))
                                                   + 1j * rng.standard_normal((6, D.shape[1])))
    idx, *_ = match.match(X, D, lut)
    assert list(idx) == [_brute(x, D) for x in X]


def test_pd_clamp_and_phase(small_dict):
    lut, D = small_dict
    X = np.stack([-2.0 * D[5], 1.5 * np.exp(1j * 0.7) * D[9], np.zeros(D.shape[1])])
    idx, _, _, pd = match.match(X, D, lut)
    assert idx[0] == 5 and pd[0] == 0.0                  # negatively phased: PD clamped
    assert idx[1] == 9 and pd[1] == pytest.approx(1.5 * np.cos(0.7), rel=1e-12)
    assert idx[2] == 0 and pd[2] == 0.0                  # air: lowest index, PD 0


def test_literal_norm2_reading_differs():
    # two atoms along the same direction with different norms: the printed
    # ||d||^2 denominator prefers the smaller atom, the ||d|| reading ties and
    # keeps the lower index.
    D = np.array([[2.0, 0.0], [1.0, 0.0], [0.0, 1.0]], complex)
    lut = np.array([[1.0, 1.0], [2.0, 2.0], [3.0, 3.0]])
    x = np.array([[1.0, 0.1]], complex)
    assert match.match(x, D, lut)[0][0] == 0
    assert match.match(x, D, lut, literal_norm2=True)[0][0] == 1


def test_subspace_orthonormal_and_projection_idempotent(small_dict):
    _, D = small_dict
    phi = dictionary.subspace(D, 6)
    np.testing.assert_allclose(phi.conj().T @ phi, np.eye(6), atol=1e-12)
    X = D[:7] + 0.1
    P1 = dictionary.project(X, phi)
    np.testing.assert_allclose(dictionary.project(P1, phi), P1, atol=1e-12)
    # the SVD basis captures almost all dictionary energy (McGivney et al.)
    cap = np.linalg.norm(dictionary.project(D, phi)) / np.linalg.norm(D)
    assert cap > 0.999


def test_subspace_matching_equals_full_matching_on_s(small_dict):
    # for X in S, <d, X> = <d Phi, X Phi>: compressed atoms with full norms give
    # exactly the full-length result
    lut, D = small_dict
    phi = dictionary.subspace(D, 5)
    rng = np.random.default_rng(2)
    alpha = rng.standard_normal((20, 5)) + 1j * rng.standard_normal((20, 5))
    X = alpha @ phi.conj().T
    full = match.match(X, D, lut)
    comp = match.match(alpha, D @ phi, lut, atom_norm2=np.sum(np.abs(D) ** 2, 1))
    np.testing.assert_array_equal(full[0], comp[0])
    np.testing.assert_allclose(full[3], comp[3], rtol=1e-10, atol=1e-12)


def test_workload_grids():
    w = synth.WORKLOADS["mrf64_t100"]
    assert len(synth.workload_grid(w)) == 1500
    w = synth.WORKLOADS["mrf256_t1000"]
    lut = synth.workload_grid(w)
    assert 5000 < len(lut) <= 6000
    assert np.all(lut[:, 0] >= lut[:, 1])
