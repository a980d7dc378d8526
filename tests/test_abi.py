"""CPU checks of the C ABI: the library builds, loads without a GPU, exports
every entry point declared in include/mrf.h, and rejects bad arguments on the
host before any CUDA call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_05647_gb300 import build, _lib
    build.build()
    return _lib.load()


def declared():
    src = open(os.path.join(ROOT, "include", "mrf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mrf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for n in ["mrf_nufft_plan", "mrf_nufft_forward", "mrf_nufft_adjoint", "mrf_match", "mrf_recon_iter",
              "mrf_recon_create", "mrf_epg_fisp", "mrf_dict_subspace", "mrf_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2310_05647_gb300 import _lib
    for n in declared():
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, f"{n} missing from the Python binding"
    assert lib.mrf_abi_version() == 1


def _err(lib):
    return lib.mrf_last_error().decode()


def test_host_validation_without_gpu(lib):
    h = C.c_void_p()
    dummy = C.c_void_p(16)
    assert lib.mrf_nufft_plan(C.byref(h), 32, 32, 4, 10, dummy, 3, 4, None) == 1
    assert "os" in _err(lib)
    assert lib.mrf_nufft_plan(C.byref(h), 32, 32, 4, 10, dummy, 2, 5, None) == 1
    assert lib.mrf_nufft_plan(C.byref(h), 33, 32, 4, 10, dummy, 2, 4, None) == 1
    assert lib.mrf_nufft_plan(C.byref(h), 600, 600, 4, 10, dummy, 2, 4, None) == 1
    assert lib.mrf_nufft_plan(C.byref(h), 32, 32, 4, 10, None, 2, 4, None) == 1
    assert lib.mrf_match(None, 4, 10, dummy, None, dummy, 5, 0, None, None, None, None) == 1
    assert lib.mrf_match(dummy, 4, 0, dummy, None, dummy, 5, 0, None, None, None, None) == 1
    assert lib.mrf_match(dummy, 4, 10, dummy, None, dummy, 5, 7, None, None, None, None) == 1
    assert lib.mrf_match(dummy, 4, 10, dummy, None, dummy, 5, 0x101, None, None, None, None) == 1
    assert lib.mrf_epg_fisp(dummy, 3, dummy, dummy, 0, C.c_float(2.94), C.c_float(20.0), 1, dummy, None) == 1
    assert lib.mrf_epg_fisp(dummy, 3, dummy, dummy, 5000, C.c_float(2.94), C.c_float(20.0), 1, dummy, None) == 1
    assert lib.mrf_nufft_forward(None, dummy, dummy, None) == 1
    assert lib.mrf_gridding_match(None, dummy, dummy, None, dummy, 5, 0, None, None, None, None, None) == 1
    assert lib.mrf_gridding_match(dummy, dummy, dummy, None, dummy, 0, 0, None, None, None, None, None) == 1
    assert lib.mrf_recon_run_host(None, None, dummy, 10, dummy, dummy, dummy, 5, dummy, 1, None, None, None,
                                  None, None) == 1
    assert lib.mrf_match(dummy, 0, 10, dummy, None, dummy, 5, 0, None, None, None, None) == 0   # empty: no-op


def test_host_validation_of_seeded_matching_knn_sigma2_and_svt_counters(lib):
    dummy = C.c_void_p(16)
    d = [C.c_double() for _ in range(3)]
    # seeded matching: only the BF16 forms, and a candidate buffer unless n == 0
    assert lib.mrf_match_seeded(dummy, 4, 10, dummy, None, dummy, 5, 0, dummy, None, None, None, None) == 1
    assert "precision" in _err(lib)
    assert lib.mrf_match_seeded(dummy, 4, 10, dummy, None, dummy, 5, 3, dummy, None, None, None, None) == 1
    assert lib.mrf_match_seeded(dummy, 4, 10, dummy, None, dummy, 5, 2, None, None, None, None, None) == 1
    assert "cand" in _err(lib)
    assert lib.mrf_match_seeded(dummy, 0, 10, dummy, None, dummy, 5, 2, None, None, None, None, None) == 0
    # sigma^2: negative counts and null pointers
    assert lib.mrf_graph_sigma2(dummy, -1, dummy, None) == 1
    assert lib.mrf_graph_sigma2(None, 5, dummy, None) == 1
    assert lib.mrf_graph_sigma2(dummy, 5, None, None) == 1
    # seeded kNN: the seed list is required
    assert lib.mrf_patch_knn_seeded(dummy, 20, 8, 8, 4, None, dummy, dummy, None) == 1
    assert "seed" in _err(lib)
    # SVT work counters of no reconstruction
    assert lib.mrf_recon_svt_stats(None, *[C.byref(v) for v in d], None) == 1
    assert lib.mrf_recon_svt_stats(dummy, None, C.byref(d[1]), C.byref(d[2]), None) == 1


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2310_05647_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()
