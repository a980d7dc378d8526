"""ctypes declarations of the C ABI in include/mrf.h (argument marshalling only).

Loading fails loudly (ImportError) when libmrf.so has not been built: there is
no CPU or PyTorch fallback for any operation of this package.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmrf.so")

vp = C.c_void_p
i32 = C.c_int
f32 = C.c_float
f64p = C.POINTER(C.c_double)


class ReconParams(C.Structure):
    """Mirror of mrf_recon_params."""
    _fields_ = [("mu", f32), ("lam1_0", f32), ("lam2", f32), ("beta", f32),
                ("patch", i32), ("stride", i32), ("knn", i32), ("power_iters", i32),
                ("pd_target", f32), ("a_norm", f32), ("x_scale", f32),
                ("flags", i32), ("match_precision", i32), ("mlp", vp)]


# name -> (restype, argtypes); every entry point declared in include/mrf.h
SIGNATURES = {
    "mrf_last_error": (C.c_char_p, []),
    "mrf_abi_version": (i32, []),
    "mrf_nufft_plan": (i32, [C.POINTER(vp), i32, i32, i32, i32, vp, i32, i32, vp]),
    "mrf_nufft_destroy": (i32, [vp]),
    "mrf_nufft_forward": (i32, [vp, vp, vp, vp]),
    "mrf_nufft_adjoint": (i32, [vp, vp, vp, vp]),
    "mrf_nufft_forward_subspace": (i32, [vp, vp, vp, i32, f32, vp, vp, i32, vp]),
    "mrf_nufft_adjoint_subspace": (i32, [vp, vp, vp, i32, f32, vp, i32, vp]),
    "mrf_epg_fisp": (i32, [vp, i32, vp, vp, i32, f32, f32, i32, vp, vp]),
    "mrf_dict_subspace": (i32, [vp, i32, i32, i32, vp, vp, vp, vp]),
    "mrf_match": (i32, [vp, i32, i32, vp, vp, vp, i32, i32, vp, vp, vp, vp]),
    "mrf_match_seeded": (i32, [vp, i32, i32, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp]),
    "mrf_match_noalloc": (i32, [vp, i32, i32, vp, vp, vp, i32, i32, vp, vp, vp, vp]),
    "mrf_gridding_match": (i32, [vp, vp, vp, vp, vp, i32, i32, vp, vp, vp, vp, vp]),
    "mrf_recon_run_host": (i32, [vp, C.POINTER(ReconParams), vp, i32, vp, vp, vp, i32, vp, i32, vp, vp, vp,
                                 f64p, vp]),
    "mrf_nufft_gather_tuning": (i32, [vp, C.POINTER(i32), C.POINTER(i32)]),
    "mrf_nufft_tuning": (i32, [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]),
    "mrf_patch_knn": (i32, [vp, i32, i32, i32, i32, vp, vp, vp]),
    "mrf_patch_knn_seeded": (i32, [vp, i32, i32, i32, i32, vp, vp, vp, vp]),
    "mrf_graph_sigma2": (i32, [vp, i32, vp, vp]),
    "mrf_batch_create": (i32, [C.POINTER(vp), C.POINTER(vp), i32, vp]),
    "mrf_batch_iter": (i32, [vp, i32, vp]),
    "mrf_batch_destroy": (i32, [vp]),
    "mrf_wait_selftest": (i32, [i32, vp]),
    "mrf_mlp_create": (i32, [C.POINTER(vp), vp, i32, vp, i32]),
    "mrf_mlp_destroy": (i32, [vp]),
    "mrf_mlp_get_params": (i32, [vp, vp, vp]),
    "mrf_mlp_grad": (i32, [vp, vp, vp, i32, vp, vp, vp]),
    "mrf_mlp_train_step": (i32, [vp, vp, vp, i32, f32, vp, vp]),
    "mrf_mlp_infer": (i32, [vp, vp, i32, vp, vp]),
    "mrf_mlp_set_engine": (i32, [vp, i32]),
    "mrf_mlp_check": (i32, [vp, vp]),
    "mrf_mlp_training_set": (i32, [vp, vp, vp, vp, vp, i32, i32, vp, i32, vp, vp, vp, vp]),
    "mrf_recon_checkpoint_size": (i32, [vp, C.POINTER(C.c_size_t)]),
    "mrf_recon_checkpoint": (i32, [vp, vp, C.c_size_t, vp]),
    "mrf_recon_restore": (i32, [vp, vp, C.c_size_t, vp]),
    "mrf_recon_create": (i32, [C.POINTER(vp), vp, C.POINTER(ReconParams), vp, i32, vp, vp, vp, i32, vp, vp]),
    "mrf_recon_iter": (i32, [vp, i32, f64p, vp]),
    "mrf_recon_maps": (i32, [vp, vp, vp, vp, vp, vp]),
    "mrf_recon_alpha": (i32, [vp, vp, vp]),
    "mrf_recon_info": (i32, [vp, f64p, f64p, f64p, f64p, vp]),
    "mrf_recon_svt_stats": (i32, [vp, f64p, f64p, f64p, vp]),
    "mrf_recon_destroy": (i32, [vp]),
    "mrf_launch_count": (C.c_longlong, []),
    "mrf_profile_enable": (i32, [i32]),
    "mrf_profile_mark": (i32, [vp]),
    "mrf_profile_collect": (i32, []),
    "mrf_profile_entry": (i32, [i32, C.c_char_p, i32, f64p, C.POINTER(C.c_longlong)]),
}

STATUS = {0: "MRF_OK", 1: "MRF_EINVAL", 2: "MRF_ENOMEM", 3: "MRF_ECUDA", 4: "MRF_ETIMEOUT",
          5: "MRF_EUNSUPPORTED"}


class MRFError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn} -> {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libmrf.so once and attach the signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def call(name, *args):
    """Call an entry point and raise MRFError on a non-zero status."""
    lib = load()
    st = getattr(lib, name)(*args)
    if st != 0:
        raise MRFError(name, st, lib.mrf_last_error().decode(errors="replace"))
    return st
