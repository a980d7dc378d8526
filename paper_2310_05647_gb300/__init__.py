"""GB300 (sm_103a) hot path of the MS-LLR MR-fingerprinting reconstruction.

Thin PyTorch-facing binding over the C ABI of ``include/mrf.h``: tensors are
passed as device pointers plus the current CUDA stream; every computation runs
in this package's CUDA kernels (``csrc/``).  Importing the package does not
touch the GPU; the first call loads ``libmrf.so`` and fails loudly if it has
not been built.
"""
from .api import (Batch, MRFError, Mlp, NufftPlan, Recon, ReconParams, mlp_training_set, train_matcher, dict_subspace, epg_fisp, gridding_match, launch_count, match, match_seeded,
                  nufft_adjoint, nufft_adjoint_subspace, nufft_forward, nufft_forward_subspace,
                  nufft_plan, patch_knn, graph_sigma2, profile_enable, profile_mark, profile_read, recon_run_host,
                  wait_selftest)

__all__ = ["Batch", "MRFError", "Mlp", "mlp_training_set", "train_matcher", "NufftPlan", "Recon", "ReconParams", "dict_subspace", "epg_fisp", "gridding_match", "match", "match_seeded",
           "nufft_adjoint", "nufft_adjoint_subspace", "nufft_forward", "nufft_forward_subspace",
           "nufft_plan", "patch_knn", "graph_sigma2", "launch_count", "profile_enable", "profile_mark", "profile_read",
           "recon_run_host", "wait_selftest"]
