"""CPU FP64 oracle for the MS-LLR MR-fingerprinting reconstruction.

TEST INFRASTRUCTURE ONLY.  Plain, slow, obviously-correct NumPy code written
from the paper (Li, Ji, Hu, "Exploiting Manifold Structured Data Priors for
Improved MR Fingerprinting Reconstruction").  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it.  It shares no code with the CUDA path and never imports the package.

Modules
  kb        Kaiser-Bessel kernel psi, its Fourier transform, Beatty's beta.
  nufft     exact NUDFT (Eq. 1, A = F_u with one coil) and an FP64 KB-gridding
            NUFFT (deapodise, zero-pad, FFT, interpolate) and its adjoint.
  epg       extended-phase-graph FISP simulation, the Bloch map B(eta; theta)
            of Eq. 2 / Eq. 3.
  dictionary  dictionary D with PD = 1 (Eq. 3), look-up table, SVD subspace.
  match     dictionary matching Phi_D (Eq. 5).
  patches   patch extraction Q_q, Casorati Q and adjoint Q^* (Eq. 6, 9).
  graph     parameter-manifold weights (Eq. 7), Laplacian (Eq. 9-10), kNN graph.
  llr       singular value thresholding (Eq. 18) and the X update (Eq. 19).
  recon     Algorithm 1 (MS-LLR).
  metrics   SNR (Eq. 20) and NMSE (Eq. 21).

Parity status: every function is pinned by a ``-m "not gpu"`` test against
closed forms, library routines on special cases, brute force or independent
simulation.  ``recon.MSLLR`` end to end has no published maps to compare
against (the paper's data are unavailable); it is pinned by its steps and by
one special case with a known answer: noiseless, fully sampled data of
tissues that are dictionary atoms must give back the true maps.
"""
