/*
 * mrf.h -- C ABI of the GB300 (sm_103a) MS-LLR MR-fingerprinting hot path.
 *
 * Method: Li, Ji, Hu, "Exploiting Manifold Structured Data Priors for
 * Improved MR Fingerprinting Reconstruction" (MS-LLR).  The calls below
 * follow its problem statement b = A X + n (Eq. 1), the matching operator
 * Phi_D (Eq. 5) and Algorithm 1.
 *
 * Conventions shared by every call
 *  - Complex numbers are interleaved float pairs (mrf_c64 = {re, im}); all
 *    arrays are dense and row-major with the shapes given per argument.
 *  - "dev" pointers are CUDA device (or managed) memory of the current
 *    device; "host" pointers are ordinary host memory.  The caller owns every
 *    pointer argument; the library never frees them.  Plans and recon
 *    objects own their internal workspace and release it in *_destroy.
 *  - Every call is asynchronous and stream-ordered on `stream` (a
 *    cudaStream_t passed as void*, NULL = legacy default stream) unless its
 *    comment says it synchronises.  Inputs must stay valid until the work
 *    completes.
 *  - Sizes and pointers are validated on the host before any launch; a
 *    rejected call returns MRF_EINVAL and launches nothing.  Errors are
 *    reported as an mrf_status plus a thread-local message from
 *    mrf_last_error(); nothing is thrown across the ABI.
 *  - Image index: x[t][iy][ix] with centred coordinates
 *    n = (ix - nx/2, iy - ny/2).  k-space positions are (kx, ky) in radians
 *    per voxel in [-pi, pi).
 */
#ifndef MRF_H
#define MRF_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MRF_OK = 0,
    MRF_EINVAL = 1,        /* bad argument (size, null pointer, unsupported combination) */
    MRF_ENOMEM = 2,        /* device allocation failed */
    MRF_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    MRF_ETIMEOUT = 4,      /* a bounded device wait gave up */
    MRF_EUNSUPPORTED = 5   /* valid request this build does not implement */
} mrf_status;

typedef struct { float re, im; } mrf_c64;
typedef void* mrf_stream;                 /* cudaStream_t */
typedef struct mrf_plan_s* mrf_plan;       /* NUFFT plan (opaque) */
typedef struct mrf_recon_s* mrf_recon;     /* Algorithm 1 state (opaque) */
typedef struct mrf_batch_s* mrf_batch;     /* batch of slices advanced together (opaque) */
typedef struct mrf_mlp_s* mrf_mlp;         /* learned matcher network (opaque) */

/* Last error message of the calling thread ("" if none). */
const char* mrf_last_error(void);
/* ABI version, incremented on any signature change. */
int mrf_abi_version(void);

/* ------------------------------------------------------------------------
 * Acquisition operator A = F_u (Eq. 1 with one coil, C = I).
 * Kaiser-Bessel gridding NUFFT (the GPU NUFFT of Sec. III-D, Implementation
 * Details): A x = interp_KB(FFT_G(zero-pad(x / psi_hat))) on an os-times
 * oversampled grid G = os * n, and the exact adjoint A^H y =
 * psi_hat^-1 . crop(IFFT_G(spread_KB(y))) (unnormalised transforms, no
 * density compensation; X^0 = A^H b of Algorithm 1).
 * ---------------------------------------------------------------------- */

/* Build a plan for `nframes` frames of an ny x nx image, `ns` samples per
 * frame.  traj: dev float [nframes][ns][2] = (kx, ky) rad/voxel; read once
 * (the plan keeps its own sorted copy).  os must be 2; kb_width in {4, 6};
 * square images (nx == ny, even) with os*nx in {64, 128, 256, 512}.  Synchronises
 * `stream` (the trajectory is binned on the host).  MRF_ENOMEM if the
 * workspace (about nframes*ny*os*nx*8 bytes plus 32 bytes per sample) does
 * not fit. */
mrf_status mrf_nufft_plan(mrf_plan* out, int nx, int ny, int nframes, int ns,
                          const float* traj, int os, int kb_width, mrf_stream stream);
mrf_status mrf_nufft_destroy(mrf_plan plan);

/* Tile shape the spread autotuner chose for the grouped adjoint's gather
 * kernel (entries reduced per thread, threads per block), timed on this
 * plan's own table on its first grouped adjoint; 0, 0 before that call. */
mrf_status mrf_nufft_gather_tuning(mrf_plan plan, int* run, int* threads);
/* Everything the plan's autotuners chose for the grouped operator (0 until
 * the first grouped transform ran): the adjoint gather's entries per thread
 * and block size (as mrf_nufft_gather_tuning) and the strip width (16, 32
 * or 64 columns, 64 only where its shared tile fits) of the column FFTs of
 * the K coefficient spectra, picked by timing each candidate on the plan's
 * grid.  Each output nullable. */
mrf_status mrf_nufft_tuning(mrf_plan plan, int* gather_run, int* gather_threads, int* strip_width);

/* y = A x over all frames.  x: dev [nframes][ny][nx] mrf_c64;
 * y: dev [nframes][ns] mrf_c64 (overwritten). */
mrf_status mrf_nufft_forward(mrf_plan plan, const mrf_c64* x, mrf_c64* y, mrf_stream stream);

/* x = A^H y over all frames.  y: dev [nframes][ns]; x: dev [nframes][ny][nx]
 * (overwritten).  Spreading uses shared-memory atomics, so the float
 * summation order (and the last bits) can vary between runs. */
mrf_status mrf_nufft_adjoint(mrf_plan plan, const mrf_c64* y, mrf_c64* x, mrf_stream stream);

/* Subspace forms used by the reconstruction loop.  With X = alpha Phi^H
 * (Eq. 14, P_S(X) = X Phi Phi^H), frame t of X is x_t = sum_k alpha_k
 * conj(Phi[t][k]).
 *   forward:  y = A(alpha Phi^H) - b          (b may be NULL: no subtraction)
 *   adjoint:  alpha_out = (A^H y) Phi          i.e. alpha_out[n][k] =
 *             sum_t (A^H y)_t[n] Phi[t][k]
 * alpha: dev [ny][nx][K]; phi: dev [nframes][K]; y, b: dev [nframes][ns].
 * 1 <= K <= 16.  `scale` multiplies the operator (A/a of Algorithm 1's
 * scaled problem: pass 1/a).  mode 0 = per-frame transforms (T NUFFTs per
 * call, the literal multi-frame operator); mode 1 = grouped (the same
 * operator evaluated with K oversampled FFTs: the FFT is linear and the same
 * for every frame, so A(alpha Phi^H)_t = interp_t(sum over the K transformed
 * coefficient images weighted by conj(Phi[t][k]))).  Both modes give the
 * same values up to float rounding. */
mrf_status mrf_nufft_forward_subspace(mrf_plan plan, const mrf_c64* alpha, const mrf_c64* phi,
                                      int K, float scale, const mrf_c64* b, mrf_c64* y,
                                      int mode, mrf_stream stream);
mrf_status mrf_nufft_adjoint_subspace(mrf_plan plan, const mrf_c64* y, const mrf_c64* phi,
                                      int K, float scale, mrf_c64* alpha_out,
                                      int mode, mrf_stream stream);

/* ------------------------------------------------------------------------
 * Dictionary simulation and matching.
 * ---------------------------------------------------------------------- */

/* Dictionary atoms d_m = B(eta_m; theta) with PD = 1 (Eq. 2-3) by the
 * extended-phase-graph FISP recursion: per repetition an RF rotation of
 * flip fa_deg[t] about x, relaxation over TE, the signal F+_0, relaxation
 * over tr_ms[t] - TE and one full dephasing.  The magnetisation starts at
 * equilibrium, is inverted and relaxes ti_ms before the train when
 * `inversion` != 0.  All T+1 states are kept (no truncation).
 * t1t2: dev float [m][2] (ms); fa_deg, tr_ms: dev float [T]; out: dev
 * [m][T] mrf_c64.  1 <= T <= 4094. */
mrf_status mrf_epg_fisp(const float* t1t2, int m, const float* fa_deg, const float* tr_ms,
                        int T, float te_ms, float ti_ms, int inversion,
                        mrf_c64* out, mrf_stream stream);

/* Temporal subspace of a dictionary (Eq. 14: the orthonormal basis d of
 * P_S, approximated from D).  phi (dev [T][K]) receives the top-K right
 * singular vectors of D (dev [m][T]), computed by randomised block subspace
 * iteration on D^H D (Yang et al., cited in Sec. I) with FP64 accumulation;
 * compressed (dev [m][K], nullable) receives d_m Phi and norm2 (dev [m],
 * nullable) receives ||d_m||^2 of the full atoms.  Needs 1 <= K <= 16,
 * K + 8 <= T <= 4096.  Allocates and frees its own workspace; synchronises
 * `stream`. */
mrf_status mrf_dict_subspace(const mrf_c64* dict, int m, int T, int K, mrf_c64* phi,
                             mrf_c64* compressed, float* norm2, mrf_stream stream);

enum {
    MRF_MATCH_FP32 = 0,        /* exhaustive FP32 inner products (plain form) */
    MRF_MATCH_BF16 = 1,        /* BF16 tensor-core scores, FP32 top-8 re-rank */
    MRF_MATCH_BF16X3 = 2,      /* split BF16 (hi/lo, three products in one GEMM), FP32 top-4
                                  re-rank: tensor-core speed at ~2^-16 score error */
    MRF_MATCH_FP8 = 3,         /* FP8 e4m3 tensor-core scores (atoms scaled to unit norm x 448,
                                  fingerprints by 448 / max |x|), FP32 top-8 re-rank (len <= 64) */
    MRF_MATCH_LITERAL_NORM2 = 0x100 /* flag: argmax of |<d,x>|/||d||^2 as printed in Eq. 5 */
};

/* Phi_D of Eq. 5 for n fingerprints of length len:
 *   k_i   = argmax_m |<d_m, x_i>| / ||d_m||     (||d_m||^2 with the LITERAL flag)
 *   eta_i = LUT[k_i],  rho_i = max(Re<d_k, x_i> / ||d_k||^2, 0)
 * <a, b> = sum conj(a) b; ties go to the lowest index (an all-zero x, or
 * one whose best score is not finite -- NaN or infinite entries -- gives
 * index 0, PD 0).  x: dev [n][len]; dict: dev [m][len]; atom_norm2: dev [m]
 * ||d_m||^2 or NULL to use the rows of dict (pass the full-length norms when
 * dict holds subspace-compressed atoms d_m Phi); lut: dev float [m][2]
 * (T1, T2).  Outputs (each nullable): idx dev int [n], pd dev float [n],
 * t1t2 dev float [n][2].  1 <= len <= 2048, 1 <= m <= 2^24.  The BF16 forms
 * keep the fingerprint tile resident in shared memory while the padded
 * reduction (2 len reals, three copies for the split form) fits 128 elements
 * (len <= 64 BF16, len <= 21 split BF16), and stream both operands along the
 * reduction axis beyond that (full-length fingerprints, e.g. 1000 frames);
 * the results follow the same rules either way.  Scratch is allocated and
 * freed on the stream; a tensor-core call synchronises the stream to report
 * a device wait that gave up (MRF_ETIMEOUT). */
mrf_status mrf_match(const mrf_c64* x, int n, int len, const mrf_c64* dict,
                     const float* atom_norm2, const float* lut, int m, int precision,
                     int* idx, float* pd, float* t1t2, mrf_stream stream);

/* The plain reconstruction: X = A^H y frame by frame (the adjoint of Eq. 1,
 * the X^0 = A^* b of Algorithm 1 without the subspace projection), then
 * dictionary matching (Eq. 5) of every voxel's full fingerprint
 * X[:, iy, ix] of length T against dict.  y: dev [T][ns] of the plan;
 * dict: dev [m][T]; atom_norm2, lut, precision and the outputs idx / pd /
 * t1t2 ([ny*nx], row-major voxels) as in mrf_match with n = ny*nx and
 * len = T.  x_rows (nullable): dev [ny*nx][T], receives the fingerprints.
 * Scratch (the [T][ny][nx] adjoint output, and the rows when x_rows is NULL)
 * is allocated and freed on the stream.  Needs T <= 2048. */
mrf_status mrf_gridding_match(mrf_plan plan, const mrf_c64* y, const mrf_c64* dict,
                              const float* atom_norm2, const float* lut, int m, int precision,
                              int* idx, float* pd, float* t1t2, mrf_c64* x_rows,
                              mrf_stream stream);

/* mrf_match for repeated matching of the same n rows (an iterative
 * reconstruction matches every iterate): cand (dev int32 [n][8]) carries
 * each row's tensor-core candidates from one call to the next.  On entry
 * the first TOPK entries of row i (TOPK = 4 for MRF_MATCH_BF16X3, 8 for
 * MRF_MATCH_BF16) name seed atoms: the smallest FP32 score among them, less
 * a margin above the tensor-core score error (2^-10 ||x_i||^2 split, 2^-4
 * BF16), starts the row's candidate list, so the sweep inserts fewer atoms.
 * Any seeds give the same candidates and winners as mrf_match; seeds that
 * are not TOPK distinct indices in [0, m) (e.g. -1) leave the row unseeded.
 * On return those entries hold the row's candidates; the others are left
 * as they were.  precision: MRF_MATCH_BF16 or MRF_MATCH_BF16X3 (else
 * MRF_EINVAL), with the fingerprint tile resident (len <= 64 BF16, <= 21
 * split BF16; longer: MRF_EINVAL); other arguments as in mrf_match. */
mrf_status mrf_match_seeded(const mrf_c64* x, int n, int len, const mrf_c64* dict, const float* atom_norm2,
                            const float* lut, int m, int precision, int* cand, int* idx, float* pd,
                            float* t1t2, mrf_stream stream);

/* Same result as mrf_match with MRF_MATCH_FP32, for callers that cannot
 * allocate device memory when they match (the paper has no counterpart: this
 * is a deployment variant).  A reconstruction service that reserves the
 * GPU's memory for its own pool at start-up, or a latency-bound serving loop
 * that must not pay for cudaMalloc/cudaFree (they can block the host and
 * synchronise the device), can call this instead.  The scratch lives in one
 * fixed device array inside the library, sized for at most 262144
 * fingerprints (n) and 65536 atoms (m), about 3.6 MB that every GPU which
 * loads the library holds until the process exits; larger n or m return
 * MRF_EINVAL with a message.  Every call looks up the array's device address
 * on the current device (no allocation; a context reset cannot leave a stale
 * address behind); the first lookup on a device loads the library's module
 * there, so make that first call before any stream capture.  All calls share the one array: calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.  Every scratch word a call reads
 * is written by the same call first, so no clearing is needed between calls.
 * Arguments as in mrf_match; precision must be MRF_MATCH_FP32, optionally
 * with MRF_MATCH_LITERAL_NORM2. */
mrf_status mrf_match_noalloc(const mrf_c64* x, int n, int len, const mrf_c64* dict,
                             const float* atom_norm2, const float* lut, int m, int precision,
                             int* idx, float* pd, float* t1t2, mrf_stream stream);

/* Patch graph of Eq. 7, kept sparse: for every row i of the integer patch
 * vectors F, the knn rows j != i with the smallest squared distance
 * sum_k (F_ik - F_jk)^2 over the first fd entries, in ascending order, ties
 * to the lower j.  The distances are exact integers (Algorithm 1 builds F as
 * the 12-bit fixed point rint(4096 T / Tmax) of the matched T1 and T2 maps
 * over each patch, so tied distances are common and break alike everywhere).
 * F: dev int32 [np][ld], 0 <= F <= 4096, ld >= fd and a multiple of 4, the
 * entries fd <= k < ld zero.  nbr: dev int32 [np][knn]; d2: dev uint32
 * [np][knn].  Needs 1 <= knn <= 32, np > knn, 1 <= fd <= 255.  Scratch is
 * allocated and freed by the call, which synchronises the stream to report
 * a feature outside [0, 4096] (MRF_EINVAL) or a device wait that gave up
 * (MRF_ETIMEOUT). */
mrf_status mrf_patch_knn(const int* F, int np, int fd, int ld, int knn, int* nbr, unsigned* d2,
                         mrf_stream stream);

/* mrf_patch_knn with a seed list: seed (dev int32 [np][knn], read-only, may
 * be nbr itself) is a previous neighbour list, in the loop the graph of the
 * previous iteration.  For fd <= 128, where the seeds of row i are knn
 * distinct rows j != i, the largest distance from F_i to them bounds the
 * search for row i: no candidate farther than that can be among its knn
 * nearest, so fewer candidates pass the tensor-core epilogue.  Other seed
 * lists give no bound.  The result is the same as mrf_patch_knn's for any
 * seed values; errors as in mrf_patch_knn, plus MRF_EINVAL for a NULL seed. */
mrf_status mrf_patch_knn_seeded(const int* F, int np, int fd, int ld, int knn, const int* seed, int* nbr,
                                unsigned* d2, mrf_stream stream);

/* sigma^2 of the patch-graph weights w_ij = exp(-d2_ij / sigma^2) of Eq. 7,
 * a constant the paper does not set: the median of the non-zero entries of
 * d2 (the mean of the two middle ones for an even count), divided by 4096^2
 * so that it is in units of (T / Tmax)^2 like the distances of the 12-bit
 * patch vectors of mrf_patch_knn; 1 when no entry is non-zero (or ne == 0).
 * d2: dev uint32 [ne], any values; sigma2: dev float [1], the fp64 result
 * rounded once to float.  Asynchronous on the stream; no scratch.  ne < 0 or
 * a null pointer: MRF_EINVAL. */
mrf_status mrf_graph_sigma2(const unsigned* d2, int ne, float* sigma2, mrf_stream stream);

/* ------------------------------------------------------------------------
 * Learned matcher.  The paper's related work (Section I) cites replacing
 * dictionary matching by a fully connected network that maps a fingerprint
 * to its tissue parameters; this is that network for the subspace form:
 * 20 inputs (the K = 10 complex coefficients divided by their norm, as
 * (Re, Im) pairs) -> 3 x 256 GELU (exact erf form) -> 3 outputs
 * (u1, u2, u3): log T1 and log T2 mapped from [log Tmin, log Tmax] onto
 * [-1, 1], and PD per unit input norm divided by pd_scale.  Parameters are
 * packed per layer as W [out][in] row-major, then b [out] (137731 floats).
 * The products use a BF16 copy of the FP32 master weights (refreshed by
 * every Adam step); biases, activations and accumulation are FP32.
 * ---------------------------------------------------------------------- */
/* params: host float [137731]; decode: host float [5] = (t1min, t1max,
 * t2min, t2max, pd_scale); max_batch: rows of the largest training batch.
 * Synchronises the device. */
mrf_status mrf_mlp_create(mrf_mlp* out, const float* params, int nparams, const float* decode,
                          int max_batch);
mrf_status mrf_mlp_destroy(mrf_mlp net);
/* Host copies of the FP32 master parameters and (nullable) of the BF16
 * values the products use, widened to float.  Synchronises the device. */
mrf_status mrf_mlp_get_params(mrf_mlp net, float* params, float* params_bf16);
/* Loss L = 1/(2B) sum (y - t)^2 of B rows x: dev [B][20] against targets t:
 * dev [B][3], and its gradient with respect to the parameters as used (BF16
 * weights, FP32 biases): grad dev [137731], loss dev [1] (nullable). */
mrf_status mrf_mlp_grad(mrf_mlp net, const float* x, const float* t, int B, float* grad, float* loss,
                        mrf_stream stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on the
 * gradient of one batch; loss dev [1] nullable. */
mrf_status mrf_mlp_train_step(mrf_mlp net, const float* x, const float* t, int B, float lr, float* loss,
                              mrf_stream stream);
/* y: dev [n][3] network outputs for x: dev [n][20]. */
mrf_status mrf_mlp_infer(mrf_mlp net, const float* x, int n, float* y, mrf_stream stream);
/* Engine: tensor_cores = 1 (default) runs inference as tcgen05 BF16 products
 * with every layer's input rounded to BF16, and the training products
 * (mrf_mlp_grad, mrf_mlp_train_step) as tcgen05 split-BF16 products (hi and
 * lo parts of the FP32 operands, FP32 accumulation: FP32-accurate to ~2^-16);
 * 0 runs SIMT kernels with FP32 activations for both.  A device wait of the
 * tensor-core kernels that gives up is reported by mrf_mlp_check. */
mrf_status mrf_mlp_set_engine(mrf_mlp net, int tensor_cores);
/* MRF_ETIMEOUT if a bounded device wait of the tensor-core inference gave up
 * (synchronises `stream`). */
mrf_status mrf_mlp_check(mrf_mlp net, mrf_stream stream);
/* Training fingerprints from noiseless signals sig: dev [n][T] of the drawn
 * (T1, T2) (t1t2: dev [n][2]), PD rho: dev [n], SNR in dB snr_db: dev [n]
 * and unit-variance complex noise: dev [n][K]: alpha = rho sig Phi + sigma
 * noise with sigma^2 = ||rho sig Phi||^2 / K 10^(-snr/10); x: dev [n][2K] =
 * alpha / ||alpha|| as (Re, Im); y: dev [n][3] the encoded targets with PD
 * per unit norm rho / ||alpha||.  phi: dev [T][K]; ranges: host [5] as the
 * decode constants above. */
mrf_status mrf_mlp_training_set(const mrf_c64* sig, const float* t1t2, const float* rho,
                                const float* snr_db, const mrf_c64* noise, int n, int T,
                                const mrf_c64* phi, int K, const float* ranges, float* x, float* y,
                                mrf_stream stream);

/* ------------------------------------------------------------------------
 * Algorithm 1 (MS-LLR).  The iterate is held in the temporal subspace,
 * X = alpha Phi^H with alpha dev [ny][nx][K]; the problem is posed over
 * X in S (Eq. 11, 13), so X^0 = P_S(A^H b).  Per iteration:
 *   Z     = P_S(X - mu [A^H(A X - b) + lambda1 Q^*(Q(X) L)])        (Eq. 12)
 *   P_i   = SVT_{1/beta}(Q_i(X))                                    (Eq. 18)
 *   X     = (Z + mu lambda2 beta Q^*(P)) / (1 + mu lambda2 beta cnt)  (Eq. 19)
 *   cost  = 1/2||A X - b||^2 + lambda1 Tr(Q L Q^H) + lambda2 sum||Q_i X||_*
 *   M     = Phi_D(X);  L = D - W of the k-nearest-patch graph of M  (Eq. 7-10)
 *   lambda1 = lambda1^0 / max(L)
 * A is scaled by 1/a, a = ||A P_S|| (power iteration), and b by gamma so
 * that the largest PD matched from X^0 equals pd_target.
 * ---------------------------------------------------------------------- */
enum {
    MRF_RECON_LITERAL_XUPDATE = 1,  /* Eq. 19 as printed: divide by 1 + mu lambda2 beta */
    MRF_RECON_LITERAL_LAMBDA1 = 2,  /* lambda1 = lambda1^0 * max(L) as printed */
    MRF_RECON_NO_COST = 4,          /* skip the cost evaluation */
    MRF_RECON_GROUPED = 8,          /* data term through the grouped subspace operator */
    MRF_RECON_LEARNED = 16,         /* maps from the learned matcher (params.mlp, K = 10); fingerprints
                                       it maps outside the dictionary's T1/T2 box, or to T1 < T2, are
                                       matched exhaustively instead (needs a tensor-core precision) */
    MRF_RECON_SERIAL = 32,          /* run an iteration's steps one after another on the caller's
                                       stream (default: the forward operator, the SVT and matching +
                                       graph rebuild run concurrently on internal streams, joined into
                                       the caller's stream; same results) */
    MRF_RECON_EAGER = 64            /* launch every iteration's kernels one by one (default: from the
                                       second iteration on, one iteration is recorded once as a CUDA
                                       graph on the caller's stream and replayed; same results) */
};

typedef struct {
    float mu, lam1_0, lam2, beta;   /* step and weights; paper: 1, 0.1, 0.1, 1/5 */
    int patch, stride, knn;         /* patch side p, stride s, graph neighbours */
    int power_iters;                /* iterations of the ||A P_S|| power method */
    float pd_target;                /* PD scale of the matched initial maps (100) */
    float a_norm, x_scale;          /* > 0: use these instead of deriving a, gamma */
    int flags;                      /* MRF_RECON_* */
    int match_precision;            /* MRF_MATCH_*: the matcher (and the learned matcher's fallback) */
    mrf_mlp mlp;                    /* with MRF_RECON_LEARNED: the trained network (borrowed) */
} mrf_recon_params;

/* Create the loop state and run Algorithm 1's initialisation (X^0, M^0,
 * L^0, lambda1).  plan: a NUFFT plan whose trajectory produced b;
 * phi: dev [T][K]; dict_c: dev [m][K] compressed atoms d_m Phi;
 * atom_norm2: dev [m] ||d_m||^2 of the full atoms; lut: dev [m][2];
 * b: dev [T][ns] k-space.  The pointers must stay valid for the object's
 * lifetime (they are not copied).  Requires K <= 16, patch <= 16, knn <= 32,
 * at least knn + 1 patches.  Synchronises `stream`. */
mrf_status mrf_recon_create(mrf_recon* out, mrf_plan plan, const mrf_recon_params* params,
                            const mrf_c64* phi, int K, const mrf_c64* dict_c,
                            const float* atom_norm2, const float* lut, int m,
                            const mrf_c64* b, mrf_stream stream);
/* Run n_iters iterations.  cost_out: host double [n_iters] (nullable); when
 * given (and costs are enabled) the call synchronises to return them.
 * Unless MRF_RECON_EAGER or MRF_RECON_SERIAL is set (or the per-kernel
 * profiler is on), the first iteration after the first one is recorded as a
 * CUDA graph (stream capture of the caller's stream, which must then not be
 * capturing already) and every later iteration replays it. */
mrf_status mrf_recon_iter(mrf_recon r, int n_iters, double* cost_out, mrf_stream stream);
/* Current maps: t1, t2, pd (PD divided back by gamma): dev float [ny][nx];
 * idx: dev int [ny][nx].  Each nullable. */
mrf_status mrf_recon_maps(mrf_recon r, float* t1, float* t2, float* pd, int* idx,
                          mrf_stream stream);
/* Copy of the coefficient images alpha (dev [ny][nx][K]). */
mrf_status mrf_recon_alpha(mrf_recon r, mrf_c64* alpha, mrf_stream stream);
/* Work counters of the SVT step (Eq. 18) since mrf_recon_create: sweeps and
 * rotations = the one-sided Jacobi sweeps and column-pair rotations executed,
 * summed over patches (two patches share a warp, and a warp sweeps until
 * both are done); patch_svts = patches x SVT launches.  For measurement: the
 * SVD is iterative, so its work depends on the data.  Synchronises the
 * stream.  NULL argument: MRF_EINVAL. */
mrf_status mrf_recon_svt_stats(mrf_recon R, double* sweeps, double* rotations, double* patch_svts,
                               mrf_stream stream);

/* Scalars of the current state (host outputs, each nullable; synchronises). */
mrf_status mrf_recon_info(mrf_recon r, double* a_norm, double* x_scale, double* lam1,
                          double* sigma2, mrf_stream stream);
mrf_status mrf_recon_destroy(mrf_recon r);
/* One whole reconstruction (Algorithm 1) from host k-space to host maps:
 * copies b_host (host [T][ns] of the plan; pinned memory lets the copy run
 * asynchronously, pageable memory is staged by the runtime) to the device,
 * runs mrf_recon_create and n_iters iterations, and copies the T1, T2 and PD
 * maps (host float [ny*nx] each, nullable) back, with the same arguments and
 * errors as those calls; cost_out (host double [n_iters], nullable) receives
 * the cost per iteration.  The plan, phi, dict_c, atom_norm2 and lut stay
 * device-resident (set up once per sequence and dictionary).  Device scratch
 * for b and the maps is allocated and freed on the stream; the call
 * synchronises the stream before it returns. */
mrf_status mrf_recon_run_host(mrf_plan plan, const mrf_recon_params* params, const mrf_c64* phi,
                              int K, const mrf_c64* dict_c, const float* atom_norm2,
                              const float* lut, int m, const mrf_c64* b_host, int n_iters,
                              float* t1_host, float* t2_host, float* pd_host, double* cost_out,
                              mrf_stream stream);
/* Checkpoint / resume.  A checkpoint is a host byte buffer holding the loop
 * state the next iteration reads (coefficient images, residual, SVT output
 * and right singular vectors, maps, cost history, iteration count) and the
 * scales a and gamma.  checkpoint_size gives its length; checkpoint fills it
 * (synchronises).  restore loads it into an object created with the same
 * plan geometry, K, patch/graph parameters, dictionary and data, and with
 * params.a_norm and params.x_scale set to the saved a and gamma (from
 * mrf_recon_info of the saved object) so that the scaled data agree;
 * MRF_EINVAL otherwise.  The graph and lambda1 are rebuilt from the restored
 * maps; iterations then continue as if uninterrupted (synchronises). */
mrf_status mrf_recon_checkpoint_size(mrf_recon r, size_t* bytes);
mrf_status mrf_recon_checkpoint(mrf_recon r, void* buf, size_t bytes, mrf_stream stream);
mrf_status mrf_recon_restore(mrf_recon r, const void* buf, size_t bytes, mrf_stream stream);


/* ------------------------------------------------------------------------
 * Batched serving (not in the paper: a deployment form of Algorithm 1).
 * A batch advances count independent slices together: each slice is an
 * mrf_recon with its own NUFFT plan (sizes, frames and trajectories may
 * differ) and the same atom count m, rank K and match precision (slices with
 * different frame counts carry the dictionary compressed in their own
 * subspace).  Per iteration the slices' operator,
 * graph, X-update and SVT steps run concurrently on one stream each, the
 * matching of every slice's fingerprints is one tensor-core launch (FP32
 * precision: one launch per slice), then the slices rebuild their graphs
 * concurrently.  Costs are not computed in batch mode.
 * ---------------------------------------------------------------------- */
/* recons: host array of count handles (1 <= count <= 64), owned by the
 * caller; destroy the batch before any of them.  Synchronises `stream`. */
mrf_status mrf_batch_create(mrf_batch* out, const mrf_recon* recons, int count, mrf_stream stream);
/* n_iters iterations of every slice.  The first call runs one iteration
 * directly and captures the next into a CUDA graph (so it must not be made
 * inside a stream capture); every later iteration is one graph launch.  The
 * call synchronises `stream` and returns MRF_ETIMEOUT when a bounded device
 * wait gave up (the results are then not valid) and MRF_EINVAL when a patch
 * feature left its fixed-point range.  Maps: mrf_recon_maps per slice. */
mrf_status mrf_batch_iter(mrf_batch b, int n_iters, mrf_stream stream);
mrf_status mrf_batch_destroy(mrf_batch b);

/* Self-test of the bounded device wait used by the tensor-core kernels: one
 * thread polls an mbarrier phase that nothing completes, gives up after
 * `polls` polls (1 <= polls <= 65536) and raises the error word; the call
 * returns MRF_ETIMEOUT with a message, and the context stays usable. */
mrf_status mrf_wait_selftest(int polls, mrf_stream stream);

/* ------------------------------------------------------------------------
 * Tracing.  Not part of the method: launch accounting and per-kernel timing
 * with CUDA events on the launching stream.
 * ---------------------------------------------------------------------- */
/* Kernels launched by this library since it was loaded (all threads). */
long long mrf_launch_count(void);
/* Turn the per-kernel event profiler on (1) or off (0); either way the
 * recorded marks and totals are cleared.  While on, every launch records one
 * event after the kernel and the interval since the previous mark on the same
 * stream is charged to that kernel. */
mrf_status mrf_profile_enable(int on);
/* Boundary mark on `stream`: the next kernel's interval starts here (use it
 * before a timed region so host work or foreign kernels are not charged). */
mrf_status mrf_profile_mark(mrf_stream stream);
/* Wait for the recorded events and fold them into per-kernel totals;
 * returns the number of distinct kernel names (or -1 on a CUDA error). */
int mrf_profile_collect(void);
/* Entry i of the totals: kernel name (NUL-terminated, truncated to
 * name_len), accumulated milliseconds and number of timed launches. */
mrf_status mrf_profile_entry(int i, char* name, int name_len, double* ms, long long* launches);

#ifdef __cplusplus
}
#endif
#endif /* MRF_H */
