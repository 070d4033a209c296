/*
 * spod.h -- C ABI of libspod.so, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of spectral proper orthogonal decomposition (SPOD)
 * as stated in Rogowski et al., arXiv 2309.11808, Sec. 2.2 ("Practical
 * implementation"):
 *
 *   Welch blocks (Eq. blocks) -> time-mean subtraction -> window ->
 *   DFT of every block in time (Eq. blocks-ft, regrouped per frequency as in
 *   Eq. blocks-k) -> weighted Gram  M_f = kappa * Qhat_f^* W Qhat_f
 *   (Eq. spod-discrete-snapshots) -> Hermitian eigen-decomposition of every
 *   M_f -> modes Phi_f = Qhat_f Psi_f Lambda_f^{-1/2} / sqrt(1/kappa)
 *   (Eq. spod-discrete-snapshots; scaled so that Phi_f^* W Phi_f = I, the
 *   property stated right after that equation).
 *
 * Conventions fixed by this library where the paper is silent:
 *   - X is laid out time-major: X[t][v][p], t < nt, v < nvars, p < npoints,
 *     row-major; the flattened row index is m = v*npoints + p and
 *     M = nvars*npoints (Eq. data-matrix stores the transpose, Q in R^{M x Nt}).
 *     X is real (SPOD_F64 / F32 / BF16) or complex (SPOD_C64 / C128,
 *     interleaved real and imaginary parts).
 *   - step = nfft - noverlap; block l covers t in [l*step, l*step + nfft);
 *     nb = floor((nt - noverlap) / step) (the paper's L); tail samples belong
 *     to no block but do enter the mean.
 *   - nf = floor(nfft/2) + 1 one-sided frequencies for real data (Eq.
 *     discrete_modes); nf = nfft (two-sided) for complex data.
 *   - qhat[f][l][m] = c * sum_n w_n (X[l*step+n][m] - mu_m) exp(-2 pi i f n / nfft),
 *     c = 1 / sum_n w_n, mu_m the mean over all nt snapshots.
 *   - kappa = 1/nb (SPOD_NORM_NB) or 1/(nb-1) (SPOD_NORM_NB_MINUS_1, the
 *     factor printed in Eq. csd-discrete).
 *   - eigenvalues descending; eigenvectors unit 2-norm, largest-modulus entry
 *     (lowest index on ties) real positive.
 *   - modes with lambda_k <= 1e-12 * lambda_1 (or not positive) are returned as zero.
 *
 * Ownership: the caller owns every buffer it passes.  A plan owns its device
 * workspace and private copies of the window and weights.
 * Streams: every call that takes a `stream` (a cudaStream_t, NULL = legacy
 * default stream) is enqueued on it and returns without waiting, except the
 * *_host calls and spod_get_* with on_device = 0, which synchronise the stream.
 * Errors: every call returns a status; spod_last_error() gives a message for
 * the calling thread.  Device-side conditions (non-finite input, eigen-solver
 * not converged) are recorded in the plan and returned by the next call that
 * synchronises (spod_get_eigs, spod_sync, the *_host calls).
 * Threads: a plan may be used by one host thread at a time.
 */
#ifndef SPOD_H_
#define SPOD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spod_plan_s* spod_plan_t;

typedef enum {
  SPOD_OK = 0,
  SPOD_EINVAL = 1,          /* invalid argument or plan description */
  SPOD_ENOMEM = 2,          /* device or host allocation failed */
  SPOD_ECUDA = 3,           /* CUDA runtime error (message in spod_last_error) */
  SPOD_ESTATE = 4,          /* call order: modes / backward / get_eigs before fit */
  SPOD_ENANINPUT = 5,       /* X contained NaN or Inf */
  SPOD_ENOTCONVERGED = 6,   /* eigen-solver hit its iteration cap */
  SPOD_ETIMEOUT = 7,        /* a bounded device wait gave up */
  SPOD_EUNSUPPORTED = 8     /* valid request the library does not implement */
} spod_status;

/* Element type of X.  SPOD_C64 / SPOD_C128: complex data (interleaved real,
 * imaginary; the paper allows a complex data matrix, Eq. data-matrix): the
 * spectrum is two-sided, nf = nfft bins f = 0 .. nfft-1 (f >= ceil(nfft/2)
 * are the negative frequencies f - nfft), the time mean is complex, and
 * spod_backward returns SPOD_EUNSUPPORTED. */
typedef enum { SPOD_F64 = 0, SPOD_F32 = 1, SPOD_BF16 = 2, SPOD_C64 = 3, SPOD_C128 = 4 } spod_dtype;

/* Arithmetic of the bulk FFT / Gram / mode work.
 *   FP64   : everything in FP64 (input F64 or F32), the eigen-solve included.
 *   FP32   : FFT, Gram and modes in FP32 SIMT arithmetic; Gram partial sums
 *            promoted to FP64 every few hundred points.
 *   BF16   : FFT in FP32; Gram and mode products on the tensor cores from
 *            BF16-rounded operands, FP32 accumulation.
 *   BF16X3 : as BF16 but every operand x is split x = hi + lo (hi = bf16(x),
 *            lo = bf16(x - hi)).  Modes: hi*hi + hi*lo + lo*hi.  Gram
 *            (symmetric): A1 = hi hi^T in short tensor-core runs drained into
 *            compensated FP32 sums, A2 = hi lo^T, and the diagonal of lo lo^T:
 *            Y Y^T = A1 + A2 + A2^T + diag(lo lo^T); the off-diagonal lo lo^T
 *            terms (2^-16 of Y Y^T, uncorrelated rounding products) are left
 *            out.
 * Partial Grams are combined in FP64.  The time mean is accumulated in FP64
 * by the separate mean pass or, taken inside the FFT pass (desc.mean_in_fft,
 * BF16 / BF16X3), in compensated FP32 sums combined per point in FP64.  The
 * eigen-solve reads the FP64 Gram; for the FP64 precision it runs in FP64,
 * for the others its Householder reduction, QL rotation chain and
 * eigenvector rotations run in double-FP32 (about 48 bits) and the rest of
 * it in FP64. */
typedef enum {
  SPOD_PREC_FP64 = 0,
  SPOD_PREC_FP32 = 1,
  SPOD_PREC_BF16 = 2,
  SPOD_PREC_BF16X3 = 3
} spod_precision;

typedef enum {
  SPOD_WIN_HAMMING = 0,           /* symmetric: 0.54 - 0.46 cos(2 pi n / (N-1)) (default) */
  SPOD_WIN_HAMMING_PERIODIC = 1,  /* 0.54 - 0.46 cos(2 pi n / N) */
  SPOD_WIN_HANN = 2,              /* symmetric: 0.5 - 0.5 cos(2 pi n / (N-1)) */
  SPOD_WIN_RECT = 3,
  SPOD_WIN_USER = 4               /* user_window[nfft], copied at plan creation */
} spod_window;

typedef enum {
  SPOD_NORM_NB = 0,               /* kappa = 1/nb (default) */
  SPOD_NORM_NB_MINUS_1 = 1        /* kappa = 1/(nb-1), Eq. csd-discrete */
} spod_norm;

typedef struct {
  int ndim;                  /* 1..3: spatial grid rank */
  int64_t dims[3];           /* grid extents; npoints = prod(dims[0..ndim-1]) */
  int nvars;                 /* variables per point (M_vars); M = nvars * npoints */
  int64_t nt;                /* snapshots N_t */
  int nfft;                  /* block length N_f, 2 <= nfft <= nt, nfft = 2^a 3^b 5^c */
  int noverlap;              /* 0 <= noverlap < nfft */
  spod_window window;
  const double* user_window; /* host [nfft] when window == SPOD_WIN_USER, else ignored */
  const double* weights;     /* host [M] quadrature weights W (all > 0, finite); NULL = all ones */
  double dt;                 /* snapshot spacing, used by spod_get_freqs only (> 0) */
  spod_dtype in_dtype;       /* element type of X */
  spod_precision precision;
  spod_norm norm;
  int subtract_mean;         /* 1 (default): subtract the temporal mean; 0: use X as is */
  int64_t chunk_points;      /* spatial points per FFT->Gram pass; 0 = automatic: the whole
                                grid when its Qhat fits in the larger of 40 GiB and 35 % of
                                the device memory free at plan creation, else chunks of that
                                size.  Bounds the device workspace (Qhat of one chunk). */
  int mean_in_fft;           /* 1 (default): where the plan allows it, the time mean is taken
                                inside the pipelined FFT pass, which then reads X only once
                                (real data, BF16 / BF16X3 precision, nfft 256 / 384 / 512 /
                                720, 2 nb not a multiple of 16): each column is centred on
                                the mean c of 128 evenly spaced snapshots, the spectra of
                                x - c are stored with one more row rho = sqrt(W) (mu - c),
                                and the Gram and the modes apply the exact rank-one
                                correction Qhat_f = Z_f - rho What_f in FP64 / in the MMA.
                                0: a separate mean pass reads X first.  Read back whether
                                it applies from spod_plan_info.mean_in_fft. */
} spod_plan_desc;

typedef struct {
  int64_t M;                 /* nvars * npoints */
  int64_t nt;
  int nfft, noverlap, step;
  int nb;                    /* Welch blocks L */
  int nf;                    /* one-sided frequencies */
  int device;                /* CUDA device the plan lives on */
  size_t workspace_bytes;    /* device memory owned by the plan */
  int64_t chunk_points;      /* spatial points per FFT->Gram pass */
  int mean_in_fft;           /* 1: the time mean is folded into the FFT pass (see the desc) */
} spod_plan_info;

/* Fill *desc with defaults (Hamming, 50 % overlap unset = 0, FP32, NORM_NB,
 * subtract_mean = 1, dt = 1): the readings this library takes where Sec. 2.2
 * is silent (window, normalisation).  Never fails for a non-NULL pointer;
 * SPOD_EINVAL for NULL. */
spod_status spod_desc_init(spod_plan_desc* desc);

/* Validate desc, copy window and weights, and allocate the plan's device
 * workspace on the current CUDA device.  Derived sizes follow Eq. blocks
 * (nb = floor((nt - noverlap) / step), step = nfft - noverlap) and the
 * one-sided count after Eq. discrete_modes (nf).  Errors: SPOD_EINVAL (bad sizes,
 * non-positive or non-finite weights, unsupported nfft factorisation ->
 * SPOD_EUNSUPPORTED), SPOD_ENOMEM, SPOD_ECUDA.  *out is NULL on failure. */
spod_status spod_plan_create(const spod_plan_desc* desc, spod_plan_t* out);

/* Free the plan and its workspace (device-synchronising).  NULL is a no-op.
 * No counterpart in the paper (resource management). */
spod_status spod_plan_destroy(spod_plan_t plan);

/* The plan's derived sizes (M, nb and step of Eq. blocks, nf, chunk) and
 * workspace into *info (host).  SPOD_EINVAL for a NULL plan or info. */
spod_status spod_plan_get_info(spod_plan_t plan, spod_plan_info* info);

/* Mean, blocks, window, batched FFT, weighted Gram, deterministic reduction and
 * batched Hermitian eigen-decomposition (Sec. 2.2, Eqs. blocks to
 * spod-discrete-snapshots).  d_X: device pointer to X[nt][M] of in_dtype,
 * 16-byte aligned.  Results stay in the plan (see spod_get_eigs).  Stream-ordered. */
spod_status spod_fit(spod_plan_t plan, const void* d_X, void* stream);

/* The paper's spatial decomposition (Sec. 3.1): each process owns a slab of
 * the points, forms its part of every M_f (Eq. spod-discrete-snapshots is a
 * sum over points), one reduction sums the parts, every process solves the
 * same eigenproblems and computes the modes of its own points.  Here a slab is
 * a plan over a contiguous range of columns of X (its own npoints / weights,
 * X given as that slab's [nt][slab columns]); the exchange of the parts
 * between processes or GPUs is the caller's.
 *
 * spod_fit_partial: the fit of the plan's points up to the weighted Gram
 * (mean, blocks, window, DFT, the plan's fixed-order reduction, kappa
 * applied), without the eigen-solve.  Writes that slab Gram to d_gram (device,
 * caller-owned, [nf][nb][nb] interleaved complex FP64, 16-byte aligned) and
 * keeps the slab's Qhat for the modes.  Stream-ordered. */
spod_status spod_fit_partial(spod_plan_t plan, const void* d_X, double* d_gram, void* stream);

/* spod_fit_from_grams (the reduction and the redundant eigen-solve of Sec. 3.1):
 * the sum of nparts slab Grams d_grams[nparts][nf][nb][nb]
 * (device, interleaved complex FP64, 16-byte aligned), taken in part order --
 * so every process that passes the same gathered parts gets bit-identical
 * results -- then the eigen-solve.  Afterwards the plan behaves as after
 * spod_fit of the whole domain: spod_get_eigs gives the global eigenpairs,
 * spod_modes the modes restricted to this plan's points, spod_backward the
 * gradient with respect to this plan's columns.  SPOD_ESTATE unless
 * spod_fit_partial ran on this plan before; SPOD_EINVAL for nparts < 1.
 * Stream-ordered. */
spod_status spod_fit_from_grams(spod_plan_t plan, const double* d_grams, int nparts, void* stream);

/* Copy the eigenvalues lambda[nf][nb] of the M_f of Eq.
 * spod-discrete-snapshots (FP64, descending per frequency) and,
 * when psi != NULL, the eigenvectors psi[nf][nb (entry)][nb (vector)] as
 * interleaved complex FP64 (column k of psi[f] is the k-th eigenvector).
 * on_device = 1: both pointers are device memory, the copy is enqueued on
 * the stream of the last fit and the call does not wait.  on_device = 0: host
 * memory; the call synchronises and also reports device-side conditions
 * (SPOD_ENANINPUT, SPOD_ENOTCONVERGED).  SPOD_ESTATE before a fit. */
spod_status spod_get_eigs(spod_plan_t plan, double* lambda, double* psi, int on_device);

/* Copy the weighted Gram matrices M_f [nf][nb][nb] of Eq.
 * spod-discrete-snapshots (interleaved complex FP64, kappa applied) to host
 * memory; synchronising.  SPOD_ESTATE before a fit. */
spod_status spod_get_gram(spod_plan_t plan, double* gram);

/* Frequencies of the bins of Eq. blocks-ft, f / (nfft * dt), f = 0 .. nf-1,
 * into host memory (complex input: bins f >= ceil(nfft/2) give
 * (f - nfft) / (nfft * dt)).  SPOD_EINVAL for a NULL plan or freqs. */
spod_status spod_get_freqs(spod_plan_t plan, double* freqs);

/* SPOD modes of the last fit (Eq. spod-discrete-snapshots): recomputes Qhat
 * from d_X (which must hold the same data as the fit) and writes
 * Phi[f][k][m] = sum_l qhat[f][l][m] psi_f[l][k] / sqrt(lambda_k,f / kappa)
 * for k < nmodes (1 <= nmodes <= nb), as interleaved complex FP32 (precision
 * FP32/BF16/BF16X3) or FP64 (precision FP64).  d_Phi: device, nf*nmodes*M
 * complex elements, 16-byte aligned.  SPOD_ESTATE before a fit. */
spod_status spod_modes(spod_plan_t plan, const void* d_X, int nmodes, void* d_Phi, void* stream);

/* Adjoint of the fit for losses on eigenvalues (not in the paper: the
 * derivative of the eigenvalues of Eq. spod-discrete-snapshots with respect
 * to the data, through Eqs. blocks to blocks-k): given d_dLdlambda[nf][nb]
 * (device FP64) writes dL/dX [nt][M] (device, FP32 for precision
 * FP32/BF16/BF16X3, FP64 for FP64).  Valid for simple eigenvalues: with
 * G_f = sum_k g_fk psi psi^H and R_f = 2 kappa W Qhat_f G_f,
 * dL/dxt[l*step+n][m] += c w_n Re(sum_f R_f[m][l] e^{+2 pi i f n/nfft})
 * (overlap-add over blocks), then the mean projection.  Qhat is recomputed
 * from d_X.  SPOD_ESTATE before a fit. */
spod_status spod_backward(spod_plan_t plan, const double* d_dLdlambda, const void* d_X,
                          void* d_dX, void* stream);

/* End-to-end call on HOST buffers: copies h_X to the device, fits, computes
 * nmodes modes (0 = none) and copies eigenvalues (h_lambda[nf][nb], may be
 * NULL) and modes (h_Phi, layout as spod_modes, may be NULL when nmodes = 0)
 * back.  Device staging buffers are owned by the plan and kept for reuse.
 * The modes are computed in frequency ranges and each range is copied back
 * (Phi is frequency-major, so a range is contiguous) while the next one is
 * computed, on a plan-owned copy stream.  Pinned host memory gives the
 * fastest copies.  Synchronises the stream.  No counterpart in the paper. */
spod_status spod_run_host(spod_plan_t plan, const void* h_X, int nmodes, void* h_Phi, double* h_lambda,
                          void* stream);

/* spod_run_host (the fit and modes of Sec. 2.2; the pipelining has no
 * counterpart in the paper) over n datasets of the plan's shape (h_X[i], h_Phi[i],
 * h_lambda[i]; h_lambda may be NULL, or hold NULL entries), processed in
 * order with two staging pairs used in turn: dataset i + 1's X is copied up
 * on one copy stream while dataset i's modes are copied down on another (the
 * host link carries both directions at once).  Results equal n spod_run_host
 * calls.  SPOD_EINVAL for n < 1 or a NULL buffer; synchronises the stream. */
spod_status spod_run_host_many(spod_plan_t plan, int n, const void* const* h_X, int nmodes, void* const* h_Phi,
                               double* const* h_lambda, void* stream);

/* Wait for the plan's work on `stream` and report device-side conditions
 * (SPOD_ENANINPUT, SPOD_ENOTCONVERGED, SPOD_ETIMEOUT).  No counterpart in the
 * paper (stream-ordered execution). */
spod_status spod_sync(spod_plan_t plan, void* stream);

/* Fit n plans on n inputs with one CUDA-graph launch (datasets of different
 * grid size, nt and nfft; Sec. 4.2 analyses several reanalysis records).
 * The results equal n spod_fit calls.  The first call captures the n fits
 * into a graph with one branch per dataset (independent datasets run
 * concurrently); later calls with the same plans, inputs and launch
 * parameters relaunch the cached graph.  All plans must be on one device and
 * distinct.  Asynchronous on `stream` like spod_fit; errors of the capture
 * are returned, device-side conditions by the next spod_sync of each plan. */
spod_status spod_fit_batch(spod_plan_t* plans, const void* const* d_X, int n, void* stream);

/* Out-of-core run for data larger than device memory (no counterpart of
 * this API shape in the paper; its data-size argument is Sec. 3.2): h_X and
 * h_Phi stay in host memory the device can address -- pinned (cudaHostAlloc or
 * cudaHostRegister), or any host memory on a device that reads pageable memory
 * through the host's page tables (cudaDevAttrPageableMemoryAccess); otherwise
 * SPOD_EINVAL -- and are read and written in column tiles of tile_points points
 * (0: about M/4, rounded to 64, at most the plan's chunk) by copy kernels
 * over the host link, overlapped with the fit (mean, FFT, Gram per tile) and
 * with the modes (each tile's Qhat recomputed).  h_X is [nt][M] in the plan's
 * input type, h_Phi [nf][nmodes][M] as spod_modes writes it (may be NULL when
 * nmodes = 0), h_lambda [nf][nb] (may be NULL).  Device memory: the plan's
 * workspace plus two X tiles and two Phi tiles; give the plan chunk_points =
 * the tile width so that its Qhat is one tile.  Results equal spod_fit +
 * spod_modes bit for bit when the plan's chunk_points equals the tile width
 * (the same spatial chunks), else to rounding (the Gram is summed over other
 * chunks).  Synchronises. */
spod_status spod_run_host_ooc(spod_plan_t plan, const void* h_X, int nmodes, void* h_Phi, double* h_lambda,
                              int64_t tile_points, void* stream);

/* Expansion coefficients (Eq. coeffs; SPOD for data compression): the
 * W-weighted oblique projection of the data onto the leading nmodes_r modes
 * of the nfreq_r one-sided bins h_freqs[] (host, distinct, 0 .. nf-1) and,
 * for the bins other than DC and Nyquist, their complex conjugates (the
 * modes of the negative frequencies; the set is then closed under
 * conjugation and the reconstruction of real data is real):
 *   A = (Phi_r^* W Phi_r)^{-1} Phi_r^* W (X^T - mu).
 * d_X: the data of the last fit (device, [nt][M]); d_Phi: modes of the last
 * fit from spod_modes with nmodes columns (>= nmodes_r), [nf][nmodes][M].
 * d_A (device, caller-owned): interleaved complex FP64 [nfreq_r][nmodes_r][nt],
 * the coefficient of mode k at bin h_freqs[j] (the conjugate bin's is its
 * conjugate).  Real data with F32 input (FP32 / BF16 / BF16X3 plans) or F64
 * input (FP64 plans) only, else SPOD_EUNSUPPORTED; at most 4096 real basis
 * vectors.  A basis that is not linearly independent is reported by the
 * next spod_sync as SPOD_ENOTCONVERGED.  The two large products run on this
 * library's SIMT GEMM kernel (FP32 or FP64 as the plan) on `stream`, with
 * stream-ordered scratch (cudaMallocAsync).  No counterpart of this API shape
 * in the paper. */
spod_status spod_coeffs(spod_plan_t plan, const void* d_X, const void* d_Phi, int nmodes, int nmodes_r, int nfreq_r,
                        const int* h_freqs, double* d_A, void* stream);

/* Reconstruction (Eq. SPODrec): d_Xrec[t][m] = mu_m + (Phi_r A_r)[m][t] from the
 * coefficients of spod_coeffs (same nmodes, nmodes_r, h_freqs), in the data's
 * type (F32 or F64), [nt][M], caller-owned. */
spod_status spod_reconstruct(spod_plan_t plan, const void* d_Phi, int nmodes, int nmodes_r, int nfreq_r,
                             const int* h_freqs, const double* d_A, void* d_Xrec, void* stream);

/* Launch-shape knobs (the autotuner's interface).  They change how work is
 * split across CTAs, never what is computed beyond floating-point grouping.
 * In spod_plan_set_tuning a zero gram_splits or gram_flush_blocks keeps the
 * plan's current value; modes_ctas, eig_max_iter and wait_timeout_us are set
 * as given (0 = their default). */
typedef struct {
  int gram_splits;        /* FP32/FP64: CTAs per frequency over the points of a chunk; BF16/BF16X3:
                             persistent CTAs of the tensor-core Gram (default one per SM);
                             1..gram_splits_max */
  int gram_splits_max;    /* read-only: bound set by the plan's workspace */
  int gram_flush_blocks;  /* tensor-core Gram: 64-point blocks per accumulation run in tensor memory
                             (1..64, default 1).  The tensor core's FP32 accumulation rounds toward
                             zero, so a longer run biases the Gram by about run length x 2^-24 */
  int modes_ctas;         /* tensor-core modes: CTAs per frequency (0 = automatic) */
  int eig_max_iter;       /* eigen-solver: implicit QL iterations allowed per eigenvalue (0 = default 60;
                             1..1000).  An eigenvalue that needs more is left as it stands and the
                             next synchronising call returns SPOD_ENOTCONVERGED. */
  int wait_timeout_us;    /* bound of every device wait (a TMA copy, an MMA, a pipeline stage), in
                             microseconds (0 = default 2 s; 1..4000000).  A wait that runs out stops
                             its kernel early (copies and MMAs in flight are let land first), the
                             call's results are invalid, and the next synchronising call returns
                             SPOD_ETIMEOUT; the plan stays usable.  Setting it synchronises the device. */
  int wait_selftest;      /* 1: self-test of the bounded waits -- the tensor-core Gram (BF16 / BF16X3
                             plans) leaves its first pipeline stage unfilled, so the waits on it run
                             out after wait_timeout_us and the fit reports SPOD_ETIMEOUT; 0 (default):
                             off.  No other effect. */
  int fft_tile_points;    /* pipelined FFT (compiled nfft): spatial points per CTA tile, 16 (two CTAs
                             per SM up to nfft 512) or 32 (one CTA per SM, whole 128-byte rows); the
                             plan picks 32 where it fits in shared memory.  0 on read: the plan does
                             not use the pipelined FFT; 0 on write: leave as is.  Changes only the
                             launch shape, not the results. */
} spod_tuning;

/* The plan's launch shape into *tuning (host).  No counterpart in the paper. */
spod_status spod_plan_get_tuning(spod_plan_t plan, spod_tuning* tuning);
/* Set the launch shape and the limits (no counterpart in the paper).
 * SPOD_EINVAL for values outside the stated ranges; takes effect from the
 * next fit/modes call. */
spod_status spod_plan_set_tuning(spod_plan_t plan, const spod_tuning* tuning);

/* Autotuner: runs spod_fit on d_X (device, as spod_fit) under candidate
 * launch shapes (the pipelined FFT's tile width, 16 or 32 points, where both
 * have a compiled form that fits; then the Gram's CTA split: persistent CTAs
 * per GPU for the tensor-core path, CTAs per frequency for the SIMT path),
 * times each with CUDA events on `stream` and keeps the fastest; gram_flush_blocks, which
 * changes rounding, is not searched.  Synchronises the stream; the plan holds
 * the last fit's results afterwards.  chosen (may be NULL) receives the
 * tuning kept.  No counterpart in the paper (an engineering aid). */
spod_status spod_plan_autotune(spod_plan_t plan, const void* d_X, void* stream, spod_tuning* chosen);

/* Phases of the hot path, for per-phase timing. */
typedef enum {
  SPOD_PHASE_MEAN = 0,     /* time mean */
  SPOD_PHASE_FFT = 1,      /* blocks, window, batched DFT */
  SPOD_PHASE_GRAM = 2,     /* weighted Gram partial sums */
  SPOD_PHASE_REDUCE = 3,   /* fixed-order reduction of the partial Grams */
  SPOD_PHASE_EIG = 4,      /* batched Hermitian eigen-decomposition */
  SPOD_PHASE_MODES = 5,    /* mode coefficients and mode reconstruction */
  SPOD_PHASE_BACKWARD = 6, /* adjoint kernels */
  SPOD_NPHASES = 7
} spod_phase;

/* Per-phase timing (the paper reports per-phase wall times, Sec. 5.1): when
 * enabled, every phase a call enqueues is bracketed by CUDA events recorded on
 * that call's stream.  spod_profile_read synchronises on the recorded events,
 * writes the summed milliseconds (ms[SPOD_NPHASES], may be NULL) and the number
 * of kernels launched (launches[SPOD_NPHASES], may be NULL, counted whether or
 * not timing is enabled) since the previous read, and resets both. */
spod_status spod_profile_enable(spod_plan_t plan, int enable);
spod_status spod_profile_read(spod_plan_t plan, double* ms, int64_t* launches);

/* Allocation-free batched Hermitian eigen-decomposition of caller-provided
 * matrices.  The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc -- code running under a host framework that owns
 * all device memory, real-time loops that cannot take the allocator's latency
 * or the device-wide synchronisation of cudaFree, programs that reserve all
 * their memory up front.  It runs a cyclic complex Jacobi solver (one CTA per
 * matrix; spod_fit uses Householder + implicit QL instead) with the same
 * conventions as spod_get_eigs, so the results agree with a fit's to
 * rounding; its cost grows as nb^3 per sweep on the FP64 pipe.
 *   d_gram   : device, [nf][nb][nb] interleaved complex FP64 Hermitian
 *              matrices (16-byte aligned), read only.
 *   d_lambda : device, [nf][nb] FP64 eigenvalues, descending (8-byte aligned).
 *   d_psi    : device, [nf][nb][nb] interleaved complex FP64, column k of
 *              psi[f] the k-th eigenvector, unit norm, largest-modulus entry
 *              real positive (16-byte aligned).
 * Scratch comes from one fixed 32 MiB device array inside the library (held
 * by every GPU that loads it until the process exits): the call needs
 * 256 + (nb > 48 ? nf * 32 * nb * nb : 0) bytes of it, so nb <= 1023 at
 * nf = 1, and returns SPOD_EINVAL when that exceeds 32 MiB, or when nf < 1
 * or nb is outside 1..1024.  No device memory is allocated.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress) and
 * keeps it for that device; do not use this entry across a cudaDeviceReset
 * (the kept address would be stale).  The call enqueues the solver on `stream` on the
 * current device, then waits for that stream and returns SPOD_ENOTCONVERGED
 * if the solver hit its sweep cap.  All calls share the one array: calls that
 * overlap on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller. */
spod_status spod_eigh_batched_noalloc(const double* d_gram, int nf, int nb, double* d_lambda, double* d_psi,
                                      void* stream);

/* Thread-local message describing the last non-OK status (no counterpart in
 * the paper).  Never NULL. */
const char* spod_last_error(void);

/* Library version string (no counterpart in the paper).  Never NULL. */
const char* spod_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPOD_H_ */
