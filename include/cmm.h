/*
 * cmm.h -- C ABI of the GB300 map-maker: maximum-likelihood CMB map-making by
 * preconditioned conjugate gradients with the binned, Jacobi and circulant
 * ("constant correlation") preconditioners of Naess & Louis, "A fast map-making
 * preconditioner for regular scanning patterns" (arXiv:1309.7473).
 *
 * Conventions for every call
 * --------------------------
 * - Every call returns an int status: CMM_OK (0) or one of CMM_ERR_*; the text of
 *   the last error of the calling thread is returned by cmm_last_error().
 * - Handles (cmm_ctx, cmm_pointing, cmm_noise, cmm_op, cmm_precon) are created and
 *   freed by the library; each *_destroy frees the device memory the handle owns.
 *   A handle keeps the handles it was made from alive (an operator its context,
 *   pointing and noise; a preconditioner its operator and correction network), so
 *   handles may be destroyed in any order: memory is released when the last
 *   handle that needs it is destroyed.  Destroying a handle twice is an error the
 *   library cannot detect.
 * - "host" arguments are ordinary host memory that the call reads (or writes)
 *   before it returns.  "device" arguments are caller-owned device memory on the
 *   context's device, at least 16-byte aligned; the library never frees them.
 * - Maps are FP64 device arrays laid out [ncomp][ny][nx] (Stokes-major, x fastest),
 *   ncomp = 1 (T) or 3 (T, Q, U).  Pixel (iy, ix) is centred at map coordinate
 *   (x, y) = (ix, iy) in pixel units.
 * - All device work is issued on the stream given to cmm_ctx_create, in order;
 *   calls return without waiting unless stated (cmm_solve waits; *_host calls wait).
 * - Calls on one handle are not thread-safe; different contexts may be used from
 *   different threads.
 */
#ifndef CMM_H
#define CMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum cmm_status {
  CMM_OK = 0,
  CMM_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, bad enum) */
  CMM_ERR_CUDA = 2,           /* a CUDA runtime call or kernel launch failed */
  CMM_ERR_OOM = 3,            /* device allocation failed */
  CMM_ERR_BREAKDOWN = 4,      /* PCG breakdown: p^T A p <= 0, r^T z <= 0 or a non-finite scalar */
  CMM_ERR_NOT_CONVERGED = 5,  /* maxit reached before the tolerance */
  CMM_ERR_TIMEOUT = 6,        /* a bounded device wait ran out */
  CMM_ERR_UNSUPPORTED = 7     /* size or mode not implemented (e.g. n_samp not a power of two) */
};

/* Arithmetic of the operator A = P^T N^-1 P.
 * F64: everything in FP64 (parity mode).
 * F32: time-ordered data, FFTs, noise filter and projection in FP32; map accumulator,
 *      CG vectors and scalars in FP64.
 * BF16: as F32, but the intermediate half-spectra are stored in BF16 between passes. */
enum cmm_precision { CMM_PREC_F64 = 0, CMM_PREC_F32 = 1, CMM_PREC_BF16 = 2 };

enum cmm_precon_kind {
  CMM_PRECON_BINNED = 0,    /* M_B, Eq. 3-4: per-pixel inverse of P^T diag(N^-1) P */
  CMM_PRECON_JACOBI = 1,    /* M_J, Eq. 5: per-pixel inverse of P^T P */
  CMM_PRECON_CIRCULANT = 2, /* M_C, Eq. 7-13 with the Gaussian regularisation */
  CMM_PRECON_IDENTITY = 3,  /* M = I (plain CG) */
  CMM_PRECON_CIRC_LEARNED = 4, /* M_C followed by a learned correction (flexible CG) */
  CMM_PRECON_CIRC_TILED = 5    /* locally varying M_C: per-tile circulants merged by a partition of unity */
};

typedef struct cmm_ctx cmm_ctx;
typedef struct cmm_pointing cmm_pointing;
typedef struct cmm_noise cmm_noise;
typedef struct cmm_op cmm_op;
typedef struct cmm_precon cmm_precon;
typedef struct cmm_unet cmm_unet;

/* Map geometry: ny rows of nx pixels, ncomp Stokes components (1 or 3);
 * periodic != 0 wraps pixel indices instead of cutting samples that fall off
 * the map. */
typedef struct {
  int32_t ny, nx, ncomp, periodic;
} cmm_map_geom;

typedef struct {
  double taper_sigma_px; /* Gaussian regularisation width in pixels (Sec. Regularization); <= 0 or inf: off */
  int64_t ref_pixel;     /* linear index of the reference pixel (Sec. Implementation); -1: nearest the centre */
  double pd_eps;         /* eigenvalue floor relative to the largest mode eigenvalue; <= 0: 1e-6 */
  int32_t tiles_y, tiles_x; /* CMM_PRECON_CIRC_TILED: tile grid (<= 0: 2 x 2).  Each tile has the
                               circulant measured at the unmasked pixel nearest its centre;
                               M = sum_t D_t M_t D_t, D_t = diag(sqrt(phi_t)), phi_t(y, x) =
                               w_i(y) w_j(x) with raised-cosine windows w_i (centres
                               (i + 1/2) n / t, half-width n / t, the outer ones held at 1
                               towards the edges) summing to 1 (Summary section's variant) */
  int32_t white_diag;    /* != 0: the detector weights diag(N^-1)_d of Eq. 3 and Eq. 7 are the
                            white level 1 / sigma_d^2 of the noise law instead of the exact
                            diagonal of the Fourier-diagonal N_d^-1 (the mean of w_d(f) over
                            the DFT grid); BINNED, CIRCULANT and CIRC_TILED */
} cmm_precon_opts;

typedef struct {
  double tol;          /* stop when ||r_k|| / ||b|| <= tol */
  int32_t maxit;       /* iteration limit */
  int32_t check_every; /* iterations per captured graph launch between host checks (>= 1) */
  int32_t use_graph;   /* != 0: replay the iteration as a CUDA graph */
  int32_t x0_given;    /* != 0: x holds the starting guess; else x0 = 0 */
  int32_t cg_f32;      /* != 0: CG vectors, dot products and scalars rounded to FP32 */
  int32_t resid_replace; /* > 0: every that many iterations r = b - A x is recomputed */
  int32_t flexible;    /* != 0: flexible CG, beta = z^T (r - r_old) / (z_old^T r_old) */
  int32_t snapshot_every; /* with a snapshot buffer: keep (x_k, r_k) every that many iterations */
  int32_t snapshot_max;   /* number of snapshot slots */
  int32_t batch_width;    /* cmm_batch_solve: concurrent lanes (<= 0: automatic) */
  int32_t skip_true_resid; /* != 0: no exit check of ||b - A x|| (true_rel_resid = -1) */
  int32_t resume;      /* != 0: continue from the state of cmm_solve_state_load; x holds that
                          state's iterate x_k, the count goes on from k (maxit counts from 0) */
  int32_t fcg_window;  /* flexible CG only: m = 2..8 keeps the last m directions and makes each
                          new one A-conjugate to them, p = z - sum_j (z^T A p_j / p_j^T A p_j) p_j,
                          step alpha = p^T r / p^T A p (truncated flexible CG, Notay 2000); 0 or 1:
                          the Polak-Ribiere form above.  Not with resume or resid_replace. */
} cmm_solve_opts;

typedef struct {
  int32_t iterations;   /* A-applications inside the loop */
  int32_t status;       /* CMM_OK, CMM_ERR_NOT_CONVERGED or CMM_ERR_BREAKDOWN (p^T A p <= 0,
                           r^T z <= 0, or a non-finite value in b, x0 or a CG scalar) */
  double rel_resid;     /* last recursive ||r|| / ||b|| (-1 when b is not finite) */
  double seconds;       /* wall time of the call */
  double true_rel_resid; /* ||b - A x|| / ||b|| recomputed from the returned x at exit
                            (one more A-application, inside `seconds`); -1 when
                            opts->skip_true_resid */
} cmm_solve_info;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, issuing all work on `stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
int cmm_ctx_create(int device, void* stream, cmm_ctx** out);
int cmm_ctx_destroy(cmm_ctx* ctx);
/* Text of the calling thread's last error ("" if none).  Valid until the next call. */
const char* cmm_last_error(void);
/* Version string of the library. */
const char* cmm_version(void);

/* ---------------------------------------------------------------- pointing
 * The pointing matrix P of Eq. 1, never stored: each sample's pixel and response
 * are computed on the fly from a boresight table and a detector table.
 *   bore    host int32 [n_samp][4]: (bx, by) boresight in units of 2^-16 pixel,
 *           |bx|, |by| <= 2^30 - 2^25; (cphi, sphi) = (cos, sin) of the sky rotation
 *           in units of 2^-15, |cphi|, |sphi| <= 2^15.
 *   det_off host int32 [n_det][2]: (dx, dy) detector offset in units of 2^-7 pixel,
 *           |dx|, |dy| < 2^14.
 *   det_pol host double [n_det][2]: (cos 2psi, sin 2psi) of the detector angle psi.
 * Sample (d, t) has the rotated offset ox = cphi*dx - sphi*dy, oy = sphi*dx + cphi*dy
 * (exact int32, units of 2^-22 pixel), lies at x = bx + (ox >> 6), y = by + (oy >> 6)
 * (units of 2^-16 pixel, arithmetic shifts) and hits pixel ix = (x + 2^15) >> 16, iy
 * likewise (nearest pixel, halves rounded up).  Its row of P is (1) for T maps and
 * (1, cos 2a, sin 2a), a = psi + phi, for TQU maps (Sec. Test setup).  Samples off
 * the map (unless periodic) and samples of masked pixels have a zero row.  A pixel is
 * masked when its unit-weight hit block sum_t P_t P_t^T has no hits or reciprocal
 * condition number below 1e-3.  The tables are copied.  Limits: ny * nx <= 2^28
 * pixels (the kernels index the 4-wide per-pixel accumulators in 32 bits),
 * 1 <= n_det <= 65535; otherwise CMM_ERR_ARG.
 */
int cmm_pointing_create(cmm_ctx* ctx, const cmm_map_geom* geom, int32_t n_det,
                        const int32_t* det_off, const double* det_pol, int64_t n_samp,
                        const int32_t* bore, cmm_pointing** out);
int cmm_pointing_destroy(cmm_pointing* pt);
/* Copy the pixel mask (host uint8 [ny*nx], 1 = solved for) and return the number
 * of unmasked pixels in *n_good (may be NULL). */
int cmm_pointing_mask(cmm_pointing* pt, uint8_t* mask_host, int64_t* n_good);

/* ---------------------------------------------------------------- noise
 * Stationary per-detector noise (Eq. 1: n gaussian with covariance N), applied as
 * the Fourier-diagonal filter N_d^-1 = F^-1 diag(w_d) F over the n_samp samples of
 * each detector, w_d(f) = 1 / (sigma_d^2 (1 + (f / fknee_d)^-alpha_d)),
 * f_k = k f_samp / n_samp; fknee_d = 0 means white noise; the k = 0 bin takes the
 * k = 1 value.  sigma, fknee, alpha: host double [n_det].
 */
int cmm_noise_create(cmm_ctx* ctx, int32_t n_det, int64_t n_samp, double f_samp,
                     const double* sigma, const double* fknee, const double* alpha,
                     cmm_noise** out);
int cmm_noise_destroy(cmm_noise* nz);
/* Tabulated noise weights instead of the law: w_host (host double
 * [n_det][n_samp/2 + 1]) holds w_d(f_k) = 1 / PSD_d(f_k) for k = 0 .. n_samp/2, e.g.
 * measured noise spectra (finite, >= 0).  diag(N^-1) (Eq. 3, 7) is recomputed from
 * the table; operators made from this noise use it at their next application
 * (4 more bytes per bin per detector read by the filter pass).  NULL restores the
 * law.  Waits for the context's stream. */
int cmm_noise_set_table(cmm_noise* nz, const double* w_host);
/* Noise correlated between detectors (an extension: the paper's test noise model
 * had inter-detector correlations without stating them).  Per frequency bin the
 * detectors' covariance becomes N(f) = D(f) + V E(f) V^T: D the per-detector law
 * above, V [n_det][r] mode templates (host, row-major; e.g. the common mode and
 * focal-plane gradients), E = diag(amp_j^2 (1 + (f / fknee_j)^-alpha_j)), DC at the
 * first bin.  N^-1 is applied bin by bin through the Woodbury identity: the filter
 * pass is split around one cross-detector solve of r x r systems per bin.
 * r = 0 removes the correlation; r <= 4.  Operators made from this noise pick the
 * model up at their next call; it needs the FP32/BF16 operator at a fast-path
 * size with every detector in one chunk (else those calls return
 * CMM_ERR_UNSUPPORTED), and the preconditioners keep the independent-noise
 * diagonal.  Waits for the context's stream. */
int cmm_noise_set_correlated(cmm_noise* nz, int32_t r, const double* modes, const double* amp,
                             const double* fknee, const double* alpha);
/* diag(N_d^-1) = mean of w_d over the two-sided DFT grid (host double [n_det]). */
int cmm_noise_diag(cmm_noise* nz, double* diag_host);

/* ---------------------------------------------------------------- operator
 * A = P^T N^-1 P (Eq. 2) in the given precision.  n_samp must be a power of two,
 * 32 <= n_samp <= 2^22.  det_chunk > 0 bounds how many detectors share one pass
 * through the intermediate spectrum buffer (<= 0: automatic).  The handle owns
 * that buffer (n_chunk, rounded up to even, * n_samp * 4 bytes in F32, 8 in F64,
 * 2 in BF16) and a few map-sized buffers.
 */
int cmm_op_create(cmm_ctx* ctx, cmm_pointing* pt, cmm_noise* nz, int32_t precision,
                  int32_t det_chunk, cmm_op** out);
int cmm_op_destroy(cmm_op* op);
/* Pointing cache (no counterpart in the paper, which recomputes nothing on a GPU):
 * enable != 0 stores the pixel index of every sample, computed once by the same
 * rule as the on-the-fly pointing, in a device array owned by the handle
 * (4 bytes x n_det x n_samp; 4.3 GB at 1024 x 2^20).  The FP32/BF16 applications
 * of A then read one index per sample instead of recomputing the pointing: more
 * HBM traffic (8 bytes per sample per application) for fewer instructions.
 * enable == 0 frees it.  Results are identical either way.  Only for the FP32 and
 * BF16 operators of non-periodic maps (else CMM_ERR_UNSUPPORTED). */
int cmm_op_set_pixel_cache(cmm_op* op, int32_t enable);
/* Two-detector FFT packing of the FP32/BF16 A-application (enable != 0, the
 * default): for 2^13 <= n_samp <= 2^20 and detectors with independent noise, the
 * noise filter of Sec. Test setup is applied to two detectors at once as one
 * complex sequence z = s_1 + i s_2 of n_samp points, so that every complex element
 * is one time sample of both and the pointing tables are read once for the two;
 * each bin pair (k, n - k) is filtered as Y(k) = a Z(k) + b conj Z(n - k) with
 * a, b = (w_1 +- w_2) / 2.  enable == 0 selects the one-detector packing (even
 * and odd samples as one complex sequence of n_samp / 2 points), which also serves
 * correlated noise, the right-hand side and operators above the FP32 hit limit.
 * Results agree to the rounding of the spectrum storage (FP32 or BF16) either way;
 * waits for the operator's stream. */
int cmm_op_set_pair_packing(cmm_op* op, int32_t enable);
/* m_out = A m_in (Eq. 2).  device double [ncomp][ny][nx] each; must not alias. */
int cmm_apply_A(cmm_op* op, const double* m_in, double* m_out);
/* Same with host buffers: copies m_in to the device, applies A, copies the result
 * back and waits. */
int cmm_apply_A_host(cmm_op* op, const double* m_in_host, double* m_out_host);
/* m_out = A m_in exactly as cmm_apply_A, but with no allocation: the paper has no
 * counterpart; this is a library service for callers that cannot have device
 * memory allocated or freed around the call (cudaMalloc/cudaFree may block on
 * other streams and fail when memory is short).  The call makes no cudaMalloc,
 * cudaFree or other allocating call; its temporaries live in one static device
 * array of 32 MiB per device, held by every GPU that loads the library until the
 * process exits.
 * - Size limit: the map buffers (npix x (8 B FP64 + 4 B FP32 accumulator) x 4 for
 *   TQU, x 1 for T, plus the gather copy) and the spectrum of at least one
 *   detector (n_samp x 4 B in F32) must fit in 32 MiB; larger operators get
 *   CMM_ERR_UNSUPPORTED.  Detectors are processed in chunks that fit.
 * - Set-up: the first call on each device looks up the array's device address
 *   (with that device current) and caches it; make that first call before any
 *   stream capture.
 * - Sharing: all calls in the process use the same array, which keeps the last
 *   call's contents (each call clears what must start at zero).  Calls that
 *   overlap on one device (from several threads, or on streams of different
 *   contexts) race on it and give wrong results; order them.
 * m_in, m_out: device double [ncomp][ny][nx]; must not alias. */
int cmm_apply_A_noalloc(cmm_op* op, const double* m_in, double* m_out);
/* Profiling: runs `reps` applications of A (as cmm_apply_A) with CUDA events
 * between its kernels and waits.  ms_host (host double [5]) receives the mean
 * duration in milliseconds of one launch of the forward pass (pointing, gather,
 * first FFT pass), of the filter pass, of the inverse pass with binning (per
 * detector chunk), of the map-side copies per application, and of one whole
 * application. */
int cmm_profile_apply(cmm_op* op, const double* m_in, double* m_out, int32_t reps, double* ms_host);
/* tod = P m (Eq. 1): device double [ncomp][ny][nx] -> device float [n_det][n_samp]
 * (tod_is_f64 = 0) or double (tod_is_f64 != 0). */
int cmm_project(cmm_op* op, const double* m, void* tod, int32_t tod_is_f64);
/* b = P^T N^-1 d (right-hand side of Eq. 2): device float or double [n_det][n_samp]
 * -> device double [ncomp][ny][nx]. */
int cmm_rhs(cmm_op* op, const void* tod, int32_t tod_is_f64, double* b);
/* *result_host = x^T y over n FP64 device elements (a deterministic tree sum);
 * waits for the result. */
int cmm_dot(cmm_op* op, const double* x, const double* y, int64_t n, double* result_host);

/* ---------------------------------------------------------------- preconditioners
 * BINNED (Eq. 3-4): blocks B_p = sum_t diag(N^-1)_d P_t P_t^T, M_B = B_p^-1 per pixel.
 * JACOBI (Eq. 5): the same with unit weights.
 * CIRCULANT (Eq. 7-13): Sigma = B_p^(1/2) (symmetric), rows A e_{ref,gamma} (Eq. 6),
 *   Q row (Eq. 13), made symmetric (q_k + q_{-k}^T)/2, multiplied by the Gaussian
 *   exp(-|k|^2 / (2 s^2)) over wrapped offsets (Sec. Regularization), H_f = (Fq)*_f
 *   (Eq. 11) inverted per Fourier mode with eigenvalues floored at pd_eps * max;
 *   applied as z = Sigma^-1 F^-1 H^-1 F Sigma^-1 r (Eq. 12).
 * opts may be NULL (taper off, centre reference pixel, pd_eps 1e-6).  The circulant
 * build runs ncomp applications of A, all in FP64; FP32/BF16 operators apply FP32
 * copies of Sigma^-1 and H^-1 with FP32 map FFTs.  The map sides must factor into
 * 2, 3 and 5 and be below 65536 pixels (else CMM_ERR_UNSUPPORTED).
 */
int cmm_precon_create(cmm_op* op, int32_t kind, const cmm_precon_opts* opts, cmm_precon** out);
int cmm_precon_destroy(cmm_precon* pc);
/* z = M r: device double [ncomp][ny][nx] each. */
int cmm_precon_apply(cmm_precon* pc, const double* r, double* z);
/* Attach (net != NULL) or detach the learned correction of a circulant
 * preconditioner: z = M_C r is followed by z <- mask (z + ||z|| U(z / ||z||)) with
 * the U-Net `net` (same context and map shape, TQU), and the kind becomes
 * CIRC_LEARNED (solved with flexible CG).  The paper has no learned component. */
int cmm_precon_set_correction(cmm_precon* pc, cmm_unet* net);
/* Training pairs for the learned correction from `count` snapshots (x_k, r_k) of a
 * solve (layout of cmm_solve's snapshot buffer) and its converged solution x_star:
 * with z = M r_k (this preconditioner), inputs[k] = z / ||z|| and targets[k] =
 * (x_star - x_k - z) / ||z|| (device FP32 [count][ncomp][ny][nx]).  Since
 * A (x_star - x_k) = r_k, the target is what the correction should add. */
int cmm_harvest_pairs(cmm_precon* pc, const double* snapshots, int32_t count, const double* x_star,
                      float* inputs, float* targets);
/* Number of Fourier modes whose eigenvalues were floored (circulant), else 0. */
int cmm_precon_clamped(cmm_precon* pc, int64_t* n_clamped);

/* ---------------------------------------------------------------- solver
 * Preconditioned conjugate gradients on A x = b (Eq. 2, with M ~ A^-1 as in the
 * Introduction's footnote).  b, x: device double [ncomp][ny][nx]; x receives the
 * solution (and holds x0 if opts->x0_given).  resid_hist (device double
 * [maxit + 1], may be NULL) receives ||r_k|| / ||b||; anorm_terms (device double
 * [maxit], may be NULL) receives alpha_k r_k^T z_k, whose sums over the next d
 * steps estimate the squared error A-norm (Results footnote).  snapshots (device
 * double [snapshot_max][2][ncomp*ny*nx], may be NULL) receives (x_k, r_k) at
 * k = 0, snapshot_every, 2 snapshot_every, ... (the paper writes intermediate maps
 * every 5 steps, Sec. Test setup).  Waits for the result; info->status reports
 * convergence.  A CIRC_LEARNED preconditioner always runs flexible CG.
 */
int cmm_solve(cmm_op* op, cmm_precon* pc, const double* b, double* x,
              const cmm_solve_opts* opts, double* resid_hist, double* anorm_terms,
              double* snapshots, cmm_solve_info* info);

/* cmm_solve from host memory: b_host (and x_host when opts->x0_given or
 * opts->resume) are copied to device buffers of the operator (allocated on the
 * first call), the solve runs as cmm_solve without history or snapshots, and the
 * solution is copied back to x_host; waits.  b_host, x_host: host double
 * [ncomp][ny][nx] (pinned memory makes the copies asynchronous). */
int cmm_solve_host(cmm_op* op, cmm_precon* pc, const double* b_host, double* x_host,
                   const cmm_solve_opts* opts, cmm_solve_info* info);

/* Checkpoint and resume of a solve.  The paper writes intermediate maps every 5
 * steps (Sec. Test setup); a checkpoint here keeps the whole PCG state, so that a
 * solve stopped after k iterations (maxit reached) and resumed continues the same
 * iterates as one that was never stopped (FP64 mode: equal to the rounding of the
 * operator's atomic sums).  The caller keeps x_k (the stopped solve's x).
 * state: device double [*n_doubles] = (r_k, p_{k-1}, r_{k-1}) of ncomp*ny*nx each,
 * then rho_{k-1}, k, ||r_k|| / ||b||, the FP32-CG flag and a format tag; it may go
 * through host memory and another process.  cmm_solve_state_save copies the state
 * of this operator's last cmm_solve (CMM_ERR_ARG if there is none or it broke
 * down) and waits; cmm_solve_state_load makes it the state that the next
 * cmm_solve with opts->resume continues (CMM_ERR_ARG if the buffer is not a saved
 * state), and waits.  Resume with the same b, preconditioner and CG mode. */
int cmm_solve_state_size(cmm_op* op, int64_t* n_doubles);
int cmm_solve_state_save(cmm_op* op, double* state);
int cmm_solve_state_load(cmm_op* op, const double* state);

/* ---------------------------------------------------------------- learned correction
 * A U-Net (no counterpart in the paper) that refines the circulant preconditioner
 * inside flexible CG.  widths[levels] (levels 1..4): encoder level l has two 3x3
 * convolutions with ReLU to widths[l] channels and 2x2 average pooling between
 * levels; decoder level l has a 2x2 stride-2 transposed convolution, the
 * concatenation [up, skip] and two 3x3 convolutions with ReLU; a 1x1 convolution
 * maps widths[0] to 3 channels.  Weights and activations are BF16, accumulation,
 * biases and gradients FP32.  Parameters are one flat FP32 vector, per layer
 * weights then biases, conv weights [cout][cin][k][k], transposed [cin][cout][2][2].
 * Maps are FP32 device arrays [batch][3][ny][nx], nx <= 64, ny and nx divisible by
 * 2^(levels-1).  Training minimises 0.5 mean((U(in) - target)^2) with Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).
 */
int cmm_unet_create(cmm_ctx* ctx, int32_t ny, int32_t nx, int32_t levels, const int32_t* widths,
                    int32_t batch_max, cmm_unet** out);
int cmm_unet_destroy(cmm_unet* net);
/* The 3x3 convolutions (forward, input gradient, weight gradient) run as implicit
 * GEMMs on the tensor cores (BF16 mma.sync, FP32 accumulation; the default,
 * enable != 0) or on the FP32 CUDA cores (enable == 0, kept as a timed
 * comparison).  On the tensor cores the FP32 gradients entering the input- and
 * weight-gradient convolutions are rounded to BF16. */
int cmm_unet_set_tensor_cores(cmm_unet* net, int32_t enable);
int cmm_unet_param_count(cmm_unet* net, int64_t* n);
/* Copies FP32 parameters (device) in, refreshes the BF16 copy, resets Adam. */
int cmm_unet_set_params(cmm_unet* net, const float* params);
int cmm_unet_get_params(cmm_unet* net, float* params);
/* Seeded He-normal initialisation (std sqrt(2 / fan_in), fan_in = c_in x kernel
 * taps; zero biases; the output layer scaled by 1e-2 so that an untrained
 * correction starts near zero); resets Adam.  Draws on the host (64-bit Mersenne
 * twister), uploads, and waits. */
int cmm_unet_init(cmm_unet* net, uint64_t seed);
/* out = U(in): device FP32 [batch][3][ny][nx] each, 1 <= batch <= batch_max (else
 * CMM_ERR_ARG).  in is rounded to the BF16 activations first, so in and out may be
 * the same buffer. */
int cmm_unet_forward(cmm_unet* net, int32_t batch, const float* in, float* out);
/* Loss and its gradient w.r.t. the parameters (grad: device FP32 [n], may be NULL);
 * *loss_host (may be NULL) receives the loss and makes the call wait. */
int cmm_unet_loss_grad(cmm_unet* net, int32_t batch, const float* in, const float* target, float* grad,
                       double* loss_host);
/* One Adam step with learning rate lr on the batch. */
int cmm_unet_train_step(cmm_unet* net, int32_t batch, const float* in, const float* target, float lr,
                        double* loss_host);

/* ---------------------------------------------------------------- diagnostics
 * Flat-sky binned power spectra of TQU maps (the convergence diagnostic of the
 * Results section: spectra of PCG iterates against the input map's, in units of
 * cosmic variance).  maps: device double [nmaps][3][ny][nx] (2, 3, 5-smooth sides),
 * square pixels of pix_rad radians.  Modes l = 2 pi (ky / (ny pix), kx / (nx pix))
 * (signed frequencies); E = Q cos 2phi + U sin 2phi, B = -Q sin 2phi + U cos 2phi,
 * phi = atan2(ly, lx); C_b = pix^2 / (ny nx) times the mean of |X|^2 over the modes
 * with lmax b / nbins <= |l| < lmax (b + 1) / nbins (l = 0 excluded).
 * cls_host: host double [nmaps][3][nbins] (TT, EE, BB); nmodes_host (may be NULL):
 * host int64 [nbins] modes per bin.  nbins <= 1024.  Allocates work buffers;
 * waits for the result. */
int cmm_spectra(cmm_ctx* ctx, int32_t ny, int32_t nx, double pix_rad, int32_t nmaps, const double* maps,
                int32_t nbins, double lmax, double* cls_host, int64_t* nmodes_host);
/* When each spectrum bin of a sequence of PCG iterates has converged (Results
 * section: the step after which the iterate's spectrum stays within `level`
 * (the paper uses 0.1) times cosmic variance of the input map's).  Host-only
 * arithmetic, no device call.  iters: host int32 [n_snap], the iteration of each
 * snapshot; cls_iter: host double [n_snap][nspec][nbins] (cmm_spectra of the
 * snapshots); cls_true: host double [nspec][nbins], the input map's spectra;
 * nmodes: host int64 [nbins] modes per bin.  sigma_b = cls_true * sqrt(2 /
 * max(nmodes_b, 1)); out: host int32 [nspec][nbins] receives iters[k + 1] for the
 * last snapshot k with |cls_iter - cls_true| >= level sigma_b (iters[0] when there
 * is none, -1 when it is the last snapshot).  A bin whose cls_true is 0 has no
 * scale and reads as converged at iters[0].  CMM_ERR_ARG on a NULL pointer, a
 * non-positive count or level <= 0. */
int cmm_spectra_converged_at(int32_t n_snap, const int32_t* iters, int32_t nspec, int32_t nbins,
                             const double* cls_iter, const double* cls_true, const int64_t* nmodes, double level,
                             int32_t* out);

/* ---------------------------------------------------------------- batches and tuning
 * Batched solves (many Monte-Carlo realisations or patches of uneven size): n
 * independent PCG solves, one per (ops[i], pcs[i], b[i], x[i]), are advanced
 * together; every `check_every` iterations of the whole batch are one CUDA graph
 * launch.  Inside it the solves run in opts->batch_width parallel lanes (solves
 * assigned largest first to the least loaded lane, one after another within a
 * lane), each solve on the stream of its own context (give each operator its own
 * context for the lanes to overlap).  Automatic width: 1 when the solves average
 * 10^8 samples or more (each alone fills the GPU, and concurrent ones only share
 * the L2 their maps live in), else up to 8.  A solve that has converged keeps
 * returning early inside the graph.  opts as in
 * cmm_solve (resid_replace must be 0); infos[i] receives each solve's result, its
 * `seconds` the wall time of the whole batch.  Waits for the result.
 */
int cmm_batch_solve(int32_t n, cmm_op* const* ops, cmm_precon* const* pcs, const double* const* b,
                    double* const* x, const cmm_solve_opts* opts, cmm_solve_info* infos);
/* Chooses how the time-ordered FFTs of this operator run, by timing `reps`
 * applications of A for every candidate: the two-detector packing (where it
 * applies; its split of n_samp is fixed) and every split N = R C of the
 * one-detector packing that the kernels support.  Keeps the fastest and remembers
 * it for operators of the same (n_samp, n_det, precision, ncomp) in this process
 * and, if cache_path is not NULL, in that text file (read first, appended to; the
 * last field is 0 for the two-detector packing, else log2 R).  *chosen_logR (may
 * be NULL) receives log2 R of the chosen split, *chosen_pair (may be NULL) 1 for
 * the two-detector packing, else 0; *best_ms (may be NULL) the time of one
 * application, or -1 when the decision came from a cache. */
int cmm_autotune(cmm_op* op, int32_t reps, const char* cache_path, int32_t* chosen_logR, int32_t* chosen_pair,
                 double* best_ms);

#ifdef __cplusplus
}
#endif
#endif /* CMM_H */
