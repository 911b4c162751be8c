/*
 * qsel.h -- C ABI of the GB300 selected-inversion library.
 *
 * The library computes the marginal variances diag(Q^-1) and the log-determinant
 * gradients tr(Q^-1 dQ/dtheta_j) of the posterior precision of a space-time
 * latent Gaussian model (Zhumekenov, Krainski, Rue, "Parallel selected
 * inversion for space-time Gaussian Markov random fields", Section 1 and
 * Section 2.3, Eq. lgm:4) with the overlapping Rao-Blackwellized Monte Carlo
 * estimator of Section 3.2.3 (Algorithm 4) and the trace estimator of
 * Section 3.4.2 (Eq. hyperpar:4):
 *
 *   Q = tau (Q_t (x) Q_s) + A^T A / sigma^2,
 *   Q_s = (kappa^2 C + G) C^-1 (kappa^2 C + G)      (Section 2.1, alpha = 2),
 *   Q_t = unit-marginal-variance AR(1) precision     (Section 2.2, separable),
 *   theta = (log kappa, log tau, logit rho).
 *
 * Nodes are ordered space-fastest: global index = t * n_s + i for time slab t
 * and spatial node i (Section 2.2, Eq. spde:7).  Q is block tridiagonal in
 * time with n_s x n_s blocks.
 *
 * Pipeline run by qsel_diag_inv (all on the GPU, stream-ordered):
 *   1. perturbation right-hand sides r = F^T z1 + A^T z2 / sigma from
 *      Philox4x32-10 noise (Sections 2.4 and 3.3),
 *   2. one multi-right-hand-side preconditioned conjugate-gradient solve
 *      Q X = R for all samples at once (Section 3.3),
 *   3. per overlapping time subdomain Omega_p^*: exact block-tridiagonal
 *      factorisation and Takahashi selected inversion (Section 3.2.3; in the
 *      mixed form concurrently with step 2, which only step 4 needs),
 *   4. the Rao-Blackwell correction w = Q_{**}^-1 Q_{*S} x_S and its squares
 *      (Algorithm 4), restricted to Omega_p.
 *
 * Conventions
 *   - Every function returns a qsel_status; QSEL_OK is 0.  Nothing aborts,
 *     traps or exits.  A failed call leaves a message in qsel_last_error().
 *   - The caller owns every input and output buffer.  Inputs are copied at
 *     qsel_create; the context owns all device memory it allocates.
 *   - Work is issued on the CUDA stream given in qsel_options (NULL = the
 *     legacy default stream); every call returns after the stream has reached
 *     the end of its work (results are ready on return).  Inside a call the
 *     context may fork work onto non-blocking streams of its own (the PCG
 *     beside the first wave's factorisation, the sweep's look-ahead) and
 *     joins them back into that stream before it returns.
 *   - One context must not be used from two threads at the same time.
 *   - A CUDA error inside a call is reported as QSEL_ECUDA; the context must
 *     then be destroyed.
 */
#ifndef QSEL_H
#define QSEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qsel_ctx qsel_ctx;

typedef enum {
  QSEL_OK = 0,
  QSEL_EINVAL = 1,    /* invalid argument (shape, pointer, partition, option)   */
  QSEL_ENOMEM = 2,    /* device or host allocation failed                       */
  QSEL_ECUDA = 3,     /* CUDA runtime or launch error                            */
  QSEL_ENOTSPD = 4,   /* a pivot of a dense factorisation was not positive       */
  QSEL_ENOCONV = 5,   /* the conjugate-gradient solve hit pcg_max_iter           */
  QSEL_ETIMEOUT = 6,  /* a bounded device-side wait gave up (tensor-core GEMM)  */
  QSEL_ESTATE = 7     /* call not valid in the context's current state           */
} qsel_status;

/* Samplers of the global samples (qsel_options.sampler). */
enum {
  QSEL_SAMPLER_PCG = 0,
  QSEL_SAMPLER_LANCZOS = 1
};

/* Precision of the 64 x 64 pivot-tile inverses of the QSEL_MIXED dense
 * factorisation (qsel_options.pivot_precision); QSEL_FP64 always uses binary64. */
enum {
  QSEL_PIVOT_DOUBLE_FLOAT = 0,  /* hi + lo binary32 pairs (Dekker), about 48 bits  */
  QSEL_PIVOT_FP64 = 1           /* binary64                                         */
};

/* Preconditioners of the sampler's PCG (qsel_options.preconditioner). */
enum {
  QSEL_PRECOND_BLOCK_JACOBI = 0,
  QSEL_PRECOND_KRON = 1
};

/* Order of the one-part block factorisation (qsel_options.chain). */
#define QSEL_CHAIN_TWO_ENDED 0
#define QSEL_CHAIN_FORWARD 1

/* Space-time prior of qsel_create (qsel_options.model). */
enum {
  QSEL_MODEL_SEPARABLE = 0,     /* tau Q_t (x) Q_s, AR(1) in time (Section 2.2,
                                   separable case); theta = (log kappa, log tau,
                                   logit rho)                                    */
  QSEL_MODEL_DIFFUSION = 1,     /* the diffusion-based non-separable model of
                                   Section 2.2 (Eqs. spde:5-8) with (alpha_t,
                                   alpha_s, alpha_e) = (1, 2, 1), "critical
                                   diffusion":
                                     Q_u = gamma_e^2 [M0 (x) K3 + 2 gamma_t M1 (x) K2
                                                      + gamma_t^2 M2 (x) K1],
                                   K1 = gamma_s^2 C + G, K2 = K1 C^-1 K1,
                                   K3 = K2 C^-1 K1, and the temporal finite-element
                                   matrices of unit spacing: lumped mass M0 =
                                   diag(1/2, 1, .., 1, 1/2), boundary term M1 =
                                   diag(1/2, 0, .., 0, 1/2), Neumann stiffness M2;
                                   theta = (log gamma_s, log gamma_t, log gamma_e)
                                   in the fields (log_kappa, log_tau, logit_rho)
                                   of qsel_theta.  No factored form of Q exists:
                                   needs sampler = QSEL_SAMPLER_LANCZOS.         */
  QSEL_MODEL_BLOCK_TRIDIAGONAL = 2  /* a user-given matrix (qsel_create_bt)     */
};

/* Arithmetic of the pipeline. */
enum {
  QSEL_FP64 = 0,      /* every kernel computes in IEEE binary64                  */
  QSEL_MIXED = 1      /* binary32 solves and factorisations, extended-precision
                         pivot tiles (double-float or binary64, see
                         pivot_precision), binary64 refinement residuals and
                         accumulators.  The dense blocks are binary32, so the
                         diagonal's accuracy depends on the conditioning of the
                         pivot blocks in their smallest eigen-directions:
                         about 2e-4 relative (RMS) on observed models such as
                         the 96 x 96 bench workload, but tens of percent on an
                         unobserved prior with cond(Q_s) >= 1e4 (or
                         QSEL_ENOTSPD); use QSEL_FP64 for weakly observed,
                         ill-conditioned models                                   */
};

/*
 * Model inputs (Sections 2.1-2.3).  All pointers are HOST pointers, read
 * during qsel_create only.
 *   n_s, n_t       spatial nodes and time slabs, n = n_s * n_t.
 *   c_diag[n_s]    lumped mass matrix C (strictly positive).
 *   g_rowptr[n_s+1], g_col[nnz], g_val[nnz]
 *                  stiffness G in CSR, full symmetric pattern, 0-based.
 *   obs_mask[n]    1 where node t*n_s+i is observed (A selects these), else 0.
 *   sigma          observation standard deviation (Q_y = I / sigma^2), > 0.
 */
typedef struct {
  int32_t n_s, n_t;
  const double *c_diag;
  const int32_t *g_rowptr;
  const int32_t *g_col;
  const double *g_val;
  const uint8_t *obs_mask;
  double sigma;
} qsel_model;

/* Hyperparameters: kappa = exp(log_kappa), tau = exp(log_tau),
 * rho = 1 / (1 + exp(-logit_rho)). */
typedef struct {
  double log_kappa, log_tau, logit_rho;
} qsel_theta;

/*
 * Non-overlapping time partition Omega_p = slabs [slab_start[p], slab_start[p+1])
 * (Section 3.2.2; Section 4 partitions in time).  slab_start is a HOST array of
 * n_parts + 1 strictly increasing offsets from 0 to n_t, or NULL for the
 * balanced partition (the first n_t mod n_parts parts get one more slab).
 */
typedef struct {
  int32_t n_parts;
  const int32_t *slab_start;
} qsel_partition;

typedef struct {
  int32_t n_samples;      /* k >= 1: RBMC samples (columns of the PCG solve)       */
  uint64_t seed;          /* Philox key for the perturbation noise                 */
  int32_t precision;      /* QSEL_FP64 or QSEL_MIXED                               */
  double pcg_tol;         /* per-column stop: ||b_c - Q x_c|| <= tol ||b_c||        */
  int32_t pcg_max_iter;   /* > 0                                                   */
  int32_t precond_block;  /* block-Jacobi block size: 1 (Jacobi), 16, 32 or 64;
                             0 = library default                                   */
  int32_t control_variate;/* reserved, must be 0                                    */
  void *cuda_stream;      /* cudaStream_t, or NULL for the legacy default stream   */
  int32_t profile_kernels;/* non-zero: time every launch of the dense tile GEMM,
                             the sweep update and the SpMM with CUDA events on
                             the stream (reported in qsel_stats_t)                 */
  int32_t tensor_passes;  /* QSEL_MIXED dense products: 0 = default (3 when the
                             GPU has tcgen05 tensor cores, else CUDA cores),
                             3 = 3xTF32 (FP32-level accuracy), 1 = plain TF32,
                             -1 = FP32 CUDA cores.  Ignored for QSEL_FP64.        */
  int32_t sampler;        /* QSEL_SAMPLER_PCG (0): perturbation right-hand sides
                             solved by PCG (Sections 2.4, 3.3); QSEL_SAMPLER_LANCZOS
                             (1): the preconditioned Krylov sampler of
                             Algorithm 5.1 (FP64; needs no factored form of Q)  */
  int32_t lanczos_steps;  /* Krylov dimension m of the Lanczos sampler, 1..1024 */
  int32_t preconditioner; /* PCG preconditioner: QSEL_PRECOND_BLOCK_JACOBI (0,
                             blocks of precond_block rows, Section 3.3) or
                             QSEL_PRECOND_KRON (1): for m x m grid meshes
                             (stiffness T (x) D + D (x) T of the unit grid,
                             lumped mass D (x) D away from the corners), the
                             prior with C ~= D (x) D plus the mean observation
                             weight, inverted exactly in the basis of the 1-D
                             eigenvectors (QSEL_EINVAL for other meshes; not
                             in a batch)                                       */
  const int32_t *part_overlap;/* HOST array of n_parts overlaps n_l,p >= 0 (one per
                             part, read at qsel_create), or NULL: every part uses
                             the `overlap` argument.  Lets a planner
                             (qsel_cv_plan) extend each subdomain differently. */
  int32_t pivot_precision;/* QSEL_MIXED pivot-tile inverses:
                             QSEL_PIVOT_DOUBLE_FLOAT (0, default; on the binary32
                             pipe, which GB300 runs 64x faster than binary64) or
                             QSEL_PIVOT_FP64 (1).  Ignored for QSEL_FP64.       */
  int32_t model;          /* qsel_create: QSEL_MODEL_SEPARABLE (0) or
                             QSEL_MODEL_DIFFUSION (1); ignored by qsel_create_bt */
  int32_t chain;          /* order of the one-part (n_parts = 1) block
                             factorisation: QSEL_CHAIN_TWO_ENDED (0, default;
                             Schur complements from slab 0 and from slab n_t-1
                             toward the middle slab, two chains batched side by
                             side, the selected inverse then outward from the
                             middle; n_t >= 3) or QSEL_CHAIN_FORWARD (1; one
                             chain from slab 0).  Both are exact; they differ
                             in rounding order only.  Ignored with n_parts > 1 */
} qsel_options;

#define QSEL_PROF_CLASSES 11

/* Per-call statistics of the last qsel_diag_inv. */
typedef struct {
  int32_t pcg_iterations;     /* iterations until every column met pcg_tol         */
  double pcg_max_rel_residual;/* max over columns of ||b - Q x|| / ||b|| at exit   */
  double ms_rhs;              /* device time of each phase, milliseconds           */
  double ms_pcg;
  double ms_factor;           /* forward block factorisation (all subdomains)      */
  double ms_takahashi;        /* backward selected inversion (all subdomains)      */
  double ms_correction;       /* RB correction sweeps, squares and trace forms     */
  double ms_total;
  int64_t kernel_launches;    /* kernels this library launched in the call         */
  /* With profile_kernels: summed event time (ms), algorithmic work and launch
   * count per kernel class.  Work is FLOPs for the dense tile GEMM and the
   * sweep update, bytes (x read + y written once) for the SpMM. */
  double gemm_ms, gemm_flop;
  int64_t gemm_launches;
  double sweep_ms, sweep_flop;
  int64_t sweep_launches;
  double spmm_ms, spmm_bytes;
  int64_t spmm_launches;
  /* With profile_kernels: event time (ms) and launches per kernel class:
   * 0 dense tile GEMMs, 1 sweep updates (rank 64, or rank 256 per panel in
   * the mixed form), 2 SpMM, 3 pivot-tile inverses, 4 sweep panels (gathers,
   * panel steps and patches, scatters, mirror), 5 Schur assembly, 6 sparse
   * row and column gathers, 7 preconditioner apply (block Jacobi or the
   * Kronecker passes), 8 other PCG and
   * refinement vector kernels, 9 RB correction terms, 10 diagonal and pattern
   * extraction.  Kernels outside these classes are not timed.  class_work is
   * the algorithmic work where defined (FLOPs for 0, 1, 3, 7; bytes for 2),
   * else 0. */
  double class_ms[QSEL_PROF_CLASSES];
  int64_t class_launches[QSEL_PROF_CLASSES];
  double class_work[QSEL_PROF_CLASSES];
} qsel_stats_t;

/*
 * Create a context: validate and copy the model, build the Q_s sparsity
 * pattern and the partition (Omega_p extended by `overlap` slabs on each
 * side, clipped to [0, n_t); separators are the slabs just outside,
 * Algorithm 3), and allocate device memory.  No estimator work runs yet.
 *   out        receives the context (set to NULL on failure).
 *   overlap    n_l >= 0 slabs.
 * Errors: QSEL_EINVAL (shapes, mesh, mask, partition, options; a row of
 *         Q_s = K C^-1 K with more than 64 pattern entries),
 *         QSEL_ENOMEM, QSEL_ECUDA.
 */
qsel_status qsel_create(qsel_ctx **out, const qsel_model *model, const qsel_theta *theta,
                        const qsel_partition *partition, int32_t overlap,
                        const qsel_options *opt);

/* Replace the Philox key of the perturbation noise (qsel_options.seed); the
 * next qsel_diag_inv / qsel_trace_grads draw new samples.  Injected samples
 * are dropped. */
qsel_status qsel_set_seed(qsel_ctx *ctx, uint64_t seed);

/* Replace theta (structure, partition and options are kept).  The next
 * qsel_diag_inv / qsel_trace_grads recompute everything.  QSEL_EINVAL for
 * non-finite values or rho outside (0, 1). */
qsel_status qsel_set_theta(qsel_ctx *ctx, const qsel_theta *theta);

/*
 * Run the pipeline (if not already run for the current theta) and write the
 * RBMC estimate of diag(Q^-1) (Algorithm 4): n doubles in global node order.
 *   diag_out       caller-allocated, n doubles; HOST memory if out_is_device
 *                  is 0, DEVICE memory of the context's GPU otherwise.
 * Errors: QSEL_EINVAL (NULL), QSEL_ENOTSPD, QSEL_ENOCONV, QSEL_ECUDA.
 */
qsel_status qsel_diag_inv(qsel_ctx *ctx, double *diag_out, int32_t out_is_device);

/*
 * RBMC estimate of tr(Q^-1 dQ/dtheta_j) for the model's three
 * hyperparameters (separable: log kappa, log tau, logit rho; diffusion: log
 * gamma_s, log gamma_t, log gamma_e), by Eq. hyperpar:4: over rows of
 * Omega_p and columns of Omega_p^*, the selected entries Sigma*_il + (1/k)
 * sum_s w_i w_l times (dQ_j)_il.  Runs the pipeline if needed.  grads_out: 3
 * HOST doubles.  Requires overlap >= 1 or a single part (QSEL_EINVAL
 * otherwise): with no overlap the neighbours of the rows of Omega_p would lie
 * in the separator.  QSEL_EINVAL for a user-given matrix whose n_theta is not
 * 3 (use qsel_trace_grads_n).
 */
qsel_status qsel_trace_grads(qsel_ctx *ctx, double grads_out[3]);
/* The same for any number of derivatives: n must equal the context's n_theta
 * (3 for the built-in models); grads_out: n HOST doubles. */
qsel_status qsel_trace_grads_n(qsel_ctx *ctx, double *grads_out, int32_t n);

/*
 * A user-given block-tridiagonal precision (the generic form of the
 * estimator: Algorithm 4 needs only the block structure in time, Section
 * 3.2.3).  Q has n_t x n_t blocks of n_s x n_s on ONE spatial pattern:
 * diagonal blocks A_t and couplings B_t = Q[t, t+1] = Q[t+1, t]; every block
 * must be symmetric to 1e-12 relative per entry pair (the built-in models'
 * blocks are), and Q positive definite.  All pointers are HOST pointers, read during the call.
 *   rowptr[n_s + 1], col[nnz]   the pattern in CSR, 0-based, symmetric, with
 *                               every diagonal entry
 *   diag_vals[n_t * nnz]        A_t on the pattern, block after block
 *   off_vals[(n_t - 1) * nnz]   B_t on the pattern
 *   n_theta                     0..4 hyperparameters with trace gradients
 *   ddiag_vals[n_theta * n_t * nnz], doff_vals[n_theta * (n_t - 1) * nnz]
 *                               dA_t / dtheta_j and dB_t / dtheta_j, j major
 *                               (NULL when n_theta is 0)
 */
typedef struct {
  int32_t n_s, n_t;
  const int32_t *rowptr;
  const int32_t *col;
  const double *diag_vals;
  const double *off_vals;
  int32_t n_theta;
  const double *ddiag_vals;
  const double *doff_vals;
} qsel_bt_model;

/*
 * Create a context for a user-given block-tridiagonal precision; partition,
 * overlap and options as qsel_create.  There is no factored form, so the
 * global samples come from the Lanczos sampler (opt->sampler must be
 * QSEL_SAMPLER_LANCZOS) or from qsel_debug_set_samples; the preconditioner
 * is block Jacobi; theta plays no role (qsel_set_theta returns QSEL_EINVAL:
 * use qsel_set_bt_values).  The posterior-mean and hyperparameter calls are
 * not available (QSEL_EINVAL).
 * Errors: QSEL_EINVAL (shapes, pattern not symmetric or without a diagonal
 * entry, block values not symmetric or not finite, a row of more than 64
 * pattern entries, options), QSEL_ENOMEM, QSEL_ECUDA.
 */
qsel_status qsel_create_bt(qsel_ctx **out, const qsel_bt_model *model, const qsel_partition *partition,
                           int32_t overlap, const qsel_options *opt);
/* New values on the same pattern (layouts as qsel_bt_model; the derivative
 * arrays may be NULL when n_theta is 0).  The next qsel_diag_inv recomputes
 * everything.  QSEL_EINVAL for a context not made by qsel_create_bt or for
 * values that are not finite or not symmetric. */
qsel_status qsel_set_bt_values(qsel_ctx *ctx, const double *diag_vals, const double *off_vals,
                               const double *ddiag_vals, const double *doff_vals);

/*
 * Posterior mean and the gradient of the hyperparameter marginal, for the
 * model without fixed effects (Section 2.3, Eq. mean:5 with n_beta = 0;
 * Section 3.4, Eqs. hyperpar:1, 3, 4).
 *
 * qsel_set_data: the data y on the observed nodes, y_obs[q] for the q-th
 * observed node in increasing index order (n_obs HOST doubles, copied).
 * Errors: QSEL_EINVAL (NULL, no observed nodes), QSEL_ECUDA.
 */
qsel_status qsel_set_data(qsel_ctx *ctx, const double *y_obs);

/*
 * mu = Q^-1 A^T y / sigma^2 at the current theta, by the sampler's solver
 * (multi-RHS PCG in FP64, or FP32 PCG with FP64 refinement for QSEL_MIXED,
 * to pcg_tol).  mu_out: n doubles (host, or device with out_is_device).  The
 * solve reuses the sampler's right-hand-side and sample buffers
 * (qsel_debug_get_samples / get_rhs no longer return the last run's, and
 * samples injected by qsel_debug_set_samples are dropped: the next pipeline
 * run samples afresh); results of qsel_diag_inv / qsel_trace_grads are kept.
 * Errors: QSEL_ESTATE (no data), QSEL_ENOCONV, QSEL_ECUDA.
 */
qsel_status qsel_posterior_mean(qsel_ctx *ctx, double *mu_out, int32_t out_is_device);

/*
 * grad_out[j] = d log p(y | theta) / d theta_j (the marginal without the
 * hyperprior; add its gradient for log pi(theta | y)):
 *   1/2 d log|Q_x| / d theta_j - 1/2 tr(Q^-1 dQ_j) - 1/2 mu^T dQ_j mu,
 * with Q_x = tau Q_t (x) Q_s, dQ_j = dQ_x_j, the trace the RBMC estimate of
 * qsel_trace_grads (exact with a single part), mu the posterior mean, and
 * d log|Q_x| in closed form: 4 n_t kappa^2 tr(K^-1 C), n, n_s 2 rho^2
 * (n_t - 1) / (1 + rho) (K^-1 by the blocked sweep in binary64 on a dense
 * n_pad x n_pad matrix allocated at the first call).  Runs the pipeline if
 * needed.  terms_out (9 HOST doubles, or NULL): the prior log-determinant
 * derivatives, the traces and the quadratic forms mu^T dQ_j mu.
 * Errors: QSEL_EINVAL (NULL grad_out; overlap 0 with several parts),
 * QSEL_ESTATE (no data), QSEL_ENOTSPD, QSEL_ENOCONV, QSEL_ECUDA.
 */
qsel_status qsel_loglik_grad(qsel_ctx *ctx, double grad_out[3], double terms_out[9]);

/*
 * Fixed effects: y = A u + Z beta + eps with beta ~ N(0, I / beta_prec)
 * (Section 2.3, Eqs. mean:4-5, var:1; Eq. hyperpar:3).  Z: n_obs x n_beta
 * row-major HOST array (rows in the order of y_obs), copied; 0 <= n_beta <=
 * 63; n_beta = 0 removes them.  With fixed effects qsel_posterior_mean
 * returns mu_u and qsel_loglik_grad adds tr(S^-1 W^T dQ_j W) to the trace
 * term (S the Schur complement of Q_uu in the joint precision, W =
 * Q_uu^-1 A^T Z / sigma^2, both from the same multi-RHS solve as mu).
 * Errors: QSEL_EINVAL (range, NULL Z, beta_prec <= 0), QSEL_ECUDA.
 */
qsel_status qsel_set_covariates(qsel_ctx *ctx, int32_t n_beta, const double *Z, double beta_prec);

/*
 * mu_beta (n_beta HOST doubles), Var(beta) = S^-1 (n_beta^2, row-major HOST)
 * and the correction diag(W S^-1 W^T) that Eq. var:1 adds to diag(Q_uu^-1)
 * (n doubles, host or device with corr_is_device); any output may be NULL.
 * Solves as qsel_posterior_mean.
 * Errors: QSEL_ESTATE (no data or no covariates), QSEL_ENOTSPD, QSEL_ENOCONV,
 * QSEL_ECUDA.
 */
qsel_status qsel_fixed_effects(qsel_ctx *ctx, double *mu_beta_out, double *var_beta_out, double *var_u_corr_out,
                               int32_t corr_is_device);

/* Statistics of the last pipeline run. */
qsel_status qsel_stats(const qsel_ctx *ctx, qsel_stats_t *stats);

/*
 * Sample-based error estimate of the last diag(Q^-1) estimate.  The
 * correction of node i is the mean of k values w_i^2 (Algorithm 4); its
 * variance is estimated by (m4_i - m2_i^2) / (k - 1) with m2, m4 the sample
 * means of w_i^2 and w_i^4.  Reported per part p as the root mean square over
 * the rows of Omega_p of (standard error / estimate):
 *   part_err   HOST array of n_parts doubles, or NULL;
 *   global_err HOST double, the same over all rows (NULL allowed).
 * Parts without separators have zero error.  QSEL_ESTATE if the pipeline has
 * not run, QSEL_EINVAL if n_samples < 2.
 */
qsel_status qsel_error_estimate(qsel_ctx *ctx, double *part_err, double *global_err);

/*
 * Stage-wise checking hooks.
 *
 * qsel_debug_set_samples: use X (HOST, n rows x n_samples columns, row-major
 *   with leading dimension ld >= n_samples) as the global samples instead of
 *   running steps 1-2; only the separator slabs are read.  Stays in effect
 *   until qsel_set_theta or a solve of qsel_posterior_mean /
 *   qsel_fixed_effects / qsel_loglik_grad, which reuses the sample buffers.
 * qsel_debug_get_samples: copy the samples of the last run to X (HOST, same
 *   layout).
 * qsel_debug_get_rhs: copy the perturbation right-hand sides R of the last
 *   run (HOST, same layout).  QSEL_ESTATE if the samples were injected.
 * qsel_debug_get_selinv_diag: copy diag(Q_{Omega_p^* Omega_p^*}^-1) restricted
 *   to the rows of Omega_p, for every p, in global node order (HOST, n doubles):
 *   the exact subdomain selected inverse before the correction.
 */
qsel_status qsel_debug_set_samples(qsel_ctx *ctx, const double *X, int32_t ld);
qsel_status qsel_debug_get_samples(const qsel_ctx *ctx, double *X, int32_t ld);
qsel_status qsel_debug_get_rhs(const qsel_ctx *ctx, double *R, int32_t ld);
qsel_status qsel_debug_get_selinv_diag(const qsel_ctx *ctx, double *diag_out);
/* Lanczos sampler: the coefficients of T for every column of the last run,
 * alpha[j * ld + s] and beta[j * ld + s] for step j < lanczos_steps and
 * column s < n_samples (HOST, ld >= n_samples; beta[j] = ||w_j|| after step
 * j).  QSEL_ESTATE unless the last run used the Lanczos sampler. */
qsel_status qsel_debug_get_lanczos(const qsel_ctx *ctx, double *alpha, double *beta, int32_t ld);
/* Apply the context's PCG preconditioner to R (HOST, n x n_samples,
 * row-major, leading dimension ld) at the current theta and write Z = M^-1 R
 * (HOST, same layout).  A QSEL_MIXED context applies its binary32
 * preconditioner (R rounded to float, on the tensor cores where the mixed
 * sampler uses them). */
qsel_status qsel_debug_apply_precond(qsel_ctx *ctx, const double *R, double *Z, int32_t ld);

/*
 * Test hook for the bounded device-side waits of the tensor-core GEMM (the
 * mixed form's tcgen05 products).  Nothing faults: with skip_loads non-zero
 * the GEMM's producer issues no TMA load, so the waits of its other warps on
 * the empty stages run out after wait_cycles clock cycles (0 = the default,
 * about 2 s); every CTA then sets its error bit, waits (bounded) for the
 * tensor-core work it issued, frees its tensor memory and returns, and the
 * calling qsel_diag_inv reports QSEL_ETIMEOUT (its results are then
 * meaningless; destroy the context).  wait_cycles alone shortens the limit of
 * every wait.  Process-wide; qsel_debug_tc_wait(0, 0) restores normal
 * operation.  Errors: QSEL_EINVAL for wait_cycles < 0.
 */
qsel_status qsel_debug_tc_wait(int32_t skip_loads, int64_t wait_cycles);

/*
 * Scheduling hook of the mixed form's panel-blocked sweep (every pivot block
 * inverse), for measuring how its two streams share the GPU.  No work is
 * skipped and results are unchanged.  serial non-zero: each panel's
 * rank-64 bw update of the rest runs on the same stream as the pivot chain,
 * after it, instead of beside the next panel's pivots.  update_ctas > 0: the
 * persistent update kernel runs on at most that many CTAs (one per SM), so
 * that SMs stay free for the pivot chain; 0 = one per SM.  update_stages 2
 * or 3: the update's shared-memory ring (3 stages leave no room for the
 * pivot chain's CTAs on the update's SMs); 4: the update on 128 x 256
 * tiles by the persistent split-operand GEMM; 0 = the default.  By default
 * each pivot CTA asks for unused shared memory so that it cannot share an SM
 * with an update CTA, and the update (unless update_ctas says otherwise)
 * leaves one SM per pivot CTA free; shared_pivot non-zero lets the pivot CTAs
 * run beside update CTAs instead.  Process-wide;
 * qsel_debug_sweep_schedule(0, 0, 0, 0) restores the default.  Errors:
 * QSEL_EINVAL for update_ctas < 0 or update_stages not 0, 2, 3 or 4.
 */
qsel_status qsel_debug_sweep_schedule(int32_t serial, int32_t update_ctas, int32_t update_stages,
                                      int32_t shared_pivot);

/*
 * Allocation-free SPD inverse.  The paper has no counterpart: this entry point
 * exists for callers that cannot let a library call cudaMalloc -- code inside
 * a framework whose caching allocator owns the device memory budget (an
 * allocation outside it can fail or fragment memory the framework has
 * reserved), and long-running services that must keep their device memory
 * footprint fixed after start-up.  It runs the library's blocked
 * symmetric-sweep inverse (the kernel that inverts the pivot blocks of the
 * subdomain factorisation) on one caller-owned matrix and allocates nothing.
 *   a_dev        DEVICE pointer to an n x n symmetric positive definite
 *                matrix, row-major with leading dimension lda; overwritten
 *                in place with its inverse (both triangles).
 *   n, lda       1 <= n <= QSEL_NOALLOC_MAX_N, lda >= n.
 *   cuda_stream  cudaStream_t for the work, or NULL for the legacy default
 *                stream.  The call copies its pivot status back to the host
 *                and synchronises this stream before it returns (on the
 *                legacy stream that also waits for the other work on it).
 * Scratch: a file-scope device array of QSEL_NOALLOC_MAX_N^2 + 2 * 64 *
 *   QSEL_NOALLOC_MAX_N + 64^2 doubles (about 9 MiB), held by every GPU that
 *   loads this part of the library until the process exits.  The first call
 *   on each device looks up the array's device address with that device
 *   current (set-up); make that first call before any stream capture.  The
 *   looked-up address does not survive a device reset (cudaDeviceReset):
 *   calls after a reset are not supported.  Every call shares the array and
 *   overwrites what the last call left there (the status word is cleared at
 *   the start of each call), so calls that overlap on the GPU (other streams,
 *   other host threads) race: the caller must serialise them.
 * Errors: QSEL_EINVAL (NULL pointer, n out of range, lda < n), QSEL_ENOTSPD
 *   (non-positive pivot), QSEL_ECUDA; the message is in qsel_last_error(NULL).
 */
#define QSEL_NOALLOC_MAX_N 1024
qsel_status qsel_spd_inverse_noalloc(double *a_dev, int32_t n, int32_t lda, void *cuda_stream);

/*
 * Learned control variate.  The paper has no learned component; this part
 * serves the choice of overlap and sample count that the paper makes by hand
 * from the correlation range (Section 3.2.3, Section 6).  A 14-64-64-1 MLP
 * with GELU (erf form) activations, BF16 weights and FP32 accumulation
 * predicts, for every node, y_i = log(c_i / v_i): the share of the variance
 * v_i = Sigma*_ii + c_i that the Rao-Blackwell correction c_i = E[w_i^2]
 * carries.  Under Gaussian w the relative standard error of the k-sample
 * estimate of node i is sqrt(2 / k) c_i / v_i, so the prediction tells how
 * many samples and how much overlap a target error needs.  The estimate
 * itself stays plain RBMC at the chosen (overlap, k): it is unbiased whatever
 * the network predicts, and qsel_error_estimate judges the choice afterwards.
 *
 * Features of node (t, i), 14 floats per node, node order t * n_s + i:
 *   0      log Q_ii
 *   1..8   log |Q_il| of the 8 largest non-zero off-diagonal entries of the
 *          row, descending (log 1e-30 where the row has fewer)
 *   9      time distance from slab t to the nearest separator slab of the
 *          subdomain that owns it, capped at 16 (16 when it has none)
 *   10     graph distance of spatial node i to the mesh boundary (nodes with
 *          fewer stiffness neighbours than the maximum), capped at 8
 *   11..13 theta
 * Parameters (float, QSEL_CV_PARAMS_ALL values): W1 (64 x 14, row-major),
 * b1 (64), W2 (64 x 64), b2 (64), W3 (64), b3 (1), then the per-feature mean
 * (14) and scale (14) that standardise the inputs.  The first QSEL_CV_PARAMS
 * are trained.
 */
#define QSEL_CV_FEATURES 14
#define QSEL_CV_PARAMS 5185
#define QSEL_CV_PARAMS_ALL 5213

typedef struct qsel_cv qsel_cv;

/* Create a network with seeded Glorot-uniform weights, zero biases, mean 0
 * and scale 1; work is issued on cuda_stream (NULL = legacy default). */
qsel_status qsel_cv_create(qsel_cv **out, uint64_t seed, void *cuda_stream);
/* Copy all QSEL_CV_PARAMS_ALL parameters from / to HOST memory (Adam state is
 * kept on set). */
qsel_status qsel_cv_set_params(qsel_cv *cv, const float *params);
qsel_status qsel_cv_get_params(const qsel_cv *cv, float *params);
/* y_dev[s] = network(X_dev[s, :]) for n samples; DEVICE buffers, X row-major
 * n x QSEL_CV_FEATURES. */
qsel_status qsel_cv_predict(const qsel_cv *cv, const float *X_dev, float *y_dev, int32_t n);
/* Mean squared error (1/n) sum (network(X_s) - y_s)^2 and its gradient with
 * respect to the QSEL_CV_PARAMS trained parameters (as used: BF16 weights),
 * written to HOST grad_host (QSEL_CV_PARAMS floats) and loss_host (NULL
 * allowed).  X_dev, y_dev as in qsel_cv_predict. */
qsel_status qsel_cv_grad(qsel_cv *cv, const float *X_dev, const float *y_dev, int32_t n, float *grad_host,
                         float *loss_host);
/* `steps` full-batch Adam steps (beta 0.9 / 0.999, eps 1e-8, learning rate
 * lr) on the FP32 master parameters, refreshing the BF16 copies after each.
 * With set_input_stats the input mean and scale (standard deviation, at
 * least 1e-3) are first set from X.  loss_out (HOST, NULL allowed) receives
 * the loss of the final parameters. */
qsel_status qsel_cv_train(qsel_cv *cv, const float *X_dev, const float *y_dev, int32_t n, int32_t steps, float lr,
                          int32_t set_input_stats, float *loss_out);
void qsel_cv_destroy(qsel_cv *cv);

/* Features of ctx's model at its current theta and partition, with every
 * part extended by `overlap` slabs (the context's own overlap is not used),
 * written to F_dev (DEVICE, n x QSEL_CV_FEATURES floats). */
qsel_status qsel_cv_features(qsel_ctx *ctx, int32_t overlap, float *F_dev);

/* Training targets y_i = log(cbar_i / (Sigma*_ii + cbar_i)), cbar_i the mean
 * correction over `count` contexts that ran the same model and theta with
 * different seeds (their average is the RBMC estimate with all their samples);
 * ratios below 1e-9 are clamped (they add less than 1e-18 to any planned
 * squared error).  Each context must have run
 * (qsel_diag_inv).  y_dev: DEVICE, n floats. */
qsel_status qsel_cv_targets(qsel_ctx *const *ctxs, int32_t count, float *y_dev);

/*
 * Planner.  The network predicts every node's ratio c_i / v_i at each time
 * distance d = 1..16 to the nearest separator (16 = the feature's cap); for a
 * part p extended by n_l slabs, m_p = mean over Omega_p of the predicted
 * (c_i / v_i)^2 at the node's distance, so that k samples give the
 * predicted error e_p(k) = sqrt(2 m_p / k) (a part without a separator is
 * exact: e_p = 0).  For every candidate partition the planner picks one
 * sample count k (a multiple of 32 in [min_samples, max_samples]; the
 * samples are shared by every part) and per part the smallest overlap
 * 1..max_overlap with e_p(k) <= target, minimising the modelled time
 *   cost_pcg * k * n + sum_p T_p (cost_dense * n_pad^3 + cost_corr * k * n_pad^2),
 * T_p = slabs of the extended part, n_pad = n_s rounded up to 64; it returns
 * the cheapest candidate.  Candidates: the balanced partitions into each of
 * part_counts (a count of 1 is the exact one-part form, cost cost_dense *
 * n_t * n_pad^3, no samples: n_samples = 0), or, with n_part_counts = 0, the
 * context's own partition.  The plan also reports the modelled cost of the
 * exact one-part alternative.  Cost coefficients of 0 take GB300
 * mixed-precision defaults (seconds: 1.53e-8, 1.10e-13, 2.2e-13).  When no
 * candidate meets the target everywhere the plan takes the first candidate
 * at max_samples and max_overlap and sets feasible = 0.
 */
typedef struct {
  double target_rel_err;      /* RMS relative standard error per part, > 0      */
  int32_t max_overlap;        /* >= 1                                          */
  int32_t min_samples, max_samples; /* 32 <= min <= max <= 512                  */
  double cost_pcg, cost_dense, cost_corr;
  const int32_t *part_counts; /* HOST, n_part_counts entries in 1..n_t, or NULL */
  int32_t n_part_counts;      /* 0 = plan the context's own partition           */
} qsel_cv_plan_options;

typedef struct {
  int32_t n_samples;          /* chosen k (0 for the one-part form)             */
  int32_t feasible;           /* 1 if every part meets the target              */
  double predicted_cost;      /* modelled seconds                              */
  double predicted_err;       /* max over parts of the predicted error         */
  double single_part_cost;    /* modelled seconds of the exact alternative: one
                                 part (no separator, no samples), cost_dense *
                                 n_t * n_pad^3                                   */
  int32_t *part_overlap;      /* caller-allocated HOST, room for the largest
                                 candidate's part count: chosen n_l,p           */
  double *part_pred_err;      /* caller-allocated HOST, same size, or NULL      */
  int32_t n_parts;            /* part count of the chosen partition            */
  int32_t *slab_start;        /* caller-allocated HOST (largest count + 1), or
                                 NULL: offsets of the chosen partition          */
} qsel_cv_plan_t;

qsel_status qsel_cv_plan(qsel_ctx *ctx, const qsel_cv *cv, const qsel_cv_plan_options *opt, qsel_cv_plan_t *plan);

/*
 * Batch of independent models (uneven sizes), solved together: the whole
 * pipeline of every model is captured once into one CUDA graph, one branch
 * per model on a pool of streams (models placed longest-first on the least
 * loaded stream), with the sampler's convergence loops as conditional while
 * nodes driven by the device (no host round trip per check; every loop is
 * bounded by pcg_max_iter and 30 refinement steps).  Later runs replay the
 * graph; qsel_batch_set_theta changes a model's theta between replays.
 * The paper has no batch; it serves many small problems at once (one
 * problem of the size used here leaves most of a GB300 idle).
 *   models, thetas, partitions, overlaps: HOST arrays of n_models entries
 *                (read during the call), as for qsel_create.
 *   opt          shared options; model i uses seed opt->seed + i.
 *                opt->cuda_stream is the stream the graph is launched on
 *                (NULL: the batch creates its own; the legacy default stream
 *                cannot be captured).  profile_kernels and part_overlap must
 *                be 0 / NULL, sampler QSEL_SAMPLER_PCG, preconditioner
 *                QSEL_PRECOND_BLOCK_JACOBI.
 *   n_streams    1..64 streams in the pool.
 *   autotune     non-zero: for every grid size (n_s) the smallest model of
 *                that size is run with every block-Jacobi block in {16, 32,
 *                64} and, in the mixed form with tensor cores, both dense
 *                tile paths (128x128 tcgen05 tiles, 64x64 CUDA-core tiles);
 *                the fastest pair is used for every model of that size.
 * Errors: as qsel_create (message in qsel_batch_last_error(NULL)).
 */
typedef struct qsel_batch qsel_batch;

typedef struct {
  int32_t n_models, n_streams;
  double ms_replay;           /* device time of the last replay (CUDA events)  */
  double ms_capture;          /* host time of capture + instantiation          */
  double ms_autotune;         /* host time of the autotuner at creation        */
  int64_t launches_per_replay;/* kernels in the graph outside the loop bodies,
                                 plus one pass of every loop body              */
  int32_t max_pcg_iterations; /* over models, last replay                      */
} qsel_batch_info_t;

qsel_status qsel_create_batch(qsel_batch **out, int32_t n_models, const qsel_model *models,
                              const qsel_theta *thetas, const qsel_partition *partitions, const int32_t *overlaps,
                              const qsel_options *opt, int32_t n_streams, int32_t autotune);
/* Capture (first call) and replay the graph; returns when every model is
 * done.  A failure names the model (QSEL_ENOTSPD, QSEL_ENOCONV,
 * QSEL_ETIMEOUT, QSEL_ECUDA). */
qsel_status qsel_batch_run(qsel_batch *b);
qsel_status qsel_batch_set_theta(qsel_batch *b, int32_t model, const qsel_theta *theta);
/* Results of model `model` (runs the batch first if needed); layouts as
 * qsel_diag_inv / qsel_trace_grads. */
qsel_status qsel_batch_diag_inv(qsel_batch *b, int32_t model, double *diag_out, int32_t out_is_device);
qsel_status qsel_batch_trace_grads(qsel_batch *b, int32_t model, double grads_out[3]);
/* Per-model statistics of the last replay: pcg_iterations and
 * pcg_max_rel_residual (no phase times in a graph). */
qsel_status qsel_batch_stats(const qsel_batch *b, int32_t model, qsel_stats_t *stats);
qsel_status qsel_batch_info(const qsel_batch *b, qsel_batch_info_t *info);
/* The tuned settings of a model and the stream it runs on (NULL allowed). */
qsel_status qsel_batch_tuning(const qsel_batch *b, int32_t model, int32_t *precond_block, int32_t *tensor_passes,
                              int32_t *stream);
/* Message of the last failed call on b (NULL: of the last failed
 * qsel_create_batch on this thread). */
const char *qsel_batch_last_error(const qsel_batch *b);
void qsel_batch_destroy(qsel_batch *b);

/* Message of the last failed call on ctx, or, when ctx is NULL, of the last
 * failed qsel_create, qsel_spd_inverse_noalloc or qsel_cv_* call (those that
 * take no context) on this thread.  Never NULL; owned by the library. */
const char *qsel_last_error(const qsel_ctx *ctx);

/* Free the context and its device memory.  NULL is allowed. */
void qsel_destroy(qsel_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* QSEL_H */
