/*
 * hmle.h -- C ABI of the GB300-native H-MLE library (libhmle.so).
 *
 * The library evaluates the Gaussian log-likelihood of Eq. 1 (Sec. 1),
 *
 *     L(theta) = -n/2 log(2 pi) - 1/2 log|C(theta)| - 1/2 Z^T C(theta)^{-1} Z,
 *
 * for the Matern covariance of Eq. 2 (Sec. 1),
 *
 *     C(h; theta) = sigma^2 / (2^(nu-1) Gamma(nu)) (h/ell)^nu K_nu(h/ell) + tau^2 I,
 *
 * with C(theta) held as a hierarchical matrix (Sec. 2): a cluster tree and a
 * block tree partition C into admissible blocks, approximated by low-rank
 * factors built on the fly, and inadmissible leaf blocks kept dense.  The
 * H-Cholesky factor C ~= L L^T gives log|C| = 2 sum log L_ii and
 * Z^T C^{-1} Z = |L^{-1} Z|^2 (Sec. 2, "Storage and complexity").  The
 * maximum-likelihood estimate maximises L over theta (Sec. 2,
 * "Maximization of the log-likelihood"; positivity transform of Sec. 5).
 *
 * Every numerical step runs in CUDA kernels on the current device; the host
 * only plans (θ-independent schedules), launches and runs the optimiser's
 * 4-dimensional simplex bookkeeping.
 *
 * Conventions
 *  - All functions return an hmle_status and never abort.  On failure the
 *    context keeps a message, readable with hmle_last_error().
 *  - Pointers to caller data may be host or CUDA device memory; the kind is
 *    detected with cudaPointerGetAttributes.  The caller keeps ownership of
 *    every array it passes; the library copies what it keeps.
 *  - Handles (hmle_ctx, hmle_tree, hmle_hmatrix, hmle_hfactor) are owned by
 *    the library and released with the matching *_destroy call (NULL is a
 *    no-op).  A tree refers to its context, an H-matrix to its tree and a
 *    factor to its H-matrix: destroy them in the reverse order of creation.
 *    A handle must not be used concurrently from two host threads.
 *  - theta is passed by name, in the order (ell, nu, sigma2, tau2).
 *  - Z is always given in the caller's point order; the internal cluster
 *    permutation never leaks out.
 */
#ifndef HMLE_H
#define HMLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMLE_OK = 0,
  HMLE_ERR_INVALID_ARG = 1,    /* bad size, NULL, non-finite or out-of-range value */
  HMLE_ERR_NOT_SPD = 2,        /* a non-positive pivot in a diagonal leaf factorisation */
  HMLE_ERR_OOM = 3,            /* device or host allocation failed */
  HMLE_ERR_CUDA = 4,           /* a CUDA runtime call failed (message has the detail) */
  HMLE_ERR_RANK_OVERFLOW = 5,  /* a low-rank block needed more than max_rank terms */
  HMLE_ERR_TIMEOUT = 6,        /* a bounded device wait ran out */
  HMLE_ERR_NOT_CONVERGED = 7,  /* hmle_fit hit max_iter before its tolerance */
  HMLE_ERR_NOT_IMPLEMENTED = 8
} hmle_status;

/* Arithmetic of the factorisation.
 *  HMLE_FP64        every step in FP64.
 *  HMLE_MIXED_FP32  the mixed form: the products of the Schur-complement
 *                   updates, of the Grams and of the W-panel updates run on
 *                   the tensor cores (tcgen05.mma, BF16 operands, FP32
 *                   accumulation), every operand split into three BF16
 *                   slices (24 bits, the FP32 significand; six products per
 *                   step of k); the QR / SVD recompression, the diagonal
 *                   POTRF, the TRSM, the W-panel triangular solves, the
 *                   log-determinant and the solves used as a preconditioner
 *                   stay FP64.  log|C~| comes from the mixed factor;
 *                   Z^T C~^{-1} Z is won back by preconditioned conjugate
 *                   gradients on the FP64 H-matrix of C with the mixed factor
 *                   as preconditioner (pcg_tol, pcg_max_iter).  The mixed
 *                   factor is truncated at max(aca_eps, 1e-7).
 *  HMLE_MIXED_BF16  the same with every operand split into two BF16 slices
 *                   (16 bits; three products per step of k); the factor is
 *                   truncated at max(aca_eps, 1e-5).  A single BF16 slice
 *                   (8 bits) is not offered: its error, about 2^-9 of the
 *                   updates' norm, exceeds the smallest eigenvalues of the
 *                   diagonal leaves of a covariance with a small nugget, and
 *                   the POTRF of such a leaf would fail. */
typedef enum { HMLE_FP64 = 0, HMLE_MIXED_FP32 = 1, HMLE_MIXED_BF16 = 2 } hmle_precision;

/* Matern parameters of Eq. 2: range ell > 0, smoothness nu > 0,
 * variance sigma2 >= 0, nugget tau2 >= 0. */
typedef struct {
  double ell, nu, sigma2, tau2;
} hmle_theta;

/* H-matrix options (the paper leaves the H-matrix construction to the
 * library it used; these are the knobs of this implementation).
 *  leaf_size  b: clusters with at most b points are leaves; a multiple of
 *             16 in [16, 128].
 *  eta        admissibility: block (t, s) is low-rank when
 *             min(diam t, diam s) <= eta * dist(t, s) (bounding boxes).
 *  aca_eps    relative accuracy of every low-rank block, in (0, 1): ACA of C
 *             stops at |u_k||v_k| <= eps |S_k|_F; the truncation of a
 *             Schur-complement block S drops the trailing singular values
 *             whose energy sum is <= eps^2 max(|S|_F^2, |C_block|_F^2).
 *  max_rank   capacity (columns) of every low-rank block of L~; a multiple
 *             of 8 in [8, 64].  ACA of C may use up to max_rank + 16 (at
 *             most 64).
 *  oversample extra random samples beyond max_rank for the compression of
 *             updated low-rank blocks; >= 4 with max_rank + oversample <= 64.
 *  seed       seed of the counter-based random signs used by that
 *             compression (the result is deterministic for a given seed).
 *  leaf_lowrank  0 (default): admissible blocks between two leaf clusters
 *             (at most leaf_size^2 entries) are kept dense and exact; 1: they
 *             are held low-rank like the coarser admissible blocks.
 *  pcg_tol, pcg_max_iter  mixed form only: PCG stops when |r| <= pcg_tol |Z|
 *             (default 1e-10) or fails with HMLE_ERR_NOT_CONVERGED after
 *             pcg_max_iter iterations (default 50).
 *  fixed_rank 0 (default): fixed accuracy, every block at eps (Sec. 2, the
 *             accuracy-fixed approximation); k in 1..max_rank: fixed rank,
 *             every block of C~ and of L~ at most k (Sec. 2, the rank-fixed
 *             approximation; the accuracy then varies from block to block and
 *             no rank overflow is reported).
 *  batch_size evaluations of hmle_loglik_batch served by one launch of every
 *             sweep kernel (gridDim.z), in [1, 64]; default 2.  A batch of
 *             concurrency evaluations runs as ceil(concurrency / batch_size)
 *             such launches sequences on their own streams, side by side, and
 *             the mixed forms' PCG solves all of them in one lockstep
 *             iteration.  Results do not depend on it (hmle_autotune picks
 *             it with the leaf size and the concurrency). */
typedef struct {
  int32_t leaf_size;
  double eta;
  double aca_eps;
  int32_t max_rank;
  int32_t oversample;
  int32_t precision; /* hmle_precision */
  uint64_t seed;
  int32_t leaf_lowrank;
  double pcg_tol;
  int32_t pcg_max_iter;
  int32_t fixed_rank;
  int32_t batch_size;
} hmle_opts;

/* Nelder-Mead options of hmle_fit (Sec. 2: threshold 1e-4, <= 400 iterations). */
typedef struct {
  double ftol;      /* stop when max |f_i - f_best| over the simplex <= ftol ... */
  double xtol;      /* ... and max |x_i - x_best|_inf (transformed coords) <= xtol */
  int32_t max_iter; /* iteration cap */
  double step[4];   /* initial simplex steps in transformed coordinates
                       (sigma0, ell0, nu0, tau0); all 0 means 1.0 each */
} hmle_fit_opts;

typedef struct {
  int64_t n;            /* number of points */
  int32_t d;            /* dimension (2 or 3) */
  int32_t depth;        /* leaves are at this level; root is level 0 */
  int32_t n_leaves;     /* 2^depth */
  int32_t n_dense;      /* dense leaf blocks in the lower triangle (incl. diagonal) */
  int32_t n_lowrank;    /* admissible blocks in the lower triangle */
  int64_t dense_words;  /* doubles held by dense blocks */
  int64_t lowrank_words;/* doubles reserved for low-rank factors (C and L) */
  int64_t device_bytes; /* device memory held by the tree and its plan */
} hmle_tree_info;

typedef struct {
  double logdet;        /* log|C~| */
  double quad;          /* Z^T C~^{-1} Z */
  double loglik;        /* Eq. 1 */
  int32_t max_rank_c;   /* largest ACA rank among blocks of C~ */
  int32_t max_rank_l;   /* largest rank among low-rank blocks of L~ */
  double mean_rank_l;   /* mean rank of low-rank blocks of L~ */
  int32_t status;       /* hmle_status of the evaluation */
  int64_t kernel_launches; /* CUDA kernels this evaluation launched */
  int32_t pcg_iters;    /* mixed form: PCG iterations (0 in FP64) */
  double pcg_relres;    /* mixed form: final |r| / |Z| */
  double flops;         /* algorithmic flops of the factorisation sweep (the plan's
                           products at this evaluation's ranks; FP32 ones included
                           in the mixed form) */
} hmle_eval_info;

typedef struct hmle_ctx hmle_ctx;
typedef struct hmle_tree hmle_tree;
typedef struct hmle_hmatrix hmle_hmatrix;
typedef struct hmle_hfactor hmle_hfactor;

/* The H-matrix options of Sec. 2's construction (the knobs of this
 * implementation; the paper leaves them to its library).
 * Fill *opts with defaults: leaf 64, eta 2, aca_eps 1e-8, max_rank 32,
 * oversample 8, FP64, seed 0x5eed, leaf_lowrank 0, pcg_tol 1e-10,
 * pcg_max_iter 50, fixed_rank 0, batch_size 2.  HMLE_OK for non-NULL opts, else
 * INVALID_ARG. */
hmle_status hmle_opts_default(hmle_opts *opts);

/* Fill *opts with the paper's optimiser settings: ftol = xtol = 1e-4,
 * max_iter = 400, unit steps. */
hmle_status hmle_fit_opts_default(hmle_fit_opts *opts);

/* Plumbing, no counterpart in the paper.
 * Create a context on the current CUDA device.  stream: a cudaStream_t to
 * launch on, or NULL for a stream owned by the context.  One context per
 * stream; a context must not be shared between host threads. */
hmle_status hmle_ctx_create(hmle_ctx **ctx, void *stream);
void hmle_ctx_destroy(hmle_ctx *ctx);

/* Message of the last failure on this context ("" when none).  The string
 * stays valid until the next call on the context. */
const char *hmle_last_error(const hmle_ctx *ctx);

/* a1-a2 (Sec. 2, recursive block partition): build the geometric cluster
 * tree (bounding boxes, median split along the longest axis, stable point
 * permutation) and the block tree (admissibility by eta) on the device, then
 * the θ-independent factorisation schedule.
 *  locs  n x d doubles, row-major (point i at locs[i*d .. i*d+d-1]), host or
 *        device memory; copied.
 *  n     >= 2 points;  d in {2, 3};  opts may be NULL for defaults.
 * Errors: INVALID_ARG (sizes, non-finite coordinates, bad options), OOM, CUDA. */
hmle_status hmle_build_tree(hmle_ctx *ctx, const double *locs, int64_t n,
                            int32_t d, const hmle_opts *opts, hmle_tree **out);
void hmle_tree_destroy(hmle_tree *tree);
/* a1-a2 (Sec. 2): sizes of the cluster and block trees and of the schedule
 * (host struct).  Errors: INVALID_ARG. */
hmle_status hmle_tree_get_info(const hmle_tree *tree, hmle_tree_info *info);
/* a1 (Sec. 2): the cluster order of the tree's points: perm[k] = caller
 * index of the point at cluster position k (host array of n int32).
 * Errors: INVALID_ARG, CUDA. */
hmle_status hmle_tree_permutation(const hmle_tree *tree, int32_t *perm);

/* a3-a4 (Eq. 2; Sec. 2, low-rank approximation on the fly): assemble
 * C~(theta) on the device -- Matern entries of the dense leaf blocks and
 * adaptive-cross-approximation factors U V^T of the admissible blocks,
 * built from rows and columns of the kernel without forming the block.
 * Errors: INVALID_ARG (theta out of range), RANK_OVERFLOW, OOM, CUDA. */
hmle_status hmle_assemble(hmle_ctx *ctx, const hmle_tree *tree,
                          const hmle_theta *theta, hmle_hmatrix **out);
void hmle_hmatrix_destroy(hmle_hmatrix *h);

/* Sec. 2 (the H-matrix approximation of Eq. 2's covariance): y = C~ x for
 * one vector (caller order, host or device, n doubles each); a check of the
 * assembled H-matrix, and the operator of the mixed forms' PCG (a14).
 * Errors: INVALID_ARG, OOM, CUDA. */
hmle_status hmle_hmatrix_matvec(hmle_ctx *ctx, const hmle_hmatrix *h,
                                const double *x, double *y);

/* a6-a10 (Sec. 2, H-Cholesky and solve): factor C~ = L~ L~^T by a
 * left-looking sweep over the leaf clusters (dense diagonal and near-field
 * leaves; every low-rank block compressed once from all its Schur-complement
 * updates: randomised range sampling, Householder TSQR, column-pivoted QR and
 * a Jacobi SVD truncated at eps), and, when Z is not NULL, run the forward
 * solve w = L~^{-1} P Z inside the same sweep.  With precision =
 * HMLE_MIXED_FP32 the update products run in FP32 and, when Z is given, the
 * quadratic form comes from PCG (see hmle_precision).
 *  h  the assembled matrix; it is not modified and may be reused.
 *  Z  n doubles in caller order (host or device) or NULL.
 * Errors: NOT_SPD, RANK_OVERFLOW, OOM, CUDA. */
hmle_status hmle_factor(hmle_ctx *ctx, const hmle_hmatrix *h, const double *Z,
                        hmle_hfactor **out);
void hmle_factor_destroy(hmle_hfactor *f);

/* a9-a12 (Eq. 1): log-likelihood from a factor.  With Z (n doubles, caller
 * order, host or device) the forward solve w = L~^{-1} P Z runs as a sweep
 * through the stored factor and q = |w|^2; with Z = NULL the solve fused
 * into hmle_factor is used (INVALID_ARG if the factor was built without Z).
 * loglik must not be NULL; logdet and quad may be.  Errors: INVALID_ARG, CUDA. */
hmle_status hmle_loglik(hmle_ctx *ctx, const hmle_hfactor *f, const double *Z,
                        double *loglik, double *logdet, double *quad);

/* a10-a11 (the linear solve of Sec. 2 and Eq. 4's C11^{-1} Z1): X =
 * C~^{-1} Z = P^T L~^{-T} L~^{-1} P Z, by the forward sweep and the reverse
 * (backward) sweep through the factor.  Z, X: n doubles in caller order,
 * host or device (they may not alias).  Afterwards hmle_loglik(f, NULL)
 * returns L for this Z.
 * Errors: INVALID_ARG, OOM, CUDA. */
hmle_status hmle_solve(hmle_ctx *ctx, const hmle_hfactor *f, const double *Z, double *X);

/* The MLE with the variance profiled out (Sec. 7 suggests updating instead
 * of recomputing; with C = sigma2 (R(ell, nu) + rho I), rho = tau2 / sigma2,
 * the maximiser over sigma2 is sigma2 = Z^T R_rho^{-1} Z / n in closed form).
 * Nelder-Mead runs over 3 coordinates (ell0, nu0, r0) with ell = 1 / 1.5^ell0,
 * nu = 1 / 1.2^nu0 (Sec. 5) and rho = (1 / 2^r0)^2 on the profile likelihood
 *   L_p = -n/2 log(2 pi) - n/2 log(Z^T R_rho^{-1} Z / n) - 1/2 log|R_rho| - n/2,
 * each trial point one evaluation at (ell, nu, 1, rho).  It maximises the same
 * likelihood as hmle_fit with one coordinate less.  fit_opts as hmle_fit
 * (step[1..3] are the steps of ell0, nu0, r0; step[0] is unused).
 * theta_hat = (ell, nu, sigma2_hat, rho sigma2_hat); *ll_hat = L(theta_hat).
 * Errors: as hmle_fit. */
hmle_status hmle_fit_profiled(hmle_ctx *ctx, const hmle_tree *tree, const double *Z,
                              const hmle_theta *theta0, const hmle_fit_opts *fit_opts,
                              hmle_theta *theta_hat, double *ll_hat, int32_t *n_iter,
                              int32_t *n_evals);

/* Cross-covariance products between the tree's n points and m new locations
 * (the C21 / C12 blocks of Sec. 1, without a nugget) at theta:
 *  trans = 0: y (m) = C21 x (x: n doubles, caller order);
 *  trans = 1: y (n, caller order) = C12 x (x: m doubles).
 * locs2: m x d row-major, m >= 1.  Every pointer host or device.  Used with hmle_solve
 * for the prediction variances of Eq. 5-6.  Errors: INVALID_ARG, OOM, CUDA. */
hmle_status hmle_cross_matvec(hmle_ctx *ctx, const hmle_tree *tree, const hmle_theta *theta,
                              const double *locs2, int64_t m, int32_t trans, const double *x,
                              double *y);

/* next 1 (Eq. 5-6): the prediction errors of the kriging predictor at m
 * test locations, for a true model theta_t (the factor f_true of C~ at
 * theta_t, and its H-matrix) and an approximated model theta_a (f_approx at
 * theta_a), both factors on one tree.  With c_x(j) the column C12 at theta_x
 * for test location s_j (no nugget), C~_x the training covariance (nugget
 * included) and v_x = sigma2_x + tau2_x the variance of Z(s_j):
 *   e_tt(j) = v_t - c_t^T C~_t^{-1} c_t          E_t[(Z_t - Z)^2]
 *   e_aa(j) = v_a - c_a^T C~_a^{-1} c_a          E_a[(Z_a - Z)^2]
 *   e_ta(j) = v_t - 2 l_a^T c_t + l_a^T C~_t l_a, l_a = C~_a^{-1} c_a
 *                                                E_t[(Z_a - Z)^2]
 *   MLOE = mean_j (e_ta / e_tt - 1) (Eq. 5), MMOM = mean_j (e_aa / e_ta - 1)
 * (Eq. 6).  All of it runs on the device in rounds of up to 256 locations:
 * the columns generated from the Matern function, the solves C~^{-1} as one
 * cooperative forward and one backward sweep over all the round's columns
 * (multi-vector form of hmle_solve's sweeps), C~_t l_a as H-matvecs of 32
 * columns per launch, the dot products per column in a fixed order.  The
 * solves use the factors as they are (a mixed-form factor carries its
 * FP32-class products into them).
 *  locs2      m x d row-major (host or device), 1 <= m <= 2^24;
 *  mloe, mmom the means (either may be NULL);
 *  per_point  NULL or 3 m doubles (host): e_tt, e_aa, e_ta per location.
 * Device memory: 5 x 256 x n doubles of columns plus workspaces, freed
 * before returning.  Errors: INVALID_ARG (factors of two trees, m out of
 * range, no output), NOT_IMPLEMENTED (no cooperative launch on the
 * device), OOM, CUDA, TIMEOUT (a barrier wait of a sweep ran out). */
hmle_status hmle_prediction_errors(hmle_ctx *ctx, const hmle_hfactor *f_true,
                                   const hmle_hfactor *f_approx, const double *locs2, int64_t m,
                                   double *mloe, double *mmom, double *per_point);

/* Kriging prediction (Eq. 4): Z2 = C21 C11^{-1} Z1 at m new locations, the
 * conditional mean of the field there given Z1 (Sec. 1).  C11^{-1} Z1 comes
 * from the factor f of C11 (forward and backward sweeps, as hmle_solve); C21
 * is generated from the Matern function at f's theta, without a nugget (the
 * new locations are other points).  Z1: n doubles in caller order; locs2:
 * m x d row-major, m >= 1; Z2: m doubles (host or device each).  Afterwards
 * hmle_loglik(f, NULL) returns L for this Z1.
 * Errors: INVALID_ARG, OOM, CUDA, TIMEOUT. */
hmle_status hmle_predict(hmle_ctx *ctx, const hmle_hfactor *f, const double *Z1,
                         const double *locs2, int64_t m, double *Z2);

/* One full evaluation L(theta): assemble + factor with the fused solve +
 * combine, on a tree.  info may be NULL.  This is the unit of work of the
 * MLE (Sec. 2: one H-Cholesky, one solve and one scalar product per
 * iteration).  Errors: as hmle_assemble and hmle_factor. */
hmle_status hmle_loglik_eval(hmle_ctx *ctx, const hmle_tree *tree,
                             const hmle_theta *theta, const double *Z,
                             double *loglik, hmle_eval_info *info);

/* a15 (batched form): m evaluations L(theta_i) on one tree, up to
 * `concurrency` of them in flight at once (0 means 8), each on its own
 * evaluation buffers, stream pair and captured graph, so that independent
 * trial points of the optimiser fill the GPU together.
 *  thetas  m >= 0 parameter sets (m = 0 returns HMLE_OK at once);
 *          Z  n doubles (caller order, host or device),
 *          shared by all evaluations;  ll  m outputs (-inf for a failed one);
 *  status  m per-evaluation statuses, or NULL.
 * Returns the first hard error (CUDA, OOM, INVALID_ARG, TIMEOUT), or
 * HMLE_OK; NOT_SPD, RANK_OVERFLOW and NOT_CONVERGED (the mixed form's PCG)
 * are reported per evaluation only.  Device memory holds
 * one evaluation's buffers per concurrent slot, carved from one allocation
 * and kept with the tree while the batch shape stays the same. */
hmle_status hmle_loglik_batch(hmle_ctx *ctx, const hmle_tree *tree, const hmle_theta *thetas,
                              int32_t m, const double *Z, int32_t concurrency, double *ll,
                              int32_t *status);

/* a15 (batched form over instances): one task = one field on one tree at
 * one theta.  Tasks may mix trees of different sizes n (instances of uneven
 * n) and repeat a tree with many thetas (simplex vertices, line-search
 * trials); they run in waves of up to `concurrency` (0 means 8), each on a
 * buffer of its own tree, streams and captured graph as in
 * hmle_loglik_batch.  Z of a task: n_tree doubles in caller order, host or
 * device; tasks that pass the same Z pointer share one staged copy.  ntask
 * = 0 returns HMLE_OK at once.  A tree's evaluation buffers are released
 * after the wave of its last task, so the device holds at most the buffers
 * of the trees of two waves: many trees of uneven n fit in one call when
 * their tasks are grouped by tree.
 * Outputs and errors as hmle_loglik_batch. */
typedef struct {
  const hmle_tree *tree;
  hmle_theta theta;
  const double *Z;
} hmle_task;
hmle_status hmle_loglik_multi(hmle_ctx *ctx, const hmle_task *tasks, int32_t ntask,
                              int32_t concurrency, double *ll, int32_t *status);

/* a15, robust form (project-written; the paper runs each evaluation once):
 * hmle_loglik_multi, then every task whose evaluation failed is evaluated
 * again, up to max_retries (0..8) times, on a tree derived from its own (the
 * same points and cluster tree, a new plan), one rung further on this ladder
 * per retry:
 *  RANK_OVERFLOW   first the rank capacity raised to its largest (max_rank
 *                  56, oversample 8, ACA capacity 64) if it was lower, then
 *                  aca_eps x 10 per retry up to 1e-3 (a coarser H-matrix, so
 *                  the result is that of the looser accuracy: see retry);
 *  NOT_CONVERGED, NOT_SPD of a mixed form   the products in FP64.
 * Other failures are not retried.  Derived trees are built once per (tree,
 * options) in the call and destroyed before it returns.
 *  ll, status  as hmle_loglik_multi, for the last attempt of each task;
 *  retry       may be NULL; per task: the retries spent and the options of
 *              the attempt that produced ll (the tree's own when retries =
 *              0).
 * Errors: INVALID_ARG (max_retries outside 0..8), and as hmle_loglik_multi. */
typedef struct {
  int32_t retries;   /* retries spent on this task */
  int32_t max_rank;  /* rank capacity of the attempt that produced ll */
  int32_t precision; /* its hmle_precision */
  double aca_eps;    /* its accuracy */
} hmle_retry_info;
hmle_status hmle_loglik_multi_retry(hmle_ctx *ctx, const hmle_task *tasks, int32_t ntask,
                                    int32_t concurrency, int32_t max_retries, double *ll,
                                    int32_t *status, hmle_retry_info *retry);

/* a15: autotuner of the batched form (project-written; the paper has no
 * counterpart).  For this point set (locs n x d, row-major, host or device)
 * and theta it builds trees with leaf sizes 32, 64 and 128 (the tile of the
 * leaf sweep; other options from base) and times hmle_loglik_batch at
 * concurrency 1, 2, 4, ... up to max_concurrency (0 means 16), stopping a
 * leaf size once doubling the concurrency gains less than 5 %; at each
 * concurrency c it tries the batch sizes (evaluations per launch) c, c / 2
 * and c / 4 (at least 1).  Each trial is one warm-up batch (buffers, graph
 * capture) and one timed batch.
 *  best    the fastest (leaf_size, concurrency, batch_size, evals_per_s);
 *          best->trials = number of trials run.
 *  trials  if not NULL, up to max_trials trial results in run order;
 *          *ntrials (may be NULL) receives the number run.
 * The trees are destroyed before returning.  Errors: INVALID_ARG, OOM,
 * CUDA, or the first evaluation error if no trial succeeded. */
typedef struct {
  int32_t leaf_size;
  int32_t concurrency;
  double evals_per_s;
  int32_t trials;
  int32_t batch_size;
} hmle_tune_result;

/* a15: set the evaluations per launch (opts.batch_size, 1..64) of a tree's
 * later hmle_loglik_batch calls.  Errors: INVALID_ARG. */
hmle_status hmle_tree_set_batch_size(hmle_tree *tree, int32_t batch_size);
hmle_status hmle_autotune(hmle_ctx *ctx, const double *locs, int64_t n, int32_t d,
                          const hmle_opts *base, const hmle_theta *theta, const double *Z,
                          int32_t max_concurrency, hmle_tune_result *best,
                          hmle_tune_result *trials, int32_t max_trials, int32_t *ntrials);

/* a13 (Sec. 2 and Sec. 5): maximise L over theta by Nelder-Mead in the
 * transformed coordinates sigma = 2/1.1^s0, ell = 1/1.5^l0, nu = 1/1.2^n0,
 * tau = 1/2^t0.  Trial points outside the admissible range of theta, or
 * whose evaluation fails with NOT_SPD, RANK_OVERFLOW or NOT_CONVERGED (the
 * mixed form's PCG), score L = -inf.
 * The candidates of one iteration (reflection, expansion, contractions) are
 * evaluated together as one batch.
 *  theta0     start point; fopts may be NULL for hmle_fit_opts_default.
 *  theta_hat  best point found; loglik_hat its L; n_iter / n_evals may be NULL.
 * Returns HMLE_OK on convergence, HMLE_ERR_NOT_CONVERGED when max_iter was
 * reached (theta_hat is still the best point seen), or the first hard error. */
hmle_status hmle_fit(hmle_ctx *ctx, const hmle_tree *tree, const double *Z,
                     const hmle_theta *theta0, const hmle_fit_opts *fopts,
                     hmle_theta *theta_hat, double *loglik_hat,
                     int32_t *n_iter, int32_t *n_evals);

/* The optimiser of hmle_fit and hmle_fit_profiled (Sec. 2, maximisation of
 * the log-likelihood; Nelder-Mead with reflection 1, expansion 2,
 * contraction 1/2, shrink 1/2) on a caller's objective, on the host: it
 * minimises f over dim coordinates (1 <= dim <= 8) from x0 with initial
 * simplex steps step (dim values, NULL = 1 each).  fopts as hmle_fit (its
 * step field is not used; NULL = hmle_fit_opts_default).  f(x, dim, user)
 * may return +inf where it is undefined; NaN counts as +inf.  Each
 * iteration asks f for all four candidates (reflection, expansion, outside
 * and inside contraction) before the acceptance rules choose, as hmle_fit
 * evaluates them as one batch; *n_evals counts the values the rules use.
 * x_best (dim values) and *f_best receive the best vertex.
 * Returns HMLE_OK when the tolerance was met, HMLE_ERR_NOT_CONVERGED after
 * max_iter iterations, INVALID_ARG for a bad dim, NULL or non-finite x0 /
 * step. */
typedef double (*hmle_objective)(const double *x, int32_t dim, void *user);
hmle_status hmle_nelder_mead(int32_t dim, hmle_objective f, void *user, const double *x0,
                             const double *step, const hmle_fit_opts *fopts, double *x_best,
                             double *f_best, int32_t *n_iter, int32_t *n_evals);

/* Field simulation (the test-data generator of the large workloads): factor
 * C~(theta) and return Z = P^T L~ P xi, a sample of the zero-mean field with
 * covariance C~ (Eq. 1's model, Sec. 1), where xi is white noise.
 *  xi, Z  n doubles each in the caller's point order, host or device.
 * Errors: as hmle_assemble and hmle_factor. */
hmle_status hmle_simulate(hmle_ctx *ctx, const hmle_tree *tree, const hmle_theta *theta,
                          const double *xi, double *Z);

/* Matern correlation M_nu(x) = x^nu K_nu(x) / (2^(nu-1) Gamma(nu)) of Eq. 2
 * as the device evaluates it (Chebyshev tables built per nu from the
 * integral representation of K_nu), for x >= 0; out[i] for x[i], host or
 * device arrays of m doubles.  A check of the device Bessel kernel. */
hmle_status hmle_matern_eval(hmle_ctx *ctx, double nu, const double *x,
                             int64_t m, double *out);

/* hmle_matern_eval without any device allocation, for callers that cannot
 * allocate: a host application that owns the device memory and gives this
 * library a fixed budget it must not grow, or code in a section where
 * cudaMalloc is not allowed (it may synchronise the device, and it is
 * refused while a stream is being captured).  The paper has no counterpart;
 * this is an interface convenience.
 *  nus  nnu values of nu (host array), 1 <= nnu <= 16: the per-nu tables
 *       live in a static device array sized for 16 of them (about 60 KB per
 *       device, held until the process exits); more is INVALID_ARG.
 *  x    m doubles already in device memory; out: nnu * m doubles in device
 *       memory, out[j*m + i] = M_{nus[j]}(x[i]).  Host pointers are
 *       INVALID_ARG: nothing is staged or copied.
 * The work is enqueued on the context's stream and the call returns without
 * waiting: synchronise that stream before reading out.  Every call made
 * outside a stream capture looks up the static array's device address
 * (cudaGetSymbolAddress), so a reset of the device inside the process is
 * followed; a call made while the context's stream is being captured uses
 * the address of the last call outside a capture, so make the first call on
 * a device before any capture begins.  The context's device must be the current device,
 * else INVALID_ARG.  Every call shares the one array and overwrites it: calls
 * whose work overlaps on the GPU (other streams, other contexts) race, and
 * must be serialised.  Errors go to hmle_last_error like every entry point. */
hmle_status hmle_matern_eval_noalloc(hmle_ctx *ctx, const double *nus, int32_t nnu,
                                     const double *x, int64_t m, double *out);

/* The positivity transform of Sec. 5 (the coordinates hmle_fit searches):
 * sigma = 2 / 1.1^x0, ell = 1 / 1.5^x1, nu = 1 / 1.2^x2, tau = 1 / 2^x3, with
 * sigma2 = sigma^2, tau2 = tau^2.  hmle_theta_to_x needs sigma2, tau2 > 0;
 * hmle_x_to_theta rejects non-finite x or a theta out of range.
 * Errors: INVALID_ARG. */
hmle_status hmle_theta_to_x(const hmle_theta *theta, double x[4]);
hmle_status hmle_x_to_theta(const double x[4], hmle_theta *theta);

/* a16 (learned start; Sec. 7 suggests precomputing the initial guess of the
 * optimiser).  A 35-256-256-256-8 perceptron (tanh) maps field statistics
 * to an initial theta (4 transformed coordinates of Sec. 5) and log initial
 * simplex steps (4), trained on the GPU with hand-written kernels on fields
 * simulated by hmle_simulate.  Its matrix products (forward, deltas, weight
 * gradients) run on the tensor cores with BF16 weights and activations and
 * FP32 accumulation; the master weights, biases, loss and Adam are FP32.
 * Parameters: W1 (256 x 35, row-major), b1, W2 (256 x 256), b2, W3, b3,
 * W4 (8 x 256), b4 -- 142856 floats.  The forward, gradient and training
 * calls also return TIMEOUT if a bounded wait of the tensor cores ran out.
 *
 * hmle_features: the 35 inputs for one field.  locs n x d row-major and Z
 * (n, caller order), host or device.  On m = min(n, 4096) points at caller
 * indices floor(i n / m): the empirical semivariogram in 32 bins of squared
 * distance h^2 (bin k: S 2^(k-32) <= h^2 < S 2^(k-31); below bin 1 -> bin 0;
 * h^2 = S -> bin 31; S = squared bounding-box diagonal of the sample):
 * feat[k] = log of the bin's mean of (Z_i - Z_j)^2 / 2 (an empty bin copies
 * the nearest non-empty bin above it, else below); feat[32] = log n,
 * feat[33] = d, feat[34] = log sqrt(S).  feat: 35 floats, host.
 * Errors: INVALID_ARG, OOM, CUDA. */
hmle_status hmle_features(hmle_ctx *ctx, const double *locs, int64_t n, int32_t d, const double *Z,
                          float *feat);

/* The perceptron.  Parameters: one flat FP32 array of hmle_mlp_nparams()
 * values: W1 (64 x 35, row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (8 x 64),
 * b3 (8); inputs are standardised with per-feature mu / sd (35 each) before
 * the first layer.  Outputs per field (8): mu_1..4 (transformed theta) and
 * s_1..4 (log steps).  Training minimises the batch mean of the Gaussian
 * negative log-likelihood sum_c [exp(-2 s_c) (t_c - mu_c)^2 / 2 + s_c] by Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8).  Every reduction is in a fixed order.
 *  create   weights uniform in +-1/sqrt(fan_in) from a counter-based
 *           generator seeded by `seed`, zero biases, mu = 0, sd = 1.
 *  set/get  parameters (host or device, may be NULL), mu, sd (host, may be
 *           NULL); set resets the Adam state.
 *  forward  m fields: feats m x 35 (host or device) -> out m x 8.
 *  grad     gradient of the batch loss at feats / targets (m x 4) -> grad
 *           (nparams), *loss = batch mean loss (either may be NULL).
 *  adam_step  one Adam update with a given gradient (host or device).
 *  train    sets mu / sd from feats, then `epochs` passes over the data in
 *           minibatches of `batch` (a seeded deterministic shuffle per
 *           epoch, remainder dropped) with learning rate lr; *loss_first /
 *           *loss_last = mean loss of the first / last epoch (may be NULL).
 * Errors: INVALID_ARG, OOM, CUDA. */
typedef struct hmle_mlp hmle_mlp;
int32_t hmle_mlp_nparams(void);
hmle_status hmle_mlp_create(hmle_ctx *ctx, uint64_t seed, hmle_mlp **out);
void hmle_mlp_destroy(hmle_mlp *mlp);
hmle_status hmle_mlp_set(hmle_ctx *ctx, hmle_mlp *mlp, const float *params, const float *mu,
                         const float *sd);
hmle_status hmle_mlp_get(hmle_ctx *ctx, const hmle_mlp *mlp, float *params, float *mu, float *sd);
hmle_status hmle_mlp_forward(hmle_ctx *ctx, const hmle_mlp *mlp, const float *feats, int32_t m,
                             float *out);
hmle_status hmle_mlp_grad(hmle_ctx *ctx, const hmle_mlp *mlp, const float *feats,
                          const float *targets, int32_t m, float *grad, float *loss);
hmle_status hmle_mlp_adam_step(hmle_ctx *ctx, hmle_mlp *mlp, const float *grad, float lr);
hmle_status hmle_mlp_train(hmle_ctx *ctx, hmle_mlp *mlp, const float *feats, const float *targets,
                           int32_t m, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                           float *loss_first, float *loss_last);

/* Failure-detection self-test of the bounded device waits (no counterpart in
 * the paper).  The persistent sweeps of the solves synchronise their CTAs with
 * a grid barrier whose waits are bounded; a wait that runs out sets an error
 * word, every CTA leaves, and the call reports HMLE_ERR_TIMEOUT with the
 * context still usable.  This runs one such barrier: extra = 0 (every CTA
 * arrives) returns HMLE_OK; extra = 1 expects one more arrival than there are
 * CTAs, so the wait must run out (after about a quarter of a second) and the
 * call returns HMLE_ERR_TIMEOUT.  *err_word (may be NULL) receives the error
 * word.  Errors: INVALID_ARG (extra not 0 or 1), OOM, CUDA. */
hmle_status hmle_selftest_barrier(hmle_ctx *ctx, int32_t extra, uint32_t *err_word);

/* Check of the tensor-core tile product of the mixed forms (no counterpart in
 * the paper; the products it serves are the Schur-complement updates of the
 * H-Cholesky factorisation, Sec. 2).  C = A B with every operand value split
 * into nslices BF16 slices (1, 2 or 3; a = a_0 + a_1 + ..., a_p the BF16
 * rounding of what the earlier slices leave of the FP32 rounding of a) and
 * the products a_p b_q with p + q < nslices accumulated in FP32 in tensor
 * memory (tcgen05.mma).  A: M x K row-major, B: K x N row-major (host
 * doubles); C: copies x (M x N column-major) host doubles, one copy per CTA
 * (copies CTAs run concurrently and must agree).  a_kfast / b_kfast select the
 * staging order of the operand (the order in which threads gather it), not
 * its layout: the result is the same.  1 <= M, N; 0 <= K; 1 <= copies <= 4096;
 * each array at most 2^28 values.  Errors: INVALID_ARG, OOM, CUDA; TIMEOUT if
 * a bounded wait for the tensor cores ran out. */
hmle_status hmle_selftest_tc_gemm(hmle_ctx *ctx, int32_t nslices, int32_t a_kfast, int32_t b_kfast,
                                  int32_t copies, int32_t M, int32_t N, int32_t K, const double *A,
                                  const double *B, double *C);

/* Measurement support (no counterpart in the paper).  Select one kernel of
 * the factorisation sweep by name (e.g. "k_tsqr_final", "k_dense_pair"; NULL
 * switches timing off).  While selected, every launch of that kernel is
 * bracketed by CUDA events on its own stream, and after each evaluation the
 * algorithmic FP64 flops of those launches are tallied from the plan and the
 * ranks the evaluation produced.  Selecting resets the counters.
 * Errors: INVALID_ARG for an unknown name. */
hmle_status hmle_profile_select(hmle_ctx *ctx, const char *kernel);
/* Measurement support (no counterpart in the paper): totals since the last
 * hmle_profile_select: summed launch durations (ms), number of launches,
 * algorithmic FP64 flops.  Any pointer may be NULL.  Errors: INVALID_ARG. */
hmle_status hmle_profile_read(hmle_ctx *ctx, double *ms, int64_t *launches, double *flops);

/* Measurement support (no counterpart in the paper): the algorithmic work of
 * the two phases outside the factorisation sweep, for the factor f and the
 * ranks its assembly and factorisation produced (Sec. 2, storage and
 * complexity of the H-matrix):
 *  asm_flops    FP64 flops of assembling C~ (a3, a4): every dense block's
 *               m x p entries, and for an admissible block of ACA rank k
 *               the k rows and columns the cross approximation generates,
 *               (m + p)(k e + k (k - 1)) with the residual updates; e =
 *               3 d + 68 flops per Matern entry (distance, scaling, the
 *               degree-20 Clenshaw recurrence of the table, sigma^2);
 *  solve_bytes  bytes of the factor that one forward and one backward sweep
 *               (hmle_solve) must read: the lower triangle of each diagonal
 *               leaf block, every entry of the other dense blocks, and U and
 *               W of each low-rank block at its rank, 8 bytes per double,
 *               twice; the vectors' own traffic is not counted.
 * Either pointer may be NULL.  Errors: INVALID_ARG, CUDA. */
hmle_status hmle_phase_work(hmle_ctx *ctx, const hmle_hfactor *f, double *asm_flops,
                            double *solve_bytes);

/* Host-only inspection of the factorisation schedule (no device work, no
 * counterpart in the paper; for checking the planner and for tools).
 * hmle_plan_build builds the θ-independent task lists of the left-looking
 * leaf sweep (Sec. 2, H-Cholesky) for a given block partition, as
 * hmle_build_tree does after its device trees:
 *  n, d        points and dimension; the clusters are the halving of the
 *              point range in cluster order down to leaves of at most
 *              leaf_size points (depth = smallest with ceil(n / 2^depth) <=
 *              leaf_size; cluster h of level l is heap entry 2^l - 1 + h and
 *              splits at b + (e - b) / 2).
 *  blocks      nblocks records of 4 int32 (level, i, j, kind): the block of
 *              row cluster i and column cluster j of that level, j <= i;
 *              kind 0 = dense (leaf level only), 1 = low-rank (i > j).  They
 *              must tile the lower triangle, the diagonal leaf blocks
 *              included, as the device block tree does.
 *  max_rank, oversample  as in hmle_opts.
 * Errors: INVALID_ARG (sizes, options, a record out of range, or a
 * partition the planner rejects), OOM.
 *
 * hmle_plan_list copies one of the planner's lists as records of int64
 * fields: *nrec records of *width fields each (either may be NULL).  With out
 * = NULL only the sizes are returned; else cap (int64 slots) must hold
 * nrec * width.  Indices are into the plan's own lists; offsets are in
 * doubles.  Fields by list:
 *  SCALARS    n, d, b, depth, nleaf, kcap, kc, r, rhs_panel, ws_max,
 *             dense_words, uc_words, u_words, w_words
 *  BLOCKS     kind, level, rbeg, rend, cbeg, cend, rleaf, cleaf, off_d,
 *             off_uc, off_vc, off_u, panel, slot  (sorted by first column
 *             leaf, dense before low-rank, then row leaf)
 *  STEPS      per leaf K: gram0, gram1, gch0, gch1, gred0, gred1, lrt0, lrt1,
 *             aent0, aent1, bent0, bent1, arow0, arow1, brow0, brow1, dns0,
 *             dns1, wpan0, wpan1, ht0, ht1, ur0, ur1, dpws, ws_words
 *  LRT        low-rank targets: blk, m, p, a0, a1, b0, b1, yoff, zoff, soff,
 *             tcoff, gm, gp, roff
 *  AENT/BENT  blocks covering a target's rows / columns left of it: target,
 *             blk, toff, soff, p0, p1 (range in APAIR / BPAIR)
 *  LRPAIRS    ae, be, goff (-1 unless both blocks are low-rank)
 *  DNS        dense targets (diagonal first per step): blk, p0, p1
 *  DPAIRS     a, b, goff
 *  PANELS     W-panels (the last is the right-hand side): rbeg, rend, width,
 *             leaf0, off
 *  WPAN       panel ids solved per step (ranges wpan0..wpan1)
 *  HTS        deferred-update products: a, panel, hoff
 *  UROWS      deferred-update rows: panel, leaf, e0, e1 (range in UENTS)
 *  UENTS      a, hoff (-1 for a dense block)
 *  GRAMS      a, b, ovb, ove, goff;  GCHUNKS  g, r0, r1, out;
 *  GREDS      g, nchunk, poff
 *  AROW/BROW  row tasks of the samples Y / Z: target, leaf, e0, e1 (range in
 *             AROW_ENT / BROW_ENT, which hold AENT / BENT indices)
 *  *_RHS, HT_RHS0, UR_RHS0  the right-hand-side panel's share of HTS /
 *             UROWS / UENTS and its per-step ranges (nleaf + 1 entries)
 *  BH_BLOCKS, BH0, BUPD, BENTS, BUPD0  the backward sweep's lists: low-rank
 *             blocks whose rows start at leaf K, per column leaf the entries
 *             to push, and their per-step ranges
 *  MV_ROW0, MV_BLOCKS    per leaf row, the blocks of L covering it (diagonal
 *             first);  MVT_ROW0, MVT_BLOCKS  per leaf, the off-diagonal
 *             blocks whose columns cover it.
 * Errors: INVALID_ARG (unknown list, cap too small). */
typedef enum {
  HMLE_PLAN_SCALARS = 0, HMLE_PLAN_BLOCKS, HMLE_PLAN_STEPS, HMLE_PLAN_LRT, HMLE_PLAN_AENT,
  HMLE_PLAN_BENT, HMLE_PLAN_LRPAIRS, HMLE_PLAN_DNS, HMLE_PLAN_DPAIRS, HMLE_PLAN_PANELS,
  HMLE_PLAN_WPAN, HMLE_PLAN_HTS, HMLE_PLAN_UROWS, HMLE_PLAN_UENTS, HMLE_PLAN_GRAMS,
  HMLE_PLAN_GCHUNKS, HMLE_PLAN_GREDS, HMLE_PLAN_AROW, HMLE_PLAN_BROW, HMLE_PLAN_AROW_ENT,
  HMLE_PLAN_BROW_ENT, HMLE_PLAN_APAIR, HMLE_PLAN_BPAIR, HMLE_PLAN_HTS_RHS,
  HMLE_PLAN_UROWS_RHS, HMLE_PLAN_UENTS_RHS, HMLE_PLAN_HT_RHS0, HMLE_PLAN_UR_RHS0,
  HMLE_PLAN_BH_BLOCKS, HMLE_PLAN_BH0, HMLE_PLAN_BUPD, HMLE_PLAN_BENTS, HMLE_PLAN_BUPD0,
  HMLE_PLAN_MV_ROW0, HMLE_PLAN_MV_BLOCKS, HMLE_PLAN_MVT_ROW0, HMLE_PLAN_MVT_BLOCKS
} hmle_plan_list_id;
typedef struct hmle_plan hmle_plan;
hmle_status hmle_plan_build(int64_t n, int32_t d, int32_t leaf_size, const int32_t *blocks,
                            int32_t nblocks, int32_t max_rank, int32_t oversample,
                            hmle_plan **out);
void hmle_plan_destroy(hmle_plan *plan);
hmle_status hmle_plan_list(const hmle_plan *plan, int32_t which, int64_t *out, int64_t cap,
                           int64_t *nrec, int32_t *width);

#ifdef __cplusplus
}
#endif
#endif /* HMLE_H */
