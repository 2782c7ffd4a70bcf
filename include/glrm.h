/*
 * glrm.h -- C ABI of libglrm, a GB300 (sm_103a) CUDA library for the
 * alternating proximal-gradient fit of a generalized low rank model (GLRM),
 * Udell, Horn, Zadeh, Boyd, "Generalized Low Rank Models" (arXiv 1410.0342).
 *
 * The model (eq. gpca, Section 4; eq. apca, Section 5):
 *
 *     minimize  sum_{(i,j) in Omega} L_j(x_i . y_j, A_ij)
 *               + sum_i r(x_i) + sum_j rt(y_j)
 *
 * over X (m x k, row x_i) and Y (k x n, column y_j).  Throughout this ABI Y
 * is passed and stored as its transpose Yt (n x k, row j = y_j), so that both
 * factors are row-major with k contiguous values per row or column.
 *
 * Conventions shared by every entry point
 *  - Pointers named *_dev are device pointers (cudaMalloc'd or equivalent),
 *    pointers named *_host are host pointers; the caller owns both.  Device
 *    pointers must be aligned to their element size; 16-byte alignment lets
 *    the kernels use vector loads.
 *  - Element type of values and factors: double for GLRM_FP64, float for
 *    GLRM_FP32 and GLRM_BF16.  The BF16 form keeps FP32 factors; its gradient
 *    passes gather the other factor's rows from a BF16 copy (products of
 *    BF16 rows with FP32 accumulation, loss derivatives in FP32), except for a
 *    row (column) whose previous step was rejected, which takes its retry's
 *    gradient from the FP32 rows; candidates are evaluated on the FP32 rows,
 *    so the accept / reject test and the objectives a sweep reports are
 *    exactly those of the FP32 form.  glrm_grad_at of a BF16 model reads
 *    BF16 copies of both factors.
 *  - All work is enqueued on the stream given to glrm_create, in order.  An
 *    entry point returns once its work is enqueued unless it says it
 *    synchronises (it must when it hands a result back in host memory).
 *  - Every entry point returns a glrm_status.  Nothing throws across the ABI.
 *    On error, glrm_last_error(h) gives a message; the handle stays usable
 *    unless the error is GLRM_ERR_CUDA from a failed kernel, after which the
 *    CUDA context itself is in error.
 *  - A handle is not thread-safe: one host thread at a time.
 */
#ifndef GLRM_H
#define GLRM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct glrm_s *glrm_t;

typedef enum {
    GLRM_OK = 0,
    GLRM_ERR_ARG = -1,       /* bad argument (null pointer, size, kind) */
    GLRM_ERR_RANGE = -2,     /* a size beyond the library's limits */
    GLRM_ERR_OMEGA = -3,     /* the observed set failed validation */
    GLRM_ERR_NONFINITE = -4, /* NaN or Inf in data */
    GLRM_ERR_CUDA = -5,      /* a CUDA runtime call failed */
    GLRM_ERR_TIMEOUT = -6,   /* a device-side wait hit its iteration limit */
    GLRM_ERR_STATE = -7,     /* call out of order (e.g. sweep before set_observed) */
    GLRM_ERR_NOMEM = -8      /* device allocation failed */
} glrm_status;

/* Per-column loss L_j(u, a).
 *   GLRM_LOSS_QUAD      (u - a)^2                                    eq. qpca, Sec. 2.1
 *   GLRM_LOSS_HUBER     huber_delta(u - a), delta = param:
 *                       0.5 x^2 if |x| <= delta, else delta (|x| - delta/2);
 *                       delta = 1 is the paper's Huber function      Sec. 4.3
 *   GLRM_LOSS_HINGE     (1 - a u)_+ with a in {-1, +1}                Sec. 5.2
 *   GLRM_LOSS_LOGISTIC  log(1 + exp(-a u)) with a in {-1, +1}         Sec. 5.2
 *   GLRM_LOSS_ORDINAL_HINGE
 *                       sum_{a'<a} (1 - u + a')_+ + sum_{a'>a, a'<=d} (1 + u - a')_+
 *                       with a in {1..d}, d = levels                 eq. ord-pca
 *   GLRM_LOSS_L1        |a - u|                                      Sec. 4.2, robust PCA
 *   GLRM_LOSS_QUANTILE  alpha (a - u)_+ + (1 - alpha) (u - a)_+, alpha = param
 *                       in (0, 1)                                   Sec. 4.2, quantile PCA
 * At a kink the derivative of the kinked term is taken as 0.  The batched
 * form takes kinds 0 .. 4. */
typedef enum {
    GLRM_LOSS_QUAD = 0,
    GLRM_LOSS_HUBER = 1,
    GLRM_LOSS_HINGE = 2,
    GLRM_LOSS_LOGISTIC = 3,
    GLRM_LOSS_ORDINAL_HINGE = 4,
    GLRM_LOSS_L1 = 5,
    GLRM_LOSS_QUANTILE = 6
} glrm_loss_kind;

/* Row / column regulariser r(x) with weight w.
 *   GLRM_REG_ZERO    0
 *   GLRM_REG_QUAD    w ||x||_2^2                      eq. qpca
 *   GLRM_REG_L1      w ||x||_1                        Sec. 3.2, sparse PCA
 *   GLRM_REG_NONNEG  indicator of x >= 0 (0 or +inf)   Sec. 3.2, NNMF
 * Their proximal operators (Sec. 7.2) are z/(1+2 alpha w), soft
 * thresholding at alpha w, max(z, 0) and the identity. */
typedef enum {
    GLRM_REG_ZERO = 0,
    GLRM_REG_QUAD = 1,
    GLRM_REG_L1 = 2,
    GLRM_REG_NONNEG = 3
} glrm_reg_kind;

typedef enum { GLRM_FP64 = 0, GLRM_FP32 = 1, GLRM_BF16 = 2 } glrm_precision;

typedef struct {
    int32_t kind;   /* glrm_loss_kind */
    int32_t levels; /* ordinal level count d >= 2; ignored otherwise */
    double param;   /* Huber delta or quantile alpha; ignored otherwise */
} glrm_loss;

/* Limits: 1 <= k <= 64; m, n >= 1; m, n, nnz < 2^31. */

/* Create a model of m rows, n columns and rank k.
 * col_loss_host: n loss descriptors, copied.  rx / ry: regulariser kind and
 * weight for the rows of X and the columns of Y (used in the model's element
 * type, so FP64 models see the weights exactly).  precision: glrm_precision.
 * stream: a cudaStream_t (NULL = legacy default stream) on which every later
 * call enqueues its work.  Allocates the factors (zero) and step sizes on the
 * current CUDA device.  Section 4 (eq. gpca) defines the model. */
int glrm_create(int64_t m, int64_t n, int32_t k, const glrm_loss *col_loss_host,
                int32_t rx_kind, double rx_weight, int32_t ry_kind, double ry_weight,
                int32_t precision, void *stream, glrm_t *out);

/* Give the model its observed set Omega (Section 2.5; Section 5) in both
 * orientations: CSR (rowptr m+1, colidx nnz, val nnz; row i's entries at
 * rowptr[i]..rowptr[i+1]-1, columns strictly ascending) and CSC (colptr n+1,
 * rowidx nnz, val nnz; rows strictly ascending).  Device pointers; values in
 * the model's element type.  The library copies and re-tiles everything into
 * buffers it owns (the caller may free its copies afterwards), validates it
 * on the device -- pointer monotonicity, index range, no duplicate (i,j),
 * CSR/CSC describing the same entries with bit-identical values (compared
 * through 64-bit digests of the entries and of their values: a mismatch goes
 * unnoticed with probability about 2^-64), finite values, values inside each
 * column loss's domain -- and resets every step size to 1/max(count, 1) (Section 7.2,
 * "Choosing a step size").  Synchronises (it reads back the validation
 * result).  Returns GLRM_ERR_OMEGA or GLRM_ERR_NONFINITE when validation
 * fails; the previous Omega is then gone and sweeps return GLRM_ERR_STATE. */
int glrm_set_observed(glrm_t h, int64_t nnz, const int32_t *csr_rowptr_dev,
                      const int32_t *csr_colidx_dev, const void *csr_val_dev,
                      const int32_t *csc_colptr_dev, const int32_t *csc_rowidx_dev,
                      const void *csc_val_dev);

/* Same as glrm_set_observed with host pointers: the library copies them to
 * the device on its stream first (pinned host memory makes that faster).
 * Both calls copy the CSR arrays first and check them (and build what the
 * chosen path needs from them) on a second, non-blocking stream the handle
 * owns while the CSC arrays are still being copied; they return after both
 * streams are done. */
int glrm_set_observed_host(glrm_t h, int64_t nnz, const int32_t *csr_rowptr_host,
                           const int32_t *csr_colidx_host, const void *csr_val_host,
                           const int32_t *csc_colptr_host, const int32_t *csc_rowidx_host,
                           const void *csc_val_host);

/* Omega from its CSR arrays alone (device / host pointers, as above): the
 * CSR arrays are copied and validated as by glrm_set_observed, and the CSC
 * orientation is then built from them on the device by a stable counting
 * sort of the entries by column (rows ascending within each column; the
 * result does not depend on scheduling), so only half the bytes cross from
 * the host.  Allocates a count table of at most 2^26 int32 for the sort
 * (freed before returning).  Synchronises. */
int glrm_set_observed_csr(glrm_t h, int64_t nnz, const int32_t *csr_rowptr_dev, const int32_t *csr_colidx_dev,
                          const void *csr_val_dev);
int glrm_set_observed_csr_host(glrm_t h, int64_t nnz, const int32_t *csr_rowptr_host,
                               const int32_t *csr_colidx_host, const void *csr_val_host);

/* Give the model a fully observed table instead: Omega = every (i, j), the
 * data matrix of Section 2 with nothing missing.  A: m x n, row-major with
 * leading dimension lda >= n (elements), FP32 (GLRM_FP32 and GLRM_BF16
 * models; GLRM_ERR_ARG otherwise; GLRM_ERR_RANGE when k > 64).  The library copies A
 * into rows padded to a multiple of 4 floats, validates it like an observed
 * set (finite values, each column's values in its loss's domain) and resets
 * the step sizes to 1/n (rows) and 1/m (columns).  Sweeps, objectives and
 * gradients then run the dense form on the tensor cores: U = X Y, the loss
 * derivatives R and R Y^T, X^T R (the contractions of Section 7.2's
 * gradient) by tcgen05 MMAs on BF16 splits, FP32 accumulation: every value
 * split in three, x = hi + mid + lo, and six products summed (error about
 * 2^-25 of sum_c |x_c y_c|, FP32 quality); everything else in FP32.  A
 * GLRM_BF16 model takes the gradient contraction R Y^T (X^T R) as the single
 * product of R's and the factor's BF16 high parts (FP32 accumulation), with
 * U, the losses, derivatives, objectives and decisions at FP32 quality as
 * above.  glrm_als_sweep and
 * glrm_set_path return GLRM_ERR_STATE on a dense table; glrm_get_path reports
 * GLRM_PATH_DENSE.  Synchronises.  A later glrm_set_observed replaces the
 * table. */
int glrm_set_dense(glrm_t h, const void *A_dev, int64_t lda);
int glrm_set_dense_host(glrm_t h, const void *A_host, int64_t lda);

/* Copy factors in: X_dev (m x k) and Yt_dev (n x k), row-major, element type
 * of the model.  Either may be NULL to leave that factor unchanged.  Step
 * sizes are not touched (glrm_reset_steps resets them). */
int glrm_set_factors(glrm_t h, const void *X_dev, const void *Yt_dev);

/* Copy factors out (same layout); either pointer may be NULL. */
int glrm_get_factors(glrm_t h, void *X_dev, void *Yt_dev);

/* Host-pointer variants of the two calls above; they synchronise. */
int glrm_set_factors_host(glrm_t h, const void *X_host, const void *Yt_host);
int glrm_get_factors_host(glrm_t h, void *X_host, void *Yt_host);

/* Offset (Section 3.4, "Offsets and scaling"; the k+1 construction): with
 * on != 0 the last coordinate of every row of X is held at 1 (its
 * regulariser is the indicator of x_ik = 1, whose prox returns 1) and the
 * last coordinate of every column of Y is not regularised, so y_jk acts as a
 * per-column offset mu_j of x_i . y_j.  The other k-1 coordinates keep the
 * model's regulariser.  A row whose last coordinate is not 1 has objective
 * +inf until its next X-step, which sets it to 1 (the step is accepted: its
 * candidate's objective is finite).  Applies to glrm_sweep,
 * glrm_sweep_until, glrm_objective* and glrm_grad* on every path (the
 * regulariser gradient of the held coordinate is taken as 0);
 * glrm_als_sweep and glrm_proxprox_sweep return GLRM_ERR_ARG while it is on.
 * Takes effect for work enqueued afterwards; on = 0 turns it off. */
int glrm_set_offset(glrm_t h, int32_t on);

/* Column statistics of the automatic loss scaling (Section 4.3, "Offsets and
 * scaling"): for each column j with c_j >= 1 observed entries a_e,
 *   mu_dev[j]     = the smallest minimiser of S_j(mu) = sum_e L_j(mu, a_e)
 *                   (the mean for quadratic loss, the lower median for l1,
 *                   the alpha-quantile for quantile loss),
 *   sigma2_dev[j] = S_j(mu_j) / (c_j - 1)   (the sample variance for
 *                   quadratic loss; NaN when c_j < 2),
 * both NaN for an empty column.  mu_j is found by bisection on the sign of
 * the FP64 sum of L_j'(mu, a_e) in [min a - 32, max a + 32], to 2^-62 of that
 * width; where S_j has no minimiser (a hinge or logistic column of one
 * label) mu_j is the bracket end it decreases towards.  Device pointers, n
 * doubles each, written on the handle's stream (returns once enqueued).
 * Reads the observed set (or the dense table). */
int glrm_column_stats(glrm_t h, double *mu_dev, double *sigma2_dev);

/* Per-column loss weights (the scaled losses of Section 4.3): with
 * w_host != NULL (n finite doubles > 0, copied) column j's loss becomes
 * w_j L_j everywhere (sweeps, objective, gradients); w_j = 1 / sigma2_j
 * gives the paper's standardised GLRM.  NULL removes them.  Weighted models
 * run on the dense form when the table is held densely (a fully observed
 * table, or an observed set on the dense path), else every half-step on the
 * chunked path (glrm_get_path reports GLRM_PATH_CHUNKED).  GLRM_BF16 models
 * return GLRM_ERR_ARG, as do glrm_als_sweep and glrm_proxprox_sweep on a
 * weighted model.  Synchronises. */
int glrm_set_column_scale(glrm_t h, const double *w_host);

/* Change the regulariser weights (kinds stay).  Takes effect for work
 * enqueued afterwards; step sizes are not touched. */
int glrm_set_reg_weights(glrm_t h, double rx_weight, double ry_weight);

/* Global optimality certificate (Section 7.6, eq. convex-certificate) of the
 * current factors, for a model whose regulariser is w (||X||^2 + ||Y||^2)
 * (both GLRM_REG_QUAD with one weight w > 0; no offset):
 *     *norm_host = || (1/gamma) G + U V^T ||_2,   gamma = 2 w,
 * G (m x n, zero off Omega) holding w_j L_j'(x_i . y_j, A_ij) (0 at a kink;
 * column weights included) and U V^T the product of the singular vectors of
 * Z = X Y with singular values above 1e-10 of the largest (singular values
 * of X or Y below 1e-7 of their largest count as zero: they are found from
 * the k x k Gram matrices).  gamma = 2 w because ||Z||_* is the infimum of
 * (||X||^2 + ||Y||^2) / 2 over X Y = Z.  A value <= 1 certifies that
 * (X, Y) solves the rank-constrained problem globally when the loss is
 * convex and differentiable (for a nondifferentiable loss a value > 1 does
 * not prove the opposite).  The 2-norm is estimated by power iteration on
 * M^T M (FP64, a deterministic start vector) until the estimate changes by
 * at most tol relative, or max_iters iterations (*iters_host, if not NULL,
 * receives the count); the estimate approaches the norm from below.
 * Sparse observed sets only (GLRM_ERR_STATE for glrm_set_dense tables).
 * Allocates O(nnz + m + n) FP64 scratch.  Synchronises. */
int glrm_certificate(glrm_t h, int32_t max_iters, double tol, double *norm_host, int32_t *iters_host);

/* Regularisation path by homotopy (Section 8.1, "Regularization paths"):
 * for t = 0 .. nvals-1 set both regulariser weights to gamma_host[t] (in the
 * order given, normally decreasing), reset the step sizes
 * (glrm_reset_steps), sweep from the current factors until
 * glrm_sweep_until(max_sweeps, rtol, no reference, window) stops, and
 * record the objective (objective_host[t]), the sweeps run (sweeps_host[t])
 * and, with cert_host not NULL, glrm_certificate(cert_iters, 1e-10)
 * (cert_host[t]).  The factors of the last weight remain in the handle.
 * Synchronises. */
int glrm_regularization_path(glrm_t h, int32_t nvals, const double *gamma_host, int32_t max_sweeps, double rtol,
                             int32_t window, double *objective_host, int32_t *sweeps_host, double *cert_host,
                             int32_t cert_iters);

/* SVD initialisation of the factors (Section 7.5).  With k' = k - 1 when
 * the offset is on (glrm_set_offset), else k: the column statistics mu_j,
 * sigma2_j of glrm_column_stats; the scaled table
 *     A~_ij = m / (sigma_j m_j) (A_ij - mu_j) on Omega, 0 elsewhere
 * (m_j = column j's observation count; a column without a finite
 * sigma_j > 0 scales to 0 and takes sigma_j = 1 below); its top k' singular
 * triples U S V^T by the randomized range finder (Section 7.5 names Halko et
 * al.): a pseudo-random n x (k' + oversample) block from `seed` (at most 96
 * columns), power_iters rounds of A~^T / A~ products each followed by an
 * orthonormalisation (FP64 Gram eigendecomposition), then the eigenvectors
 * of B B^T for B = Q^T A~; and
 *     X = U S^1/2,   Y = S^1/2 V^T diag(sigma)
 * written into the model's factors, with X's column k-1 set to 1 and Y's
 * row k-1 to mu_j (0 for an empty column) when the offset is on.
 * singular_values_host (k' doubles, may be NULL) receives S.  Step sizes are
 * not touched.  Sparse observed sets only.  Allocates FP64 scratch of
 * O(nnz + (m + n)(k' + oversample)).  Synchronises. */
int glrm_svd_init(glrm_t h, int32_t oversample, int32_t power_iters, uint64_t seed, double *singular_values_host);

/* ---- Tables of multi-dimensional features (Section 6, eq. mpca) ----------
 * Feature j of such a table is represented by a block Y_j of d_j columns of
 * Y and entry (i, j) costs L_j(x_i Y_j, A_ij):
 *   GLRM_FEATURE_SCALAR       d_j = 1, any glrm_loss;
 *   GLRM_FEATURE_CATEGORICAL  labels 1..levels, d_j = levels, the one-vs-all
 *       loss (1 - u_a)_+ + sum_{a' != a} (1 + u_a')_+ ("Categorical PCA");
 *   GLRM_FEATURE_ORDINAL      levels 1..levels, d_j = levels - 1, the loss
 *       sum_{l < levels} (1 - s_l u_l)_+ with s_l = +1 if a > l, else -1
 *       (eq. ord-mpca, its indicator read as this sign).
 * Both block losses are sums of one hinge term (1 - b_l u_l)_+ per column of
 * the block (b_l = +1 for the label's column and -1 elsewhere; b_l = s_l),
 * so a feature table is fitted as the scalar table whose entry (i, j) becomes
 * the d_j entries (i, first_j + l, b_l) with hinge loss (first_j = sum of
 * the widths before j): glrm_embed_size / glrm_embed_features build that
 * table, glrm_embed_losses its column losses, and a model of n = sum d_j
 * columns created with them runs every sweep, path and form of the library
 * unchanged (its Y-step updates the block's columns one by one, each with
 * its own step size; the step sizes start at 1 / max(count, 1) over the
 * embedded entries).  glrm_decode_features imputes labels. */
typedef enum { GLRM_FEATURE_SCALAR = 0, GLRM_FEATURE_CATEGORICAL = 1, GLRM_FEATURE_ORDINAL = 2 } glrm_feature_kind;
#define GLRM_FEATURE_MAX_LEVELS 65536

typedef struct {
    int32_t kind;   /* glrm_feature_kind */
    int32_t levels; /* label / level count, 2..GLRM_FEATURE_MAX_LEVELS; ignored for scalar features */
} glrm_feature;

/* Column losses of the embedded table: out_host (sum d_j entries) receives
 * scalar_loss_host[j] at a scalar feature's column and GLRM_LOSS_HINGE at
 * every column of a block; *ncols_host (if not NULL) the width sum d_j.
 * out_host may be NULL to ask for the width only.  Host only. */
int glrm_embed_losses(int32_t nfeat, const glrm_feature *feat_host, const glrm_loss *scalar_loss_host,
                      glrm_loss *out_host, int64_t *ncols_host);

/* Width (sum d_j) and entry count of the embedded table, from the features'
 * column pointers colptr_dev (nfeat + 1, device).  Synchronises. */
int glrm_embed_size(int32_t nfeat, const glrm_feature *feat_host, const int32_t *colptr_dev, int64_t *ncols_host,
                    int64_t *nnz_host, void *stream);

/* Build the embedded table.  Input: the feature table in CSR (rowptr m+1,
 * featidx nnz, val nnz) and CSC (colptr nfeat+1, rowidx nnz, cval nnz)
 * forms, device pointers, values in the element type of `precision` (float
 * for GLRM_FP32 / GLRM_BF16, double for GLRM_FP64): real values for scalar
 * features, labels 1..levels (integral values) for block features.  Output,
 * caller-allocated device arrays (sizes from glrm_embed_size): CSR e_rowptr
 * (m+1), e_colidx, e_val and CSC e_colptr (sum d_j + 1), e_rowidx, e_cval,
 * ready for glrm_set_observed (rows stay in order within a column, and the
 * columns of a row ascend when its features do).  Temporary device memory is
 * allocated on `stream` and freed.  GLRM_ERR_OMEGA for inconsistent pointer
 * arrays, an index out of range or a label outside 1..levels.
 * Synchronises. */
int glrm_embed_features(int32_t nfeat, const glrm_feature *feat_host, int64_t m, int64_t nnz,
                        const int32_t *rowptr_dev, const int32_t *featidx_dev, const void *val_dev,
                        const int32_t *colptr_dev, const int32_t *rowidx_dev, const void *cval_dev,
                        int32_t precision, int32_t *e_rowptr_dev, int32_t *e_colidx_dev, void *e_val_dev,
                        int32_t *e_colptr_dev, int32_t *e_rowidx_dev, void *e_cval_dev, void *stream);

/* Impute cnt (row, feature) pairs of a model fitted on the embedded table
 * (h's n must equal sum d_j): u_l = x_i . y_{first_j + l} in the model's
 * precision; a scalar feature decodes as glrm_predict with decode on, a
 * categorical feature to argmax_l u_l (Section 6, "Categorical PCA"; the
 * lowest of equal maxima), an ordinal feature to argmin_a L(u, a) (Section
 * 5.3's rule; the lowest of equal minima, from the FP64 prefix sums of
 * (1 - u_l)_+ - (1 + u_l)_+).  out_dev: cnt values in the model's element
 * type; NaN for a pair out of range.  Synchronises. */
int glrm_decode_features(glrm_t h, int32_t nfeat, const glrm_feature *feat_host, int64_t cnt,
                         const int32_t *rows_dev, const int32_t *feats_dev, void *out_dev);

/* Reset every row step size to 1/max(n_i, 1) and every column step size to
 * 1/max(m_j, 1) (Section 7.2, "Choosing a step size", scale 1). */
int glrm_reset_steps(glrm_t h);

/* Run nsweeps alternating proximal-gradient sweeps (Algorithm 2 with the
 * proximal gradient update and the step-size rule of Section 7.2).  One
 * sweep updates every row x_i against the current Y, then every column y_j
 * against the new X.  Each row (column) update computes
 *     g = sum_{j in Omega_i} L_j'(x_i . y_j, A_ij) y_j,
 *     x+ = prox_{alpha_i r}(x_i - alpha_i g),
 * and keeps x+ (alpha_i *= 1.05) when its row objective
 * sum_j L_j(x . y_j, A_ij) + r(x) is not larger than at x_i, else keeps x_i
 * (alpha_i *= 0.7).  history_host, if not NULL, receives nsweeps doubles: the
 * objective of eq. gpca after each sweep (an FP64 reduction); the call then
 * synchronises.  With history_host NULL the call returns once enqueued. */
int glrm_sweep(glrm_t h, int32_t nsweeps, double *history_host);

/* Sweeps until a convergence test on the device passes (Section 7.2; the
 * objective of eq. gpca never increases under the step-size rule, so its
 * decrease is the natural stopping signal; the paper leaves the stopping
 * condition open).  After every sweep t the FP64 objective F_t is compared on
 * the GPU:
 *   f_ref is NaN:  stop when t >= window and
 *                  F_{t-window} - F_t <= window * rtol * |F_t|
 *                  (average relative decrease over the last `window` sweeps;
 *                  F_0 is the objective before the first sweep)
 *   otherwise:     stop when F_t - f_ref <= rtol |f_ref|   (within rtol of a
 *                  reference objective, e.g. a known optimum)
 * or after max_sweeps sweeps (>= 1).  rtol >= 0, window >= 1.  FP32 and FP64
 * models run the whole loop as one launch of a CUDA graph whose conditional
 * WHILE node repeats a captured sweep and its check (captured on the first
 * call and kept until the buffers or kernel paths change); the BF16 form,
 * which keeps host-side state between sweeps, reads the device's decision back
 * after each sweep.  *sweeps_host receives the number of sweeps run;
 * history_host, if not NULL, receives their objectives (max_sweeps doubles of
 * room).  Each sweep is exactly the sweep of glrm_sweep, so the results equal
 * those of glrm_sweep(h, *sweeps_host, ...).  Synchronises. */
int glrm_sweep_until(glrm_t h, int32_t max_sweeps, double rtol, double f_ref, int32_t window,
                     int32_t *sweeps_host, double *history_host);

/* Accepted row and column steps of the last sweep run (host, 2 values);
 * synchronises. */
int glrm_last_accepts(glrm_t h, int64_t *accepts_host);

/* Objective of eq. gpca at the model's factors, reduced in FP64; written to
 * out_host; synchronises. */
int glrm_objective(glrm_t h, double *out_host);

/* Objective of eq. gpca at caller factors X_dev (m x k), Yt_dev (n x k)
 * (element type of the model), reduced in FP64 and written to the device
 * double out_dev.  Does not synchronise.  This is the forward of the
 * differentiable form. */
int glrm_objective_at(glrm_t h, const void *X_dev, const void *Yt_dev, double *out_dev);

/* Gradient of the objective at caller factors (Section 7.2, "Gradient
 * method"): GX_dev[i] = sum_{j in Omega_i} L_j'(x_i . y_j, A_ij) y_j and
 * GYt_dev[j] = sum_{i in Omega_j} L_j'(x_i . y_j, A_ij) x_i (m x k and n x k,
 * element type of the model).  With include_reg != 0 the regulariser's
 * gradient is added (2 w x for GLRM_REG_QUAD, w sign(x) for GLRM_REG_L1, 0 for
 * GLRM_REG_ZERO; GLRM_REG_NONNEG is not differentiable and returns
 * GLRM_ERR_ARG).  scale_dev, if not NULL, points to a device double that
 * multiplies both gradients (the incoming derivative of a backward pass).
 * Residuals are recomputed from the factors, never stored.  Does not
 * synchronise.  This is the backward of the differentiable form. */
int glrm_grad_at(glrm_t h, const void *X_dev, const void *Yt_dev, void *GX_dev,
                 void *GYt_dev, int32_t include_reg, const double *scale_dev);

/* Loss part of the gradient at the model's own factors (Section 7.2,
 * "Gradient method"): GX_dev[i] = sum_{j in Omega_i} L_j'(x_i . y_j, A_ij) y_j
 * (m x k) and GYt_dev[j] = sum_{i in Omega_j} L_j'(x_i . y_j, A_ij) x_i
 * (n x k), element type of the model, caller-owned device buffers.  The
 * regulariser's gradient is not added (the caller adds it where it exists).
 * Equivalent to glrm_grad_at(h, X, Yt, GX_dev, GYt_dev, 0, NULL) with the
 * handle's factors; does not synchronise. */
int glrm_grad(glrm_t h, void *GX_dev, void *GYt_dev);

/* Imputation (Section 5.3): for the cnt pairs (rows_dev[e], cols_dev[e])
 * write u = x_i . y_j (decode == 0) or the decoded value argmin_a L_j(u, a)
 * (decode != 0): u for quadratic, Huber, l1 and quantile columns, +1 if u >= 0 else -1 for
 * hinge and logistic columns, 1 + #{a in 1..d-1 : u > a + 1/2} for ordinal
 * columns (the minimiser of the ordinal hinge, ties to the lower level).
 * out_dev holds cnt values of the model's element type.  Indices out of range
 * produce NaN.  Does not synchronise. */
int glrm_predict(glrm_t h, int64_t cnt, const int32_t *rows_dev, const int32_t *cols_dev,
                 void *out_dev, int32_t decode);

/* Alternating minimisation for quadratic loss and quadratic regularisation
 * (Algorithm 1; Section 2.4 "Alternating minimization" and "Caching
 * factorizations", with each row's Gram matrix restricted to its observed
 * entries, Section 2.5): every x_i becomes the solution of
 * (sum_{j in Omega_i} y_j y_j^T + gamma I) x = sum_{j in Omega_i} A_ij y_j,
 * then every y_j likewise against the new X.  The Gram matrices accumulate in
 * the model's element type; the k x k Cholesky factorisation and the two
 * triangular solves run in FP64.  Requires every column loss to be
 * GLRM_LOSS_QUAD and rx, ry both GLRM_REG_QUAD with the same weight gamma
 * (else GLRM_ERR_ARG).  history_host as in glrm_sweep. */
int glrm_als_sweep(glrm_t h, int32_t nsweeps, double *history_host);

/* Prox-prox sweeps for quadratic loss and any of the regularisers (Section
 * 7.2, "Prox-prox method", with the cached factorisation of Section 7.3):
 * every row x_i, then every column y_j (against the new X), takes `inner`
 * updates
 *     x <- prox_{alpha r}(prox_{alpha f}(x)),
 *     prox_{alpha f}(x) = argmin_x' alpha f(x') + ||x' - x||^2 / 2
 *                       = (2 alpha G + I)^{-1} (2 alpha b + x),
 * f(x) = sum_{j in Omega_i} (x . y_j - A_ij)^2, G = sum y_j y_j^T,
 * b = sum A_ij y_j, with one FP64 Cholesky factorisation of 2 alpha G + I
 * per row reused by the `inner` updates (Gram matrices accumulated in the
 * model's element type).  The update's fixed point minimises the Moreau
 * envelope of f plus r; for r = 0 that is the least-squares row problem's
 * solution.  alpha > 0 (a constant step), inner >= 1, k <= 32; every column
 * loss must be GLRM_LOSS_QUAD (GLRM_ERR_ARG otherwise).  history_host as in
 * glrm_sweep (the objective of eq. gpca after each sweep, FP64).  A row
 * system whose factorisation fails keeps its factor; with history_host the
 * call then returns GLRM_ERR_NONFINITE. */
int glrm_proxprox_sweep(glrm_t h, int32_t nsweeps, double alpha, int32_t inner, double *history_host);

/* Serialise the fit state (factors, step sizes, sweep counter) into buf_host.
 * With buf_host NULL, *len receives the size needed.  Synchronises.
 * glrm_set_state restores it into a handle of the same m, n, k, precision;
 * continuing from a restored state is bitwise identical to not stopping. */
int glrm_get_state(glrm_t h, void *buf_host, size_t *len);
int glrm_set_state(glrm_t h, const void *buf_host, size_t len);

/* Kernel path of each half-step (a tuning knob; results agree to rounding).
 *   GLRM_PATH_CHUNKED  entries cut into chunks of <= 1024, one warp each; the
 *                      other factor read from global memory (any k, any size)
 *   GLRM_PATH_FUSED    the whole other factor staged in each CTA's shared
 *                      memory by a TMA bulk copy; one warp runs a row's (column's)
 *                      gradient, prox, re-evaluation and decision in one kernel
 *   GLRM_PATH_BLOCKED  the other factor staged panel by panel (TMA); per
 *                      (panel, segment) partials summed over panels in a fixed
 *                      order
 *   GLRM_PATH_MASKED   segments in tiles of 32, one per lane; a warp walks the
 *                      union of its tile's other-indices in order and reads each
 *                      other-factor row once as a shared-memory broadcast (the
 *                      whole factor resident, or the rows of each batch of 32
 *                      gathered with cp.async); values re-ordered at set-up and
 *                      streamed by TMA.  When there are fewer tiles than warps
 *                      on the GPU, a tile's list is split over several warps
 *                      whose partials are summed in a fixed order.
 *   GLRM_PATH_MASKED_SPLIT  the masked path with every tile split in two or
 *                      more units (glrm_get_path reports it whenever a masked
 *                      half-step runs split)
 *   GLRM_PATH_DENSE    (both half-steps) the table stored densely with NaN at
 *                      the missing cells and swept by the tensor-core form of
 *                      glrm_set_dense; FP32 and BF16 models with k <= 64
 * GLRM_PATH_AUTO picks dense for FP32 and BF16 models with k <= 64 when at least 40% of
 * the cells are observed (and the dense copy takes at most half the free
 * device memory); otherwise masked when a tile's pairs average >= 8 observed
 * lanes, else fused when the other factor fits, else blocked when a
 * (panel, segment) run holds >= 64 entries on average, else chunked.  The
 * staged paths need k <= 32.  glrm_set_path(h, xstep_path, ystep_path) may be
 * called before or after glrm_set_observed; an infeasible request returns
 * GLRM_ERR_ARG and restores GLRM_PATH_AUTO.  glrm_get_path writes the paths in
 * use (2 values, never AUTO) after glrm_set_observed. */
typedef enum {
    GLRM_PATH_AUTO = 0,
    GLRM_PATH_CHUNKED = 1,
    GLRM_PATH_FUSED = 2,
    GLRM_PATH_BLOCKED = 3,
    GLRM_PATH_MASKED = 4,
    GLRM_PATH_MASKED_SPLIT = 5,
    GLRM_PATH_DENSE = 6 /* reported for a dense table (glrm_set_dense) */
} glrm_path;
int glrm_set_path(glrm_t h, int32_t xstep_path, int32_t ystep_path);
int glrm_get_path(glrm_t h, int32_t *paths_host);

/* ------------------------------------------------------------ batched form
 * Many independent models of uneven size fitted together.  Each instance is a
 * model of eq. gpca with one loss for all its columns and its own
 * regularisers, fitted either by the proximal-gradient sweep with the
 * step-size rule (Algorithm 2, Section 7.2) or, for quadratic loss with
 * gamma ||.||^2 on both factors, by alternating minimisation (Algorithm 1 with
 * the row / column problems of Section 2.4 solved exactly: Gram matrix of the
 * observed entries in FP32, k x k Cholesky factorisation and solves in FP64).
 * All nsweeps sweeps of a call run in one persistent launch: its warps take
 * work items from a device queue -- for each sweep every instance's X-step
 * items (an instance and a range of its rows), then the Y-step items, then one
 * objective item per instance -- and per-instance completion counters order
 * them (an instance's Y-step after its X-step, its objective after its Y-step,
 * its next X-step after its objective).  Each dependency wait is bounded
 * (glrm_batch_set_wait_limit); a wait that runs out makes the call return
 * GLRM_ERR_TIMEOUT.  With GLRM_BATCH_GRAPH the launch (and the counter reset
 * before it) is captured once into a CUDA graph and replayed.  k must be 4, 8
 * or 16 (FP32). */
typedef struct glrm_batch_s *glrm_batch_t;
enum { GLRM_BATCH_PROXGRAD = 0, GLRM_BATCH_ALS = 1 };
/* sweep modes: graph replay, plain launches on the stream, and one launch per
 * instance and half-step (for comparison) */
enum { GLRM_BATCH_GRAPH = 0, GLRM_BATCH_STREAM = 1, GLRM_BATCH_PER_INSTANCE = 2 };
typedef struct {
    int64_t m, n;   /* rows, columns */
    int32_t k;      /* 4, 8 or 16 */
    int32_t method; /* GLRM_BATCH_PROXGRAD or GLRM_BATCH_ALS */
    glrm_loss loss; /* loss of every column of the instance */
    int32_t rx_kind, ry_kind;
    double rx_weight, ry_weight;
    int64_t nnz;    /* observed entries */
} glrm_batch_instance;

/* Instances are laid out one after another: instance s's CSR pointers (m_s+1
 * values, starting at 0) follow instance s-1's, its entries (nnz_s indices and
 * values, indices local to the instance) follow s-1's, likewise for CSC.
 * Device pointers, copied; validated on the device (as glrm_set_observed).
 * Factors start at zero (glrm_batch_set_factors); X is the concatenation of
 * every instance's m_s x k_s row-major X, Yt likewise.  Step sizes start at
 * 1/max(count, 1).  Synchronises.  On error *out may still hold a handle to
 * pass to glrm_batch_destroy. */
int glrm_batch_create(int32_t count, const glrm_batch_instance *inst_host, const int32_t *rowptr_dev,
                      const int32_t *colidx_dev, const float *val_dev, const int32_t *colptr_dev,
                      const int32_t *rowidx_dev, const float *cval_dev, void *stream,
                      glrm_batch_t *out);
int glrm_batch_set_factors(glrm_batch_t b, const float *X_dev, const float *Yt_dev);
int glrm_batch_get_factors(glrm_batch_t b, float *X_dev, float *Yt_dev);
/* step sizes: one float per row of every instance (ax), per column (ay) */
int glrm_batch_set_steps(glrm_batch_t b, const float *ax_dev, const float *ay_dev);
int glrm_batch_get_steps(glrm_batch_t b, float *ax_dev, float *ay_dev);
/* nsweeps sweeps of every instance; objectives_host, if not NULL, receives
 * nsweeps x count doubles (sweep-major), the objective of each instance after
 * each sweep, and the call synchronises and reports the device status:
 * GLRM_ERR_TIMEOUT when a dependency wait ran out (results invalid),
 * GLRM_ERR_NONFINITE when an ALS system was not numerically positive definite
 * (those rows / columns kept their factor).  Modes: GLRM_BATCH_GRAPH and
 * GLRM_BATCH_STREAM make the one queue launch (replayed from a graph, or
 * enqueued directly); GLRM_BATCH_PER_INSTANCE, for comparison, launches the
 * same kernel once per instance and half-step, and once per sweep for the
 * objectives. */
int glrm_batch_sweep(glrm_batch_t b, int32_t nsweeps, double *objectives_host, int32_t mode);
/* The number of polls (about 0.1 us each) a work item may spend waiting for
 * the items it depends on before it gives up and raises GLRM_ERR_TIMEOUT
 * (default 2^24).  Waits normally end within the run time of one item; a
 * small limit makes them run out on purpose (a test of the expiry path), 0
 * lets an item proceed only if its dependencies are already complete. */
int glrm_batch_set_wait_limit(glrm_batch_t b, int64_t polls);
/* Autotuner: for every bucket of instances (k, method, entries per row or
 * column class) and each half-step, times the half-step kernel on that
 * bucket's instances with 1, 2, 4 and 8 rows (columns) per work item and keeps
 * the fastest, then times the whole half-step with the work items ordered by
 * decreasing work or grouped by instance and keeps the faster order; the fit
 * state is saved and restored around the timing runs.  tiles_x / tiles_y (32
 * values each, nullable) receive the table. */
int glrm_batch_autotune(glrm_batch_t b, int32_t reps, int32_t *tiles_x_host, int32_t *tiles_y_host);
const char *glrm_batch_last_error(glrm_batch_t b);
void glrm_batch_destroy(glrm_batch_t b);

/* Tensor-core building block of the dense form: D = A B^T on the
 * fifth-generation tensor cores (tcgen05.mma, BF16 operands staged in shared
 * memory, FP32 accumulator in tensor memory).  A: M x K, B: N x K, both
 * row-major BF16 (raw 16-bit words); D: M x N row-major FP32.  Device
 * pointers; M a multiple of 128, N of 64, K one of 16, 32, 64, 128 (the
 * operands are staged in the 32-, 64- or 128-byte swizzled layouts the dense
 * form uses; GLRM_ERR_RANGE otherwise).  Synchronises; GLRM_ERR_TIMEOUT if a wait for
 * the tensor core hit its limit. */
int glrm_tc_gemm_bf16(const void *A_dev, const void *B_dev, float *D_dev, int32_t M, int32_t N,
                      int32_t K, void *stream);

/* Self-test of the device-side wait limit (not part of the method): one
 * thread waits, with the library's bounded mbarrier wait and a limit of
 * `attempts` try_wait attempts, on a barrier phase that completes only when
 * arm != 0 (the thread arrives on it first).  Returns GLRM_OK when the wait
 * completed and GLRM_ERR_TIMEOUT when it ran out (arm == 0): the same path a
 * staged copy or a tensor-core completion that never lands takes in the
 * sweep kernels, exercised without any copy or MMA in flight.  The GPU and the
 * CUDA context stay usable either way.  Synchronises.  GLRM_ERR_ARG if
 * attempts < 1. */
int glrm_wait_selftest(int64_t attempts, int32_t arm, void *stream);

/* FP32 FMA throughput of the current device (not part of the method; the
 * denominator of the CUDA-core roofline): a kernel whose threads each run 8
 * independent chains of `iters` fmaf (iters a multiple of 16, >= 16), at full
 * occupancy on every SM, timed with CUDA events over 5 launches after a
 * warm-up.  *tflops_host receives 2 x FMAs / time in TFLOP/s, *sms_host
 * (nullable) the SM count read from the device.  Synchronises. */
int glrm_fma_peak(int32_t iters, double *tflops_host, int32_t *sms_host, void *stream);

/* Instrumentation (not part of the method).  glrm_timing_enable(h, 1)
 * records a CUDA event on the handle's stream before every kernel the handle
 * launches and after the last one, so each kernel's device time is measured
 * on its own stream; glrm_timing_enable(h, 0) stops recording.  Enabling or
 * disabling clears the totals.  glrm_timing_read synchronises and returns, for
 * up to max_kernels kernel names (32-byte NUL-terminated slots in
 * names_host), the total milliseconds and launch counts recorded so far;
 * *count_host receives the number of names written.  glrm_launch_count gives
 * the number of kernels the handle has enqueued since creation. */
int glrm_timing_enable(glrm_t h, int32_t on);
int glrm_timing_read(glrm_t h, int32_t max_kernels, char *names_host, double *ms_host,
                     int64_t *launches_host, int32_t *count_host);
int glrm_launch_count(glrm_t h, int64_t *count_host);

/* Objective without any device allocation, for callers that cannot call
 * cudaMalloc where they need it: code recording into a CUDA graph capture (an
 * allocation inside a capture is not allowed), hosts whose device memory all
 * belongs to their own pool, loops that must not touch the allocator.  The
 * paper has no counterpart: this is the value glrm_objective_at computes
 * (FP32 model, per-row loss sums plus regularisers, reduced in FP64), for
 * caller-owned data and without a handle.
 *
 * Inputs (device pointers, caller-owned): CSR rowptr (m+1), colidx and val
 * (nnz each, FP32) of Omega; col_loss_dev: n glrm_loss descriptors in device
 * memory, 16-byte aligned; factors X_dev (m x k) and Yt_dev (n x k), FP32
 * row-major.  Output: the objective in the device double out_dev.  Work is
 * enqueued on `stream` (a cudaStream_t, NULL = legacy default stream); the
 * call does not synchronise.  The device data is not validated the way
 * glrm_set_observed validates it (no order or duplicate checks, no value
 * domains); what would make a read go out of range or a loss undefined turns
 * the result into NaN instead: a row range outside [0, nnz] or running
 * backwards, a column index outside [0, n), a loss descriptor with an
 * unknown kind, a Huber threshold that is not positive and finite, or fewer
 * than two ordinal levels.  Regulariser kinds and weights (finite, >= 0) are
 * checked on the host (GLRM_ERR_ARG).
 *
 * Scratch: a file-scope device array of GLRM_NOALLOC_MAX_TERMS doubles
 * (8 MiB) inside the library, held by every GPU that loads the library until
 * the process exits; m + n must not exceed GLRM_NOALLOC_MAX_TERMS and nnz
 * must be below 2^31 (GLRM_ERR_RANGE otherwise, nothing launched).  The first call on a device
 * looks up the array's device address on that device, so make that first call
 * outside any stream capture.  Every call overwrites the slots it uses; calls
 * that overlap on the GPU share the array and race.  Limits: 1 <= k <= 64. */
#define GLRM_NOALLOC_MAX_TERMS (1 << 20)
int glrm_objective_noalloc(int64_t m, int64_t n, int32_t k, int64_t nnz,
                           const int32_t *csr_rowptr_dev, const int32_t *csr_colidx_dev,
                           const float *csr_val_dev, const glrm_loss *col_loss_dev,
                           int32_t rx_kind, double rx_weight, int32_t ry_kind, double ry_weight,
                           const float *X_dev, const float *Yt_dev, double *out_dev, void *stream);

/* Per-handle message for the last error (empty string when none). */
const char *glrm_last_error(glrm_t h);

/* Message for an error that happened before a handle existed. */
const char *glrm_global_error(void);

/* Free every device buffer of the handle (after synchronising its stream). */
void glrm_destroy(glrm_t h);

#ifdef __cplusplus
}
#endif

#endif /* GLRM_H */
