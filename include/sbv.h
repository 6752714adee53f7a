/*
 * sbv.h -- C ABI of the GB300 Scaled Block Vecchia library (libsbv.so).
 *
 * Scaled Block Vecchia (SBV, arxiv 2504.12004) approximates a Gaussian-process
 * log-likelihood by a product of block conditionals (Sec. 4.2, Eq.
 * mmsearchingBV): points are scaled per dimension (Alg. 2), clustered into
 * blocks (Alg. 3), the blocks are put in random order (Alg. 1 Step 2), every
 * block conditions on the m points of earlier blocks nearest to its centre
 * (Alg. 4), and each block contributes log p(y_B | y_J) (Alg. 5).
 *
 * Conventions for every entry point
 *   - Return value: SBV_OK (0) or one of the SBV_E* codes below; the message
 *     of the last failure on a context is returned by sbv_last_error().
 *   - Pointers marked "device" are CUDA device pointers on the context's
 *     device; "host" pointers are ordinary host memory.  The caller owns every
 *     buffer it passes; the library never frees caller memory.  The library
 *     owns only the context and its internal workspace.
 *   - `stream` is a cudaStream_t (passed as void*; NULL = legacy default
 *     stream).  Calls are ordered on that stream.  sbv_blocking, sbv_knn and
 *     sbv_predict return after their work has finished; sbv_loglik only
 *     enqueues work (see its comment).
 *   - Point matrices are row-major n x d (point i occupies d consecutive
 *     values), dtype SBV_F64 (double) or SBV_F32 (float; widened exactly to
 *     double wherever a decision is taken).
 *   - Parameter rows theta are (sigma^2, tau^2, beta_1 .. beta_d): process
 *     variance, nugget and per-dimension ranges of the scaled Matern kernel
 *     K(a,b) = sigma^2 M_nu(r) + tau^2 [a is b], r^2 = sum_t ((x_at-x_bt)/beta_t)^2
 *     (Eq. scale, Eq. maternkernel), M_nu the Matern correlation for
 *     nu = nu2/2 (closed forms for nu2 in {1,3,5,7}; the FP64 paths also take
 *     any other nu2 up to SBV_MAX_NU2 through K_nu), evaluated at r itself
 *     (no sqrt(2 nu) factor, as the equation is printed).  The nugget is
 *     added only where a and b are the same data point.
 *   - Indices in outputs are original point indices (0-based).
 *   - There is no CPU fallback: every computation runs in CUDA kernels.
 */
#ifndef SBV_H
#define SBV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SBV_OK            0
#define SBV_EINVAL        1  /* invalid argument (sizes, null pointers, parameters) */
#define SBV_ENOTSPD       2  /* a covariance matrix was not positive definite */
#define SBV_ENOMEM        3  /* device or host allocation failed */
#define SBV_ECUDA         4  /* a CUDA runtime call failed (message has the CUDA error) */
#define SBV_ETIMEOUT      5  /* a bounded device wait gave up */
#define SBV_EUNSUPPORTED  6  /* size above a compiled limit, unsupported nu */

/* element types of point matrices */
#define SBV_F64 0
#define SBV_F32 1

/* arithmetic of the per-block factorisation */
#define SBV_PREC_FP64       0  /* everything in FP64 */
#define SBV_PREC_MIXED      1  /* FP32 factor of Sigma_JJ; double-float covariance, residual
                                  and Schur complement (third-order corrected); double-float
                                  LDL^T of the bs x bs conditional system */
#define SBV_PREC_MIXED_BF16 2  /* as SBV_PREC_MIXED with the residual's products on the tensor
                                  cores: exact BF16 digit products (tcgen05, TMEM) */

/* compiled limits */
#define SBV_MAX_DIM      64     /* d */
#define SBV_MAX_NU2      40     /* largest 2 nu of the FP64 paths (nu <= 20) */
#define SBV_MAX_BLOCK_N  1024   /* m_i + bs_i of one block */
#define SBV_MAX_DRAWS    (1 << 24)  /* draws per test point of sbv_simulate */

typedef struct sbv_ctx sbv_ctx;

/* Library version (major*10000 + minor*100 + patch). */
int sbv_version(void);

/* Create a context on CUDA device `device`.  *ctx receives the handle. */
int sbv_create(sbv_ctx** ctx, int device);

/* Destroy a context and release its workspace (NULL is ignored). */
void sbv_destroy(sbv_ctx* ctx);

/* Message describing the last non-zero status returned on `ctx`
 * (empty string if none; "null context" for NULL).  Owned by the context. */
const char* sbv_last_error(const sbv_ctx* ctx);

/*
 * sbv_blocking -- scaling, Random Anchor Clustering with Lloyd iterations, and
 * the random block order (Alg. 2 dimension scaling; Alg. 3; Alg. 1 Step 2).
 *
 *   X            device, n x d, dtype           input points
 *   beta_scale   host, d doubles > 0            scaling ranges: z = x / beta_scale
 *   bc           requested block count, 1 <= bc <= n
 *   kmeans_iters Lloyd iterations T >= 0 after the RAC assignment (T = 0 is RAC)
 *   seed         seed of the SplitMix64 stream that draws anchors and order
 *   blk          device, n int32     out: block of each point (compacted ids)
 *   ptr          device, bc+1 int64  out: CSR offsets, block j = pts[ptr[j] .. ptr[j+1])
 *   pts          device, n int32     out: points grouped by block, increasing index inside
 *   rank         device, bc int32    out: position of each block in the random order
 *   centres      device, bc x d f64  out: mean of each block's scaled members
 *   bc_eff       host, int64         out: number of non-empty blocks (entries
 *                                    beyond bc_eff of ptr/rank/centres are unused)
 *
 * Anchors are the first bc entries of a Fisher-Yates shuffle of [0, n) drawn
 * from SplitMix64(seed) with Lemire's bounded draw; every point joins the
 * anchor/centre with the smallest squared scaled distance (sum over
 * dimensions left to right, no fused multiply-add, ties to the smaller block);
 * Lloyd iterations recompute centres as member means (members summed in
 * increasing point index) and stop early when no assignment changes; empty
 * blocks are dropped; the order is a full Fisher-Yates shuffle from the same
 * stream, block perm[r] receiving rank r.  Results are bit-identical for a
 * given input on any GB300.
 * Errors: SBV_EINVAL (n < 1, d < 1 or > SBV_MAX_DIM, bc outside [1, n],
 * kmeans_iters < 0, beta_scale <= 0 or null pointers), SBV_ENOMEM, SBV_ECUDA.
 */
int sbv_blocking(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                 const double* beta_scale, int64_t bc, int32_t kmeans_iters,
                 uint64_t seed, int32_t* blk, int64_t* ptr, int32_t* pts,
                 int32_t* rank, double* centres, int64_t* bc_eff, void* stream);

/*
 * sbv_blocking_partitioned -- sbv_blocking with the partitioning of Alg. 2
 * first: points go to `partitions` = P slabs by int(x_dmax * P) on the
 * unscaled coordinate of the most relevant dimension d_max = argmax_j
 * 1/beta_scale_j (FP64 product and floor, clamped to [0, P-1]; ties to the
 * first dimension), then RAC and the Lloyd iterations run inside every slab
 * on its own points (Alg. 3 per partition).  Anchors per slab: one for every
 * non-empty slab, the rest of bc in proportion to the slab sizes (largest
 * remainder, ties to the lower slab), never more than the slab's points; the
 * anchors of slab q are the first k_q entries of a Fisher-Yates shuffle of
 * the slab's points in increasing index, slabs in increasing q, all from one
 * SplitMix64(seed) stream, followed by the block-order shuffle.  P = 1 is
 * sbv_blocking exactly.  1 <= P <= bc.  Outputs and errors as sbv_blocking.
 */
int sbv_blocking_partitioned(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                             const double* beta_scale, int64_t bc, int32_t kmeans_iters,
                             uint64_t seed, int32_t partitions, int32_t* blk, int64_t* ptr,
                             int32_t* pts, int32_t* rank, double* centres, int64_t* bc_eff,
                             void* stream);

/*
 * The pieces of sbv_blocking_partitioned for a distributed blocking, where
 * worker q holds only the points of slab q (Alg. 2 redistributes them with an
 * Alltoall; Alg. 3 then runs on every worker without communication).
 *
 * sbv_slabs -- slab of every point, int(x_dmax * P) as in
 * sbv_blocking_partitioned.  slab: device, n int32 out.  Asynchronous on
 * `stream`.  Errors: SBV_EINVAL, SBV_ECUDA.
 *
 * sbv_rac_plan -- the random choices of sbv_blocking_partitioned, which depend
 * only on the seed, the slab sizes and bc: host arrays, no context, no GPU.
 *   slab_counts  P sizes (the sizes of all slabs, in slab order)
 *   quota        P int64 out (or NULL): anchors k_q per slab
 *   anchor_pos   sum_q k_q int64 out (or NULL): slab by slab, the anchors of
 *                slab q as positions in that slab's points listed in
 *                increasing global index
 *   bc_eff, rank rank (or NULL): bc_eff int32 out, the block order of
 *                sbv_blocking_partitioned for bc_eff non-empty blocks numbered
 *                slab by slab (the draws that follow the anchors in the stream)
 * Errors: SBV_EINVAL (P < 1, negative counts, bc outside [max(P, 1), n],
 * bc_eff outside [1, bc] when rank is given).
 *
 * sbv_blocking_anchored -- RAC (from the given anchors) plus up to
 * kmeans_iters Lloyd iterations on one partition, as sbv_blocking does inside
 * a slab, without the block order.
 *   anchors      host, k distinct int64 point indices in [0, n)
 *   blk, ptr, pts, centres, bc_eff   as sbv_blocking (blocks in anchor order;
 *                empty ones dropped keeping that order)
 * With the points of slab q in increasing global index and the anchors
 * anchor_pos of slab q, the blocks equal those of slab q in
 * sbv_blocking_partitioned bit for bit.  Synchronises `stream`.
 * Errors: SBV_EINVAL (also for repeated or out-of-range anchors), SBV_ENOMEM,
 * SBV_ECUDA.
 */
int sbv_slabs(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
              const double* beta_scale, int32_t partitions, int32_t* slab, void* stream);
int sbv_rac_plan(uint64_t seed, int32_t partitions, const int64_t* slab_counts, int64_t bc,
                 int64_t* quota, int64_t* anchor_pos, int64_t bc_eff, int32_t* rank);
int sbv_blocking_anchored(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
                          const double* beta_scale, const int64_t* anchors, int64_t k,
                          int32_t kmeans_iters, int32_t* blk, int64_t* ptr, int32_t* pts,
                          double* centres, int64_t* bc_eff, void* stream);

/*
 * sbv_knn -- earlier-ordered m nearest neighbours of every block (Alg. 4,
 * Eq. mmsearchingBV).
 *
 *   X, dtype, n, d, beta_scale   as for sbv_blocking (same scaling)
 *   ptr, pts, rank, centres      device, output of sbv_blocking for bc blocks
 *   m            neighbours per block, 0 <= m <= SBV_MAX_BLOCK_N - 1
 *   nbr          device, bc x m int32  out: row j = neighbours of block j,
 *                                      ascending by (squared scaled distance to
 *                                      the centre, point index); -1 padded
 *   cnt          device, bc int32      out: m_j = min(m, #points of blocks
 *                                      with smaller rank)
 *
 * Candidates of block j are exactly the points of blocks with rank strictly
 * below rank[j] (a block never conditions on itself).  Distances are the
 * same bit-exact sums as in sbv_blocking.
 * Errors: SBV_EINVAL, SBV_EUNSUPPORTED (m too large), SBV_ENOMEM, SBV_ECUDA.
 */
int sbv_knn(sbv_ctx* ctx, const void* X, int dtype, int64_t n, int32_t d,
            const double* beta_scale, const int64_t* ptr, const int32_t* pts,
            const int32_t* rank, const double* centres, int64_t bc, int32_t m,
            int32_t* nbr, int32_t* cnt, void* stream);

/*
 * sbv_set_knn_mode -- how sbv_knn searches: 0 (default) chooses by size,
 * 1 always scans every earlier candidate, 2 always uses the pruned search
 * (blocks as clusters with centre and radius bounds, a 2-D grid over block
 * centres, a per-query radius standing in for the lambda of Eq.
 * distancethreshold and a check that the m-th key lies inside it, with
 * retries and the full scan as fallbacks).  All modes return the same
 * neighbours key for key.  Errors: SBV_EINVAL.
 */
int sbv_set_knn_mode(sbv_ctx* ctx, int32_t mode);

/*
 * sbv_loglik -- Block Vecchia log-likelihood for B parameter rows (Alg. 5
 * per block; Alg. 1 Step 5 for the sum).
 *
 *   X, dtype, n, d     device points (unscaled; the kernel ranges come from theta)
 *   y                  device, n doubles, observations
 *   ptr, pts           device, block CSR from sbv_blocking (bc blocks); the
 *                      offsets in ptr are absolute indices into pts, so a
 *                      contiguous range of blocks [lo, hi) is evaluated by
 *                      passing ptr + lo, nbr + lo * m, cnt + lo and bc = hi - lo
 *                      (one rank's share of an evaluation: Alg. 1 Step 5)
 *   nbr, cnt           device, neighbours from sbv_knn (row stride m)
 *   nmax               largest m_i + bs_i over the blocks, or 0: the call then
 *                      computes it (one small kernel and a device-to-host read
 *                      that waits for `stream`).  A value below the true
 *                      largest size is safe: the blocks above it get status
 *                      SBV_EUNSUPPORTED and a NaN term.
 *   theta              host, B x (2+d) doubles, rows (sigma^2, tau^2, beta_1..beta_d)
 *   nu2                2*nu: {1, 3, 5, 7} (closed forms) in every precision;
 *                      with SBV_PREC_FP64 also any other 2..SBV_MAX_NU2, where
 *                      M_nu = 2^(1-nu)/Gamma(nu) r^nu K_nu(r) with K_nu by an
 *                      exponentially convergent quadrature of its integral
 *                      representation (relative error below 1e-12)
 *   precision          SBV_PREC_FP64, SBV_PREC_MIXED or SBV_PREC_MIXED_BF16
 *   ll                 device, B doubles  out: l(theta_b) = sum_i l_{b,i}
 *   block_terms        device, B x bc doubles out (or NULL): l_{b,i}
 *   status             device, B x bc int32 out (or NULL): 0, or SBV_ENOTSPD
 *                      for a block whose matrix was not positive definite
 *                      (its term and the total are then NaN)
 *
 * Block i conditions its points B_i (in increasing index) on its neighbours
 * J_i (in the order of nbr): with Sigma the joint covariance of [J_i; B_i]
 * and L its Cholesky factor, w = L^{-1} [y_J; y_B] and
 *   l_{b,i} = -1/2 [ bs_i log(2 pi) + 2 sum_{t in B} log L_tt + sum_{t in B} w_t^2 ],
 * which equals the POTRF/TRSM/GEMM/Schur/POTRF/TRSV chain of Alg. 5 (with
 * Sigma^lk in the Schur step).  The mixed precisions follow that chain: an
 * FP32 factor of Sigma_JJ gives approximate kriging weights X, one
 * double-float residual R = Sigma_JB - Sigma_JJ X corrects the conditional
 * covariance and mean to third order in the error of X,
 *   Sigma^new = Sigma_BB - Sigma_BJ X - X^T R - (L^{-1} R)^T (L^{-1} R),
 * and a double-float LDL^T of Sigma^new gives the log-determinant and the
 * quadratic form.  A block whose FP32 or double-float pivot is not positive,
 * or whose conditional system exceeds the kernel's capacity, is recomputed
 * by the FP64 kernel in the same call (counted by sbv_fp64_reruns).  The sum
 * over blocks is a fixed-order tree, so repeated calls give bit-identical
 * results.  The call only enqueues work on `stream` and returns; failures
 * inside kernels are reported through `status`, NaN totals, and
 * sbv_sync_status().
 * Errors (argument checks, before any work): SBV_EINVAL (null pointers,
 * B < 1, sigma^2 <= 0, tau^2 < 0, beta <= 0, bad nu2 or precision),
 * SBV_EUNSUPPORTED (a block with m_i + bs_i > SBV_MAX_BLOCK_N), SBV_ENOMEM,
 * SBV_ECUDA.
 */
int sbv_loglik(sbv_ctx* ctx, const void* X, int dtype, const double* y,
               int64_t n, int32_t d, const int64_t* ptr, const int32_t* pts,
               const int32_t* nbr, const int32_t* cnt, int64_t bc, int32_t m,
               int32_t nmax, const double* theta, int32_t B, int32_t nu2,
               int32_t precision, double* ll, double* block_terms, int32_t* status,
               void* stream);

/*
 * sbv_loglik_grad -- the FP64 log-likelihood of sbv_loglik together with its
 * gradient with respect to theta = (sigma^2, tau^2, beta_1..beta_d), for B
 * parameter rows (the gradient information handed to the optimiser, Sec. 6).
 *
 * Arguments as sbv_loglik (FP64 arithmetic; no precision argument), plus
 *   grad               device, B x (2+d) doubles out: d l(theta_b) / d theta_k
 *                      (natural parameters, not their logarithms)
 *   block_grads        device, B x bc x (2+d) doubles out (or NULL):
 *                      d l_{b,i} / d theta_k
 * For block i, with S = J_i u B_i and either Gaussian system (S, and J_i),
 * d log N(y; 0, Sigma)/d theta_k = 1/2 x^T dSigma_k x - 1/2 tr(Sigma^-1 dSigma_k),
 * x = Sigma^-1 y; l_{b,i} is the S density minus the J_i one.  Derivatives of
 * the covariance: dK/dsigma^2 = M_nu(r), dK/dtau^2 = [same point],
 * dK/dbeta_t = sigma^2 h_nu(r) u_t^2 / beta_t with u_t = (x_at - x_bt)/beta_t and
 * h_nu = -M_nu'(r)/r (nu = 1/2: e^-r/r, 0 at r = 0; 3/2: e^-r; 5/2: (1+r)e^-r/3;
 * 7/2: (3+3r+r^2)e^-r/15).  The block terms (ll, block_terms) are the same
 * numbers sbv_loglik returns in FP64, bit for bit.  Sums over blocks are
 * fixed-order trees (repeatable).  Each item costs about three times the FP64
 * likelihood (the B rows of L^-1 by one backward substitution with bs + 2
 * right-hand sides, then one pass over the pairs).
 * Errors: as sbv_loglik (SBV_EINVAL, SBV_EUNSUPPORTED, SBV_ENOMEM,
 * SBV_ECUDA); a block that is not positive definite gets NaN term and
 * gradient and status SBV_ENOTSPD.
 */
int sbv_loglik_grad(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                    int32_t d, const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                    const int32_t* cnt, int64_t bc, int32_t m, int32_t nmax,
                    const double* theta, int32_t B, int32_t nu2, double* ll, double* grad,
                    double* block_terms, double* block_grads, int32_t* status, void* stream);

/*
 * sbv_sync_status -- wait for `stream`, then report whether any sbv_loglik or
 * sbv_predict kernel since the previous call met a non-positive-definite
 * matrix (SBV_ENOTSPD, message names the first block/test point) or a CUDA
 * error (SBV_ECUDA).  Clears the record.
 */
int sbv_sync_status(sbv_ctx* ctx, void* stream);

/*
 * sbv_fp64_reruns -- wait for `stream`, then write to *count (host) how many
 * (theta, block) items or test points the mixed-precision kernels handed to
 * the FP64 kernels since the last sbv_sync_status (which clears the count):
 * items with a non-positive FP32 or double-float pivot, or whose conditional
 * system exceeds the mixed kernel's capacity.  Their results are the FP64
 * path's.  Errors: SBV_EINVAL (null ctx or count), SBV_ECUDA.
 */
int sbv_fp64_reruns(sbv_ctx* ctx, void* stream, int64_t* count);

/*
 * sbv_predict -- Block Vecchia prediction with one test point per block
 * (Sec. 4.2 prediction product; Sec. 5.5).
 *
 *   X, dtype, y, n, d  device training points and observations
 *   Xtest              device, ntest x d, same dtype
 *   beta_scale         host, d doubles: scaling used to rank neighbours
 *   m_pred             neighbours per test point, 1 <= m_pred <= min(n, SBV_MAX_BLOCK_N - 1)
 *   theta              host, 2+d doubles (one parameter row)
 *   mean, var, var_latent  device, ntest doubles out: conditional mean, variance
 *                      on the observation scale (includes tau^2) and of the
 *                      latent process (var - tau^2)
 *   nbr                device, ntest x m_pred int32 out (or NULL): neighbours
 *                      of each test point, ascending by (scaled distance, index)
 *
 * Each test point conditions on its m_pred nearest training points (all n are
 * candidates): mean = Sigma_{*J} Sigma_JJ^{-1} y_J and
 * var = sigma^2 + tau^2 - Sigma_{*J} Sigma_JJ^{-1} Sigma_{J*}.
 * Errors: SBV_EINVAL, SBV_EUNSUPPORTED, SBV_ENOTSPD, SBV_ENOMEM, SBV_ECUDA.
 */
int sbv_predict(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                int64_t n, int32_t d, const void* Xtest, int64_t ntest,
                const double* beta_scale, int32_t m_pred, const double* theta,
                int32_t nu2, int32_t precision, double* mean, double* var,
                double* var_latent, int32_t* nbr, void* stream);

/*
 * sbv_predict_blocks -- sbv_predict with the neighbour search over the
 * training blocks (ptr, pts, rank, centres: device, bc blocks, as returned by
 * sbv_blocking or sbv_blocking_partitioned on the same X and beta_scale).
 * The blocks only prune the search (see sbv_set_knn_mode): the neighbours,
 * and therefore every output, equal those of sbv_predict.  Intended for large
 * n, where scanning all training points for every test point is too slow.
 * Errors: as sbv_predict, SBV_EINVAL for an incomplete block structure.
 */
int sbv_predict_blocks(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                       int32_t d, const void* Xtest, int64_t ntest, const double* beta_scale,
                       int32_t m_pred, const double* theta, int32_t nu2, int32_t precision,
                       const int64_t* ptr, const int32_t* pts, const int32_t* rank,
                       const double* centres, int64_t bc, double* mean, double* var,
                       double* var_latent, int32_t* nbr, void* stream);

/*
 * sbv_simulate -- conditional simulation at the test points (Sec. 5.5): for
 * every test point j, ndraws samples x_jk ~ N(mean_j, var_j) (var_j is the
 * variance, as sbv_predict's `var` output: the diagonal of Sigma^new), then
 * the sample mean, the sample variance s_j^2 = sum_k (x_jk - mean~_j)^2 /
 * (ndraws - 1) and the 95 % interval mean~_j -/+ z_{0.975} s_j,
 * z_{0.975} = 1.959963984540054.
 *
 *   mean, var          device, ntest doubles (var >= 0; a negative or NaN
 *                      variance gives NaN outputs for that point)
 *   ndraws             draws per test point, 2 <= ndraws <= SBV_MAX_DRAWS
 *                      (the paper takes 1000)
 *   seed               key of the generator
 *   index_base         counter index of test point 0: test point j draws as
 *                      point index_base + j, so a caller that splits its test
 *                      points into chunks (index_base = first point of the
 *                      chunk) gets the draws of one call over all of them
 *   sample_mean, sample_var, ci_lo, ci_hi   device, ntest doubles out
 *   draws              device, ntest x ndraws doubles out (row j holds the
 *                      draws of test point j in draw order), or NULL
 *
 * Draw k of test point j is a pure function of (seed, index_base + j, k): the
 * Philox4x64-10 block of counter (k / 4, index_base + j, 0, 0) under key
 * (seed, 0) (Salmon et al., SC
 * 2011) gives two pairs of uniforms u = ((w >> 12) + 1/2) 2^-52, and the
 * Box-Muller transform maps pair (u1, u2) to sqrt(-2 ln u1) cos(2 pi u2) for
 * k mod 4 in {0, 2} and sqrt(-2 ln u1) sin(2 pi u2) for {1, 3};
 * x_jk = mean_j + sqrt(var_j) z_jk.  FP64 throughout.  Asynchronous on
 * `stream`; ntest = 0 is a no-op.  Errors: SBV_EINVAL, SBV_ECUDA.
 */
int sbv_simulate(sbv_ctx* ctx, const double* mean, const double* var, int64_t ntest,
                 int32_t ndraws, uint64_t seed, uint64_t index_base, double* sample_mean,
                 double* sample_var,
                 double* ci_lo, double* ci_hi, double* draws, void* stream);

/*
 * sbv_matern -- the correlation function alone, M_nu(r) of Eq. (maternkernel)
 * with nu = nu2 / 2 at r = sqrt(d2), through the arithmetic of one precision
 * of the likelihood: SBV_PREC_FP64 takes the FP64 square root and the closed
 * form (nu2 in {1, 3, 5, 7}) or the K_nu quadrature (other nu2 up to
 * SBV_MAX_NU2); the mixed precisions split d2 into a float pair and take the
 * double-float square root, exponential and closed-form polynomial of their
 * covariance stage (nu2 in {1, 3, 5, 7}).
 *
 *   d2     device, n doubles >= 0: squared scaled distances sum_t (dx_t / beta_t)^2
 *   out    device, n doubles out
 *
 * Asynchronous on `stream`; n = 0 is a no-op.  Errors: SBV_EINVAL, SBV_ECUDA.
 */
int sbv_matern(sbv_ctx* ctx, int32_t precision, int32_t nu2, const double* d2, int64_t n,
               double* out, void* stream);

/*
 * sbv_predict_blocked -- block prediction (Sec. 5.5: prediction follows the
 * estimation pipeline): the test points are blocked like the training points
 * (RAC anchors + up to kmeans_iters Lloyd iterations in the beta_scale space,
 * bc_test blocks, seed as in sbv_blocking), each test block takes the m_pred
 * training points nearest to its centre (all training points are candidates)
 * as its conditioning set J, and every test point q of the block gets the
 * exact Gaussian conditional given y_J: mean_q = Sigma_qJ Sigma_JJ^{-1} y_J,
 * var_q = sigma^2 + tau^2 - Sigma_qJ Sigma_JJ^{-1} Sigma_Jq.  One factorisation
 * of Sigma_JJ serves the whole block.
 *
 *   X ... theta, nu2, precision   as sbv_predict
 *   bc_test            test blocks, 1 <= bc_test <= ntest (empty ones dropped)
 *   ptr, pts, rank, centres, bc   training blocks from sbv_blocking on the same
 *                      X and beta_scale (only prune the neighbour search), or
 *                      ptr = NULL for the full scan
 *   mean, var, var_latent  device, ntest doubles out (in test point order)
 *   test_block         device, ntest int32 out (or NULL): block of each test point
 *   nbr                device, bc_test x m_pred int32 out (or NULL): neighbours of
 *                      each test block (rows < *bc_test_eff), ascending by
 *                      (scaled distance to the centre, index)
 *   bc_test_eff        host (or NULL): non-empty test blocks
 *
 * Requires m_pred + the largest test block <= SBV_MAX_BLOCK_N.  Synchronises
 * `stream`.  Errors: as sbv_predict.
 */
int sbv_predict_blocked(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                        int32_t d, const void* Xtest, int64_t ntest, const double* beta_scale,
                        int32_t m_pred, int64_t bc_test, int32_t kmeans_iters, uint64_t seed,
                        const double* theta, int32_t nu2, int32_t precision, const int64_t* ptr,
                        const int32_t* pts, const int32_t* rank, const double* centres,
                        int64_t bc, double* mean, double* var, double* var_latent,
                        int32_t* test_block, int32_t* nbr, int64_t* bc_test_eff, void* stream);

/*
 * Captured evaluation (Sec. 5.4: all blocks of an evaluation in one batched
 * launch).  sbv_loglik_graph_create records one evaluation of sbv_loglik --
 * work-counter reset, the persistent block kernel over every (theta, block)
 * item, the deterministic sum -- as a CUDA graph for fixed inputs, structure,
 * B, nu2 and precision; the graph owns its scratch (and splits X once, in the
 * mixed modes) and reads the B parameter rows from a device buffer of its own.
 * sbv_loglik_graph_launch stages new rows (host, B x (2+d)) through pinned
 * memory and replays the graph on `stream`; results land in the `ll` (and
 * block_terms/status, if given) buffers passed at creation, which must stay
 * valid, as must every input, until the graph is destroyed.  Launches are
 * ordered on the stream; do not run two launches of one graph concurrently.
 * Errors: as sbv_loglik; SBV_ENOMEM for the graph's own buffers.
 */
typedef struct sbv_graph sbv_graph;

int sbv_loglik_graph_create(sbv_ctx* ctx, const void* X, int dtype, const double* y,
                            int64_t n, int32_t d, const int64_t* ptr, const int32_t* pts,
                            const int32_t* nbr, const int32_t* cnt, int64_t bc, int32_t m,
                            int32_t nmax, int32_t B, int32_t nu2, int32_t precision,
                            double* ll, double* block_terms, int32_t* status,
                            sbv_graph** graph);
int sbv_loglik_graph_launch(sbv_graph* graph, const double* theta, void* stream);
void sbv_loglik_graph_destroy(sbv_graph* graph);

/*
 * sbv_autotune -- time the launch shapes of the block kernel for one
 * structure (FP64: 1-4 resident CTAs of 256 threads per SM; mixed modes:
 * 256 threads with 2 or 1 CTAs per SM, or 512 threads with 1, each with a
 * column-block width of 16, 32 or 64 right-hand sides for the residual and
 * the conditional system, capped by the shared memory it has) on the given
 * arguments (one warm-up and two timed evaluations each, synchronising
 * `stream`) and record the fastest on the context; later sbv_loglik calls and
 * graphs with the same (precision, largest block size, d) use it.
 * *threads and *ctas_per_sm (host, may be NULL) receive the choice;
 * sbv_tuned_shape reads back the whole record.  Errors: as sbv_loglik.
 */
int sbv_autotune(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                 int32_t d, const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                 const int32_t* cnt, int64_t bc, int32_t m, int32_t nmax,
                 const double* theta, int32_t B, int32_t nu2, int32_t precision,
                 int32_t* threads, int32_t* ctas_per_sm, void* stream);

/*
 * sbv_tuned_shape -- the autotuner's record for (precision, nmax = largest
 * m_i + bs_i, d): *threads, *ctas_per_sm and *tile (host, each may be NULL;
 * tile = right-hand sides per column block in the mixed modes, 0 for FP64).
 * Returns SBV_EINVAL when no record exists.
 */
int sbv_tuned_shape(sbv_ctx* ctx, int32_t precision, int32_t nmax, int32_t d, int32_t* threads,
                    int32_t* ctas_per_sm, int32_t* tile);

/*
 * sbv_peak_probe -- measured FMA rate of the CUDA cores, for roofline
 * denominators.  The paper has no counterpart (it reports the GFLOP/s of its
 * FP64 batched kernels, Sec. 8.1, without a peak).  kind 0 times FP64 DFMA,
 * kind 1 FP32 FFMA: 8 independent chains per thread, 8 CTAs of 256 threads
 * per SM, 2 flops per FMA; one warm-up launch, then the best of three timed
 * launches (CUDA events on a private stream, which the call synchronises).
 * *tflops (host) receives TFLOP/s.  Errors: SBV_EINVAL, SBV_ECUDA.
 */
int sbv_peak_probe(sbv_ctx* ctx, int32_t kind, double* tflops);

/* Limits of the fixed scratch array of sbv_loglik_fp64_noalloc (about 8.1 MB
 * per GPU that loads the library, held until the process exits). */
#define SBV_NOALLOC_MAX_THETA 64          /* parameter rows per call */
#define SBV_NOALLOC_MAX_TERMS (1 << 20)   /* bc * B when block_terms is NULL */

/*
 * sbv_loglik_fp64_noalloc -- sbv_loglik in FP64 (SBV_PREC_FP64) without any
 * allocation.  The paper has no counterpart: this entry point exists for
 * callers that may not allocate device memory while they run, e.g. a serving
 * loop whose device memory belongs to another allocator (a framework's
 * caching allocator or a fixed budget, which a library-side cudaMalloc could
 * exceed or fragment) or a latency-bound loop that cannot afford the implicit
 * synchronisation of cudaMalloc/cudaFree.  It never calls cudaMalloc,
 * cudaFree or any other allocating routine, on the device or the host.
 *
 * Arguments and results are those of sbv_loglik (same layouts, same
 * per-block terms, bit-identical totals for the same inputs), with these
 * differences:
 *   - no context: the call runs on the current CUDA device and reports only
 *     its return code (no message); device-side failures show in `status`
 *     and as NaN terms;
 *   - B <= SBV_NOALLOC_MAX_THETA; when block_terms is NULL, bc * B <=
 *     SBV_NOALLOC_MAX_TERMS; every block (nmax + its coordinates) must fit in
 *     shared memory.  Beyond these limits the call returns SBV_EUNSUPPORTED
 *     before doing any work;
 *   - nmax = 0 makes the call compute the largest block size with one small
 *     kernel and a read into a host variable, which waits for `stream`.
 * All scratch (derived parameter rows, block terms when block_terms is NULL,
 * the work counter and the failure record) lives in one file-scope device
 * array shared by every call; it keeps the last call's contents, and the call
 * clears the parts that must start at zero.  Calls that overlap on the GPU
 * (on different streams, or from different host threads) use the same array
 * and race: serialise them.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.
 * Errors: SBV_EINVAL, SBV_EUNSUPPORTED (limits above), SBV_ECUDA.
 */
int sbv_loglik_fp64_noalloc(const void* X, int dtype, const double* y, int64_t n,
                            int32_t d, const int64_t* ptr, const int32_t* pts,
                            const int32_t* nbr, const int32_t* cnt, int64_t bc,
                            int32_t m, int32_t nmax, const double* theta, int32_t B,
                            int32_t nu2, double* ll, double* block_terms,
                            int32_t* status, void* stream);

/* ------------------------------------------------------------------------
 * Likelihood surrogate network.  The paper has no learned component; this
 * network s(x) regresses (standardised) log-likelihood values on
 * (standardised) log parameters so that the maximisation of the likelihood
 * (Alg. 1 Step 5 evaluated once per optimiser iteration, Sec. 5.4) can ask it
 * for candidates, which the exact likelihood then judges.
 *
 * Architecture: in_dim -> 256 -> 256 -> 256 -> 1, GELU(z) = z Phi(z) after
 * each hidden layer; loss L = (1/K) sum_k (s(x_k) - t_k)^2; Adam (Kingma &
 * Ba 2015) with bias correction.  The 256 x 256 layers (forward, backward and
 * weight gradients) run on the tensor cores with BF16 operands and FP32
 * accumulation; the rest in FP32.
 *
 * Parameters are FP32, packed in the order W1 (256 x in_dim), b1 (256),
 * W2 (256 x 256), b2, W3 (256 x 256), b3, w4 (256), b4 (1); weights are
 * [out][in] row-major, a layer computes z = h W^T + b.
 * Inputs X: device FP32, K x in_dim row-major; targets t: device FP32 (K).
 * Calls are ordered on `stream`; sbv_mlp_grad, sbv_mlp_train and
 * sbv_mlp_predict wait for it before returning (they check a device-side
 * timeout flag).  Errors: SBV_EINVAL, SBV_ENOMEM, SBV_ECUDA, SBV_ETIMEOUT
 * (a bounded tensor-core wait gave up; the results are then invalid).
 * ---------------------------------------------------------------------- */
#define SBV_MLP_WIDTH 256
#define SBV_MLP_MAX_IN 16

typedef struct sbv_mlp sbv_mlp;

/* Number of packed parameters for in_dim inputs (-1 if in_dim is out of range). */
int64_t sbv_mlp_num_params(int32_t in_dim);
/* Create a network on ctx's device with parameters drawn from one SplitMix64
 * stream seeded by `seed`: for each tensor in packed order, element by
 * element, u = (next() >> 11) * 2^-53 and value (2u - 1) / sqrt(fan_in)
 * rounded to FP32 (fan_in = in_dim for W1 and b1, 256 otherwise). */
int sbv_mlp_create(sbv_ctx* ctx, int32_t in_dim, uint64_t seed, sbv_mlp** mlp);
void sbv_mlp_destroy(sbv_mlp* mlp);
/* Copy the FP32 parameters from / to host memory (n = sbv_mlp_num_params);
 * set_params also clears the Adam state. */
int sbv_mlp_set_params(sbv_mlp* mlp, const float* params, int64_t n);
int sbv_mlp_get_params(sbv_mlp* mlp, float* params, int64_t n);
/* Gradient of L over all K rows: grads (device FP32, packed like the
 * parameters) and loss (device FP32 scalar), each may be NULL. */
int sbv_mlp_grad(sbv_mlp* mlp, const float* X, const float* t, int64_t K, float* grads,
                 float* loss, void* stream);
/* One Adam step on the gradient of the last sbv_mlp_grad call. */
int sbv_mlp_adam(sbv_mlp* mlp, float lr, float beta1, float beta2, float eps, void* stream);
/* `steps` Adam steps (beta1 0.9, beta2 0.999, eps 1e-8) on mini-batches of
 * `batch` rows: consecutive slices of Fisher-Yates permutations of [0, K)
 * drawn from SplitMix64(seed), a new permutation after each pass (the last
 * slice of a pass may be shorter).  *loss_out (host, may be NULL) receives the
 * loss of the last mini-batch. */
int sbv_mlp_train(sbv_mlp* mlp, const float* X, const float* t, int64_t K, int32_t steps,
                  int32_t batch, float lr, uint64_t seed, float* loss_out, void* stream);
/* s(x) for K rows into s (device FP32, K) and, if dsdx is not NULL, the
 * input gradients ds/dx (device FP32, K x in_dim). */
int sbv_mlp_predict(sbv_mlp* mlp, const float* X, int64_t K, float* s, float* dsdx,
                    void* stream);

/* ------------------------------------------------------------------------
 * Maximum-likelihood estimation.  The paper maximises the SBV log-likelihood
 * over theta with a library optimiser that re-evaluates Alg. 5 (summed as in
 * Alg. 1 Step 5) once per iteration while the data stay on the GPU
 * (Sec. 5.4; Sec. 7 runs 500 iterations); it does not name the algorithm.
 * sbv_mle runs BFGS on u = log theta inside box bounds: each iteration is one
 * batched call for a line search over `line_points` step lengths
 * 1, 1/2, 1/4, ... along the quasi-Newton direction (capped to `max_step` in
 * the max norm) and one batched call for the central-difference gradient
 * (2 (2 + d) rows) at the accepted point, or, with gradient = 1, one call of
 * sbv_loglik_grad (FP64 value and analytic gradient, chain rule to log
 * theta) at the accepted point.  It stops when an accepted step
 * gains less than ftol |l|, when no step length improves l along a fresh
 * (reset) direction, or before a call would exceed max_evals rows.
 * A parameter row whose block matrices are not positive definite counts as
 * l = -inf.  Rows: theta = (sigma^2, tau^2, beta_1..beta_d), natural scale.
 * Bounds lower/upper (host, 2 + d, NULL = defaults (1e-6, 1e-10, 1e-4 ...)
 * and (1e6, 1e3, 1e3 ...)) must satisfy 0 < lower <= upper < inf; starting
 * entries that are 0 or outside are moved to the nearest bound.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t max_evals;     /* budget of exact parameter rows per start (4000) */
  double fd_step;        /* central-difference step in log theta (1e-3) */
  double ftol;           /* relative gain below which an iteration converges (1e-10) */
  double max_step;       /* largest step in log theta, max norm (1.0) */
  int32_t line_points;   /* step lengths per line-search call, 1..64 (8) */
  int32_t precision;     /* SBV_PREC_* (SBV_PREC_MIXED) */
  int32_t nu2;           /* 2 nu in {1, 3, 5, 7} (5) */
  int32_t gradient;      /* 0 central differences, 1 analytic (sbv_loglik_grad, FP64) (0) */
} sbv_mle_opts;

typedef struct {
  double ll;             /* log-likelihood at the returned parameters */
  int32_t evals;         /* exact parameter rows evaluated */
  int32_t calls;         /* batched likelihood calls */
  int32_t iterations;    /* accepted steps */
  int32_t converged;     /* 1 gain < ftol, 2 stationary, 0 budget exhausted */
  int32_t grad_evals;    /* analytic gradients evaluated (each also one row of evals;
                            about 2.4 FP64 likelihood rows of work) */
  int32_t proposals_won; /* line-search calls that a network proposal won */
} sbv_mle_result;

/* theta0, theta_out: host, 2 + d.  opts may be NULL (defaults above).  If
 * hist_len is not NULL, up to hist_cap evaluated rows are written to hist_u
 * (log theta, hist_cap x (2 + d)) and hist_l (their l) and their number to
 * *hist_len.  Waits for `stream` after every call. */
int sbv_mle(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n, int32_t d,
            const int64_t* ptr, const int32_t* pts, const int32_t* nbr, const int32_t* cnt,
            int64_t bc, int32_t m, int32_t nmax, const double* theta0, const double* lower,
            const double* upper, const sbv_mle_opts* opts, double* theta_out,
            sbv_mle_result* result, double* hist_u, double* hist_l, int64_t hist_cap,
            int64_t* hist_len, void* stream);

/* Surrogate proposals for restarts (no counterpart in the paper). */
typedef struct {
  int32_t exact_starts;  /* starts run from their given point before proposals (4) */
  int32_t train_steps;   /* Adam steps of each fit, from the network's initial parameters (4000) */
  int32_t batch;         /* rows per Adam step (512) */
  float lr;              /* Adam step size (1e-3) */
  int32_t ascent_starts; /* points of the gradient ascent on the network (256) */
  int32_t ascent_iters;  /* sign-gradient steps of 1/200 of the data's box (300) */
  int32_t candidates;    /* distinct maximisers judged by the exact likelihood at a restart
                            (8; 0: restarts run from their given point) */
  double ascent_radius;  /* ascent points drawn uniformly within this max-norm radius (1.0) */
  uint64_t seed;         /* SplitMix64 seed of those draws and of the mini-batches (1) */
  int32_t step_candidates; /* network maximisers added to every line-search call (2; 0: none) */
  double step_radius;    /* initial trust radius of those, max-norm in log theta (0.5); it
                            doubles up to ascent_radius when a proposal wins the call and
                            halves down to step_radius / 64 when none does */
  int32_t refit_every;   /* accepted iterations between refits inside the loop (10) */
} sbv_surrogate_opts;

/*
 * sbv_mle_multistart -- sbv_mle from each of S starts (host, S x (2 + d)) in
 * turn, sharing one history of exact evaluations.  With mlp == NULL every
 * start runs from its given point.  With a network (in_dim = 2 + d), start
 * i >= exact_starts first fits the network to the standardised history
 * (inputs: log theta per coordinate, target: l), climbs it from
 * `ascent_starts` points around start i, and evaluates the best distinct
 * `candidates` maximisers together with start i in one exact call; BFGS then
 * runs from the best of them.  Inside BFGS (starts i >= exact_starts) every
 * line-search call also evaluates `step_candidates` maximisers of the
 * network within the trust radius of the iterate (the network refitted to
 * the grown history every `refit_every` accepted iterations); the best exact
 * value of the call is the next iterate, whichever row it is.  theta_out
 * (S x (2 + d)) and results (S) report each start; results[i].evals includes
 * the proposal rows.  The network keeps its last fit.  sopts may be NULL
 * (defaults above).  prior_u (host, prior_n x (2 + d), log theta) and
 * prior_l (prior_n) are (log theta, l) pairs of earlier runs on the same
 * problem (sbv_mle's history): they join the history before the first start
 * and train the network like this call's own pairs; they are not counted in
 * results[i].evals.  prior_n = 0 with NULL pointers for none; SBV_EINVAL for
 * prior_n < 0 or missing pointers.
 */
int sbv_mle_multistart(sbv_ctx* ctx, const void* X, int dtype, const double* y, int64_t n,
                       int32_t d, const int64_t* ptr, const int32_t* pts, const int32_t* nbr,
                       const int32_t* cnt, int64_t bc, int32_t m, int32_t nmax,
                       const double* starts, int32_t S, const double* lower,
                       const double* upper, const sbv_mle_opts* opts, sbv_mlp* mlp,
                       const sbv_surrogate_opts* sopts, const double* prior_u,
                       const double* prior_l, int64_t prior_n, double* theta_out,
                       sbv_mle_result* results, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SBV_H */
