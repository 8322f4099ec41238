/*
 * tucker.h - C ABI of the GB300 sketched Tucker core-update library (libtucker.so).
 *
 * The library implements the core-tensor step of regularised Tucker ALS from
 * "Fast Low-Rank Tensor Decomposition by Ridge Leverage Score Sampling"
 * (Fahrbach, Ghadiri, Fu): the ridge regression
 *
 *     argmin_g || K g - vec(X) ||_2^2 + lambda ||g||_2^2,
 *     K = A^(1) (x) A^(2) (x) ... (x) A^(N)                    (Alg. 2, core line)
 *
 * solved either exactly (the plain method) or on a row sketch of K drawn from
 * the product of the factor leverage-score distributions (Alg. 3 -> Alg. 1).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Layout: tensors are row-major with the LAST index fastest; the linear
 *    index of (i_1..i_N) is ((i_1*I_2 + i_2)*I_3 + i_3)...  A factor A^(n) is
 *    an I_n x R_n row-major matrix.  vec(G) of the core uses the same row-major
 *    order over (r_1..r_N), which is the column order of K.  (The paper writes
 *    vec as column stacking; only row-major vec makes K = A^(1) (x) ... (x)
 *    A^(N) consistent, so row-major is used throughout.)
 *  - Pointers: every array argument is a DEVICE pointer owned by the caller
 *    unless the parameter name ends in _host.  The library never frees caller
 *    memory.  Device arrays must be aligned to their element size.
 *  - Streams: every call enqueues work on the handle's stream.  Calls that
 *    return host values (counts, ranks, losses, statistics) synchronise that
 *    stream before returning; the others are asynchronous unless the handle
 *    is in synchronous-status mode (the default, see tucker_set_sync).
 *  - Errors: functions return a tucker_status; they never abort, trap or
 *    print.  tucker_last_error() gives a one-line message for the last failure
 *    on a handle.  Errors found on the device (non-SPD pivot, draw limit, hash
 *    probe limit) are reported by the call that launched the work when the
 *    handle is in synchronous-status mode, else by tucker_sync().
 *  - Determinism: the same inputs, seed and sweep give bit-identical sampled
 *    keys, counts and probabilities, equal to the CPU oracle's given the same
 *    leverage scores.
 *  - Thread safety: a handle is used by one host thread at a time.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TUCKER_MAX_ORDER 8
#define TUCKER_MAX_RANK 64      /* per-mode rank limit R_n */

typedef enum {
  TUCKER_OK = 0,
  TUCKER_EINVAL = 1,      /* invalid argument: shape, rank, dtype, null pointer, lambda */
  TUCKER_ENOMEM = 2,      /* device allocation of the handle's workspace failed */
  TUCKER_ECUDA = 3,       /* a CUDA runtime call failed (message in tucker_last_error) */
  TUCKER_ENOTSPD = 4,     /* Cholesky met a non-positive pivot: G + lambda*reg is not SPD */
  TUCKER_ERANK = 5,       /* a factor has zero total leverage (e.g. an all-zero factor) */
  TUCKER_EDRAWLIMIT = 6,  /* missing-entry sampling used max_draws before m accepted */
  TUCKER_EHASHFULL = 7,   /* observed-entry hash table exceeded its probe limit */
  TUCKER_ECAPACITY = 8,   /* a caller-provided output array is too small */
  TUCKER_ENOTSUP = 9,     /* combination not supported by the library (e.g. no sm_103a GPU) */
  TUCKER_EINTERNAL = 10   /* a device-side consistency check failed */
} tucker_status;

typedef enum { TUCKER_F32 = 0, TUCKER_F64 = 1 } tucker_dtype;

/* Arithmetic of the sketched Gram G = sum_u w_u k_u k_u^T (and of the exact
 * missing-entry Gram).  The right-hand side h, the Cholesky factorisation of
 * G + lambda*I and the iterative-refinement residual are FP64 in every mode.
 * With a reduced-precision Gram the Cholesky factor of the rounded Gram is a
 * preconditioner: g <- g + M~^-1 (h - M g) with M g evaluated in FP64 on the
 * implicit rows.  With c_k = ||correction_k|| / ||g|| (c_0 = 1) and the
 * contraction estimate rho = min(c_k / c_{k-1}, 1/2), the iteration stops once
 * the estimated remaining relative error c_k rho / (1 - rho) is below 1e-8, or
 * when the corrections stop shrinking, at most 8 iterations.  With a BF16
 * Gram (and a TF32 one under the factor solvers) at least two corrections are
 * always made; when the factors are FP32 the first of them evaluates its
 * residual in FP32 (it only has to be as accurate as the Gram's rounding),
 * every later one in FP64.  Under TUCKER_SOLVER_KRON_PCG a TF32 or FP32 Gram
 * starts with an FP64 correction (one suffices at TF32's rounding).
 * TF32/BF16 operands: each sampled row k_u = sqrt(w_u) a_1 (x) ... (x) a_N is
 * formed in FP32 and rounded once.  For order >= 3 with R_1 a power of two
 * <= 16 the Gram is grouped by the leading index instead when d / R_1 >= 128
 * or (d / R_1 <= 64, at least two sampled rows per value of i_1) (G = sum_{i_1}
 * (a a^T) (x) M_{i_1}, a = A^(1)[i_1], the rows of one i_1 adjacent in the
 * key-sorted sample).  Wide M_{i_1}: the tensor cores form each from the
 * rounded rows sqrt(w_u) a_2 (x) ... (x) a_N, and the expansion by a_{r1} a_{r1'}
 * runs on the tensor cores with both operands split into TF32 hi + lo parts.
 * Narrow M_{i_1} (d / R_1 <= 64): the tensor cores form each from rows split
 * into TF32 hi + lo parts (an FP32-level Gram, for either tensor-core
 * precision), and the expansion runs in FP32 on the CUDA cores.  Either way G
 * is FP32-accumulated and stored as FP64. */
typedef enum {
  TUCKER_PREC_FP64 = 0,   /* FP64 CUDA-core Gram; no refinement needed */
  TUCKER_PREC_FP32 = 1,   /* FP32 CUDA-core Gram, FP64 refinement */
  TUCKER_PREC_TF32 = 2,   /* tcgen05 TF32 tensor-core Gram, FP32 accumulate, FP64 refinement */
  TUCKER_PREC_BF16 = 3    /* tcgen05 BF16 tensor-core Gram, FP32 accumulate, FP64 refinement */
} tucker_prec;

/* How (G + lambda R) g = h is solved (Eq. problem_def; Appendix B, proof of
 * Thm 4.2).  Both return the FP64 solution to the tolerances stated for
 * tucker_prec; they differ in what the O(d^3) factorisation runs in.
 *   FP64_CHOLESKY  the factorisation is FP64 (default).  With an FP64 Gram
 *                  the solve is direct; with a reduced-precision Gram the
 *                  FP64 factor preconditions the refinement described above.
 *   MIXED          the factorisation and triangular solves are FP32 and only
 *                  precondition an FP64 iterative refinement,
 *                  g <- g + L32^-T L32^-1 (h - M g), with the residual h - M g
 *                  in FP64 (the explicit FP64 M for TUCKER_PREC_FP64; the
 *                  implicit FP64 rows otherwise).  It stops by the rule above
 *                  with a target of 1e-13 for an FP64 Gram (1e-8 otherwise),
 *                  at most 12 iterations.  It converges when kappa(M) * 2^-24 is
 *                  well below 1; lambda > 0 keeps kappa(M) <= (||G|| +
 *                  lambda)/lambda.  A matrix that FP32 cannot factor (a
 *                  pivot <= 0 after rounding, or below the smallest normal
 *                  FP32 value) returns TUCKER_ENOTSPD.
 *   KRON_PCG       no factorisation: the solves inside the same FP64
 *                  refinement are conjugate gradients on the rounded Gram
 *                  M~ = G~ + lambda R (FP32), preconditioned by
 *                  P = (x) V_n diag(s (x) ev_n + lbar) (x) V_n^T, where
 *                  A^(n)T A^(n) = V_n diag(ev_n) V_n^T, s = tr(G~) /
 *                  prod_n tr(A^(n)T A^(n)) and lbar = mean(lambda R).  The
 *                  sketched Gram estimates K^T K = (x) A^(n)T A^(n) without
 *                  bias (Thm A.3), so P is spectrally close to M~ and CG needs
 *                  a few iterations (each one product with M~ and 2 d sum R_n
 *                  multiply-adds for P^-1) instead of a d^3 / 3 factorisation.
 *                  Each solve stops at a relative residual of 1e-4 (BF16
 *                  Gram) or 1e-5 (TF32, FP32), at most 50 iterations; the
 *                  refinement stops by the rule above with a target of 1e-8.  If the refinement does not reach that
 *                  target (a sketch far from K^T K, e.g. a strongly
 *                  non-uniform observation mask), the call factors M~ as the
 *                  MIXED solver does and solves again, so the result meets
 *                  the same tolerances.  With an FP64 Gram (TUCKER_PREC_FP64)
 *                  this solver behaves as FP64_CHOLESKY.  The adjoint reuses
 *                  M~ and the V_n of the forward call. */
typedef enum {
  TUCKER_SOLVER_FP64_CHOLESKY = 0,
  TUCKER_SOLVER_MIXED = 1,
  TUCKER_SOLVER_KRON_PCG = 2
} tucker_solver;

/* How the lambda*I term enters the sketched problem. */
typedef enum {
  /* sketch only the rows of K and add lambda*I exactly: solve (G + lambda I) g = h */
  TUCKER_REG_EXACT = 0,
  /* Alg. 1 with d'_eff = 0: sample from the augmented distribution D(l(K), 0)
   * of Sec. 3 over the rows of [K; sqrt(lambda) I]; a coin picks a row of K
   * (mass l(K), normalised to d) or one of the d regulariser rows (mass 1
   * each); the sampled regulariser rows give lambda*diag(D) in place of
   * lambda*I */
  TUCKER_REG_AUGMENTED = 1,
  /* rows drawn from the lambda-ridge leverage distribution of K itself,
   * l^lam(K) / d_eff(K) (Lemma 4.1 with lambda > 0; see tucker_ridge_tables),
   * lambda*I added exactly; dense X only.  With m = 0 the sample count is
   * Alg. 1 line 3's s with beta' of Eq. beta_prime for these exact scores:
   * beta' = d / (d_eff + d min{1, d - d_eff}) (1/2 <= beta' <= 1), so fewer
   * rows are drawn as lambda grows and d_eff(K) shrinks. */
  TUCKER_REG_RIDGE = 2
} tucker_reg;

/* The data tensor X of the problem statement (Sec. 2): either dense or a list
 * of observed entries (Sec. 4.2, missing data).  Exactly one of `dense` and
 * (`keys`,`vals`) is non-NULL. */
typedef struct {
  int order;                        /* N, 1 <= N <= TUCKER_MAX_ORDER */
  int64_t dims[TUCKER_MAX_ORDER];   /* I_1..I_N; prod(I_n) < 2^62 */
  tucker_dtype dtype;               /* element type of dense / vals (and of the factors) */
  const void* dense;                /* device, prod(I_n) elements row-major, or NULL */
  int64_t nnz;                      /* number of observed entries (COO) */
  const uint64_t* keys;             /* device [nnz]: row-major linear indices, strictly increasing
                                       (a precondition, not checked: the row walks and the
                                       leading-index-grouped Gram rely on the order) */
  const void* vals;                 /* device [nnz]: entry values, dtype */
} tucker_tensor;

/* A deduplicated row sample of K (or of [K; sqrt(lambda) I]).  Caller-owned
 * device arrays of length `capacity`; n_unique and n_draws are written by
 * tucker_sample_rows and read by tucker_core_update_sketched when the sample
 * is passed back in (a frozen sketch, used for finite differences and the
 * adjoint). */
typedef struct {
  int64_t capacity;     /* length of keys / counts / prob */
  int64_t n_unique;     /* number of distinct sampled rows, sorted ascending by key (a
                           sample passed back in must keep that order; not checked) */
  int64_t n_draws;      /* T: draws used (= m when dense; more when entries are missing) */
  uint64_t* keys;       /* row key: linear row index of K, or prod(I)+j for regulariser row j */
  uint32_t* counts;     /* multiplicity c_u of each distinct row among the accepted draws */
  double* prob;         /* sampling probability p_u of the row (weights are c_u/(T p_u)) */
} tucker_samples;

/* Per-call statistics (host struct, optional). Times are CUDA-event
 * milliseconds per stage on the handle's stream. */
typedef struct {
  double ms_leverage, ms_sample, ms_dedupe, ms_gather, ms_gram, ms_solve, ms_total;
  int64_t n_unique;     /* distinct rows in the sketch */
  int64_t n_draws;      /* T */
  int64_t n_real;       /* distinct rows of K (the rest are regulariser rows) */
  int refine_iters;     /* refinement iterations used (tensor-core precisions) */
  double refine_rel;    /* last ||correction|| / ||g|| of the refinement */
  uint64_t solve_id;    /* identifies the cached Cholesky factor for the adjoint */
  int64_t launches;     /* CUDA kernels this call launched */
  double ms_factor;     /* the Cholesky factorisation kernel alone (inside ms_solve) */
  double ms_gram_kernel;/* the Kronecker SYRK kernel alone (inside ms_gram) */
  double ms_inner;      /* TUCKER_SOLVER_KRON_PCG: the first CG solve alone (inside ms_solve) */
  int64_t inner_iters;  /* TUCKER_SOLVER_KRON_PCG: CG iterations over all solves of the call;
                           negative when the CG refinement missed its target and the FP32
                           factor solved instead */
  int gram_prec_used;   /* the Gram precision that solved: `prec`, or TUCKER_PREC_FP32 /
                           TUCKER_PREC_FP64 when a rounded Gram or an FP32 factor met a
                           non-positive pivot and the Gram was formed again on the CUDA
                           cores with an FP64 factor */
} tucker_stats;

typedef struct tucker_handle tucker_handle;

/* Create a handle bound to the current CUDA device and `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream).  The handle owns its
 * device workspace (grown on demand), the observed-entry hash table and the
 * cached Cholesky factor of the last sketched solve.
 * Errors: EINVAL (h NULL), ENOTSUP (no sm_103 device), ECUDA. */
tucker_status tucker_create(tucker_handle** h, void* cuda_stream);

/* Release the handle and all device memory it owns (synchronises its stream). */
tucker_status tucker_destroy(tucker_handle* h);

/* One-line description of the last error on h (never NULL; "" if none). */
const char* tucker_last_error(const tucker_handle* h);

/* 1 (default): calls that launch device work synchronise and return
 * device-detected errors.  0: calls return after enqueueing; device errors
 * are returned by the next tucker_sync(). */
tucker_status tucker_set_sync(tucker_handle* h, int synchronous);

/* Select the ridge solver of later core updates and adjoints on h
 * (TUCKER_SOLVER_FP64_CHOLESKY by default).  Invalidates the cached factor.
 * Errors: EINVAL (h NULL or an unknown solver). */
tucker_status tucker_set_solver(tucker_handle* h, tucker_solver solver);

/* Wait for the handle's stream and return any pending device-side error. */
tucker_status tucker_sync(tucker_handle* h);

/* Statistical leverage scores of each factor (Alg. 3 line 1; Eq.
 * ridge_leverage_score_def with lambda = 0):
 *     l_i(A^(n)) = a_i (A^(n)T A^(n))^+ a_i^T,
 * the pseudo-inverse through a Jacobi eigendecomposition of the R_n x R_n Gram
 * in FP64, eigenvalues <= max(I_n,R_n) * 2^-52 * lambda_max treated as zero.
 *   N, I[N], R[N]   host arrays: order, dims, ranks (R_n <= TUCKER_MAX_RANK)
 *   dtype           element type of the factors
 *   A[N]            host array of device pointers to the I_n x R_n factors
 *   lev_out[N]      host array of device pointers, FP64 [I_n] each
 *   cdf_out[N]      nullable; device uint64 [I_n] each: the inclusive prefix
 *                   sums C of q_i = floor(clamp(l_i,0,1) * 2^32) used by the sampler
 *   rank_out_host   nullable host int[N]: numerical rank of each factor
 * Synchronises when rank_out_host is given.  Errors: EINVAL, ERANK. */
tucker_status tucker_leverage_scores(tucker_handle* h, int N, const int64_t* I, const int* R,
                                     tucker_dtype dtype, const void* const* A,
                                     double* const* lev_out, uint64_t* const* cdf_out,
                                     int* rank_out_host);

/* Draw m rows of K from the product distribution of the factor leverage
 * scores (Lemma 4.1 at lambda = 0; Alg. 3 line 3; Alg. 1 sampling loop) and
 * deduplicate them.  Draw t uses Philox4x64-10 with key (seed, sweep) and
 * counter (t, s, 0, 0); mode n takes word n%4 of stream s = n/4 as a 64-bit
 * uniform u and picks i_n = min{i : C_i > floor(u Q_n / 2^64)}.  With
 * TUCKER_REG_AUGMENTED the top bit of word 0 of stream 2 chooses a
 * regulariser row j = floor(u' d / 2^64) (u' = word 1 of stream 2), key
 * prod(I)+j.  With `observed` (COO), a draw whose key is not observed is
 * rejected; draws continue in counter order until m are accepted (regulariser
 * rows are always accepted).
 *   lev[N]          device FP64 [I_n] leverage scores (e.g. from tucker_leverage_scores)
 *   m               accepted draws, 1 <= m < 2^31
 *   observed        NULL (dense) or a COO tucker_tensor whose keys define Omega
 *   max_draws       limit on T in missing mode (0 = 64*m)
 *   out             caller arrays of capacity >= m; n_unique/n_draws written
 * Synchronises.  Errors: EINVAL, ERANK (sum of q is 0), EDRAWLIMIT, EHASHFULL,
 * ECAPACITY. */
tucker_status tucker_sample_rows(tucker_handle* h, int N, const int64_t* I, const int* R,
                                 const double* const* lev, int64_t m, uint64_t seed,
                                 uint32_t sweep, tucker_reg reg, const tucker_tensor* observed,
                                 int64_t max_draws, tucker_samples* out);

/* FastCoreTensorUpdate (Alg. 3 -> Alg. 1): sketched core update.
 * Builds rows k_u = A^(1)[i_1] (x) ... (x) A^(N)[i_N] of the sampled rows on
 * the fly (K is never formed), accumulates G = sum_u w_u k_u k_u^T and
 * h = sum_u w_u x_u k_u with w_u = c_u / (T p_u) (Appendix B, proof of Thm 4.2:
 * normal equations as outer products), and solves (G + lambda R) g = h by an
 * FP64 Cholesky factorisation, R = I or the sampled regulariser diagonal.
 *   X               dense or COO tensor (dtype F32 or F64; factors share it)
 *   R[N]            host ranks; d = prod(R_n) <= 8192
 *   A[N]            host array of device factor pointers
 *   lambda          >= 0 (> 0 required for TUCKER_REG_AUGMENTED)
 *   m               sample count; 0 = the paper's s of Alg. 1 line 3 at
 *                   (eps, delta): beta' = 1/2 for a dense X; for observed
 *                   entries the beta' of tucker_missing_beta's bound mode (lambda
 *                   > 0; EINVAL when that s is 2^31 or more)
 *   seed, sweep     Philox key (the sweep index keeps resumed runs identical)
 *   fixed           NULL, or a sample from tucker_sample_rows to reuse (frozen sketch)
 *   core_out        device FP64 [d]: vec(G) row-major
 *   stats_host      nullable; filled (and the stream synchronised) when given
 * Errors: EINVAL, ERANK, ENOTSPD, EDRAWLIMIT, EHASHFULL, ENOMEM, ECUDA. */
tucker_status tucker_core_update_sketched(tucker_handle* h, const tucker_tensor* X, const int* R,
                                          const void* const* A, double lambda, int64_t m,
                                          double eps, double delta, uint64_t seed, uint32_t sweep,
                                          tucker_reg reg, tucker_prec prec,
                                          const tucker_samples* fixed, double* core_out,
                                          tucker_stats* stats_host);

/* Exact core update, the plain method (Alg. 2, core line).
 * Dense X: K^T K + lambda I = (x V_n)(x S_n^2 + lambda)(x V_n)^T (proof of
 * Lemma 4.1), so g = (x V_n)[(x V_n)^T (X x_1 A^(1)T ... x_N A^(N)T)] /
 * (x S_n^2 + lambda): one streaming pass over X for the n-mode product chain,
 * Jacobi eigendecompositions of the R_n x R_n Grams, and small mode products.
 * COO X: the Gram of all observed rows sum_{i in Omega} k_i k_i^T (with
 * `prec`) and sum x_i k_i, then the FP64 Cholesky solve (+ refinement for
 * tensor-core precisions).
 *   core_out        device FP64 [d]
 * Errors: EINVAL, ENOTSPD, ENOMEM, ECUDA. */
tucker_status tucker_core_update_exact(tucker_handle* h, const tucker_tensor* X, const int* R,
                                       const void* const* A, double lambda, tucker_prec prec,
                                       double* core_out);

/* One pass of the repeat loop of Alg. 2: factor updates n = 1..N (each row a
 * ridge regression with design G_(n) ((x)_{k!=n} A^(k))^T), then the core
 * update (sketched when `sketched`, else exact).  Dense X only.
 *   A_inout[N]      device factors (dtype of X), updated in place
 *   core_inout      device FP64 [d], updated in place
 *   loss_out_host   nullable: L = ||X - X-hat||^2 + lambda(||G||^2 + sum ||A^(n)||^2) (Sec. 2),
 *                   by the Gram identity ||X - X-hat||^2 = ||X||^2 - 2 g.K^T vec(X) +
 *                   g.((x)_n A^(n)T A^(n)) g in FP64: K^T vec(X) from the last factor
 *                   update's n-mode product chain, ||X||^2 in one pass (FP32 data:
 *                   error-free squares and compensated FP32 sums, added in FP64).
 *                   The identity cancels ||X||^2 down to the residual: its relative
 *                   accuracy is about 1e-13 times ||X||^2 / ||X - X-hat||^2 (2e-8 for
 *                   a 512^3 tensor with 5e-6 of its energy in the residual);
 *                   tucker_ridge_loss sums the residual entry by entry instead
 *   rmse_out_host   nullable: sqrt(||X - X-hat||^2 / prod(I_n)), the same identity
 * Errors: EINVAL, ENOTSPD, ENOMEM, ECUDA. */
tucker_status tucker_als_sweep(tucker_handle* h, const tucker_tensor* X, const int* R,
                               void* const* A_inout, double* core_inout, double lambda,
                               int sketched, int64_t m, uint64_t seed, uint32_t sweep,
                               tucker_reg reg, tucker_prec prec, double* loss_out_host,
                               double* rmse_out_host);

/* Ridge loss of a core for the current factors (the objective of Alg. 2's
 * core line): ||K g - vec(X)||^2 + lambda ||g||^2 over all entries (dense) or
 * the observed entries (COO), evaluated entry by entry in FP64.
 *   g               device FP64 [d]
 *   loss_out_host   host double
 * Synchronises.  Errors: EINVAL, ECUDA. */
tucker_status tucker_ridge_loss(tucker_handle* h, const tucker_tensor* X, const int* R,
                                const void* const* A, double lambda, const double* g,
                                double* loss_out_host);

/* Normal equations of a given sample (Appendix B, proof of Thm 4.2: the
 * sketched A^T A and A^T b as sums of outer products over the sampled rows):
 *     G = sum_u w_u k_u k_u^T,   h = sum_u w_u x_u k_u,   w_u = c_u / (T p_u),
 * over the rows of K in the sample (regulariser rows are skipped), with the
 * Gram arithmetic of `prec` (no refinement) and h in FP64.
 *   samples         a sample from tucker_sample_rows (keys, counts, prob, T)
 *   G_out           device FP64 d x d, row-major, both triangles written
 *   h_out           nullable device FP64 [d]
 * Errors: EINVAL, ENOTSUP, ECUDA. */
tucker_status tucker_sketched_gram(tucker_handle* h, const tucker_tensor* X, const int* R,
                                   const void* const* A, tucker_prec prec,
                                   const tucker_samples* samples, double* G_out, double* h_out);

/* Adjoint (reverse-mode derivative) of the sketched solve g = M^-1 h with
 * M = sum_u w_u k_u k_u^T + lambda R and h = sum_u w_u x_u k_u, the sample
 * (keys, counts, p) held fixed.  For a cotangent gbar:
 *     v = M^-1 gbar                  (reuses the cached Cholesky factor when
 *                                     solve_id names the last sketched solve,
 *                                     else refactorises M)
 *     dx_u = w_u (k_u . v)
 *     dA^(n)[i_n, r_n] += sum_{r : r_n} w_u (x_u v - (k_u.g) v - (k_u.v) g)[r]
 *                                      * prod_{m != n} A^(m)[i_m, r_m]
 *   X               the tensor of the forward call (x_u are gathered from it)
 *   samples         the frozen sample of the forward call
 *   g               device FP64 [d] forward result; gbar device FP64 [d]
 *   dA_out[N]       device FP64 I_n x R_n each (overwritten)
 *   dx_out          device FP64 [samples->n_unique] (0 for regulariser rows)
 * Errors: EINVAL, ENOTSPD, ECUDA. */
tucker_status tucker_core_solve_adjoint(tucker_handle* h, const tucker_tensor* X, const int* R,
                                        const void* const* A, double lambda, tucker_reg reg,
                                        tucker_prec prec, const tucker_samples* samples,
                                        uint64_t solve_id, const double* g, const double* gbar,
                                        double* const* dA_out, double* dx_out);

/* Tables of the lambda-ridge leverage distribution of K (Lemma 4.1 with
 * lambda > 0; Eq. d_eff_def).  With the thin SVDs A^(n) = U^(n) S^(n) V^(n)T
 * (from the Jacobi eigendecomposition of A^(n)T A^(n), eigenpairs in
 * decreasing order, K_n = min(I_n, R_n) of them, squared singular values at
 * or below max(I_n, R_n) 2^-52 times the largest counted as zero):
 *     l^lam_i(K) = sum_t c_t prod_n usq_n[t_n][i_n],
 *     usq_n[t][i] = (u^(n)_{i t})^2,   c_t = P_t / (P_t + lambda),
 *     P_t = prod_n s^2_{t_n}(A^(n)),   d_eff(K) = sum_t c_t.
 *   usq_out[N]      host array of device pointers, FP64 K_n x I_n each
 *                   (column t contiguous; 0 for a component cut to zero)
 *   c_out           device FP64 [prod K_n], row-major over (t_1 .. t_N)
 *   K_out_host      nullable host int[N]: K_n
 *   d_eff_out_host  nullable: d_eff(K) (synchronises)
 * Errors: EINVAL. */
tucker_status tucker_ridge_tables(tucker_handle* h, int N, const int64_t* I, const int* R,
                                  tucker_dtype dtype, const void* const* A, double lambda,
                                  double* const* usq_out, double* c_out, int* K_out_host,
                                  double* d_eff_out_host);

/* Draw m rows of K from l^lam(K) / d_eff(K) given its tables (the mixture
 * over components t with weights c_t of the product distributions
 * prod_n usq_n[t_n][.]) and deduplicate them.  Fixed-point weights
 * q = floor(clamp(x, 0, 1) 2^32) of c (one CDF, row-major over t) and of each
 * column usq_n[t] (one CDF each); draw t takes its component from word 0 of
 * Philox4x64-10 stream 3 (counter (t, 3, 0, 0), key (seed, sweep)) and its
 * index in mode n from word n%4 of stream n/4, each by
 * min{i : C_i > floor(u Q / 2^64)}.  prob[u] is the exact probability of the
 * row under that arithmetic, sum_t (q^c_t / Q^c) prod_n (q^(n,t_n)_{i_n} /
 * Q^(n,t_n)) in row-major order of t (FP64).  T = m.
 *   K[N]            host: components per mode (1 <= K_n <= min(I_n, 64))
 *   usq[N], c       device tables as written by tucker_ridge_tables
 *   out             caller arrays of capacity >= m; n_unique/n_draws written
 * Synchronises.  Errors: EINVAL, ERANK (every c_t is 0), ECAPACITY. */
tucker_status tucker_sample_rows_ridge(tucker_handle* h, int N, const int64_t* I, const int* K,
                                       const double* const* usq, const double* c, int64_t m,
                                       uint64_t seed, uint32_t sweep, tucker_samples* out);

/* Sketched factor update of mode n (this library's extension of Alg. 2's
 * factor step; the paper updates the factors exactly).  The factor update is
 * the ridge regression min ||B_n A^T - X_(n)^T||^2 + lambda ||A||^2 with the
 * design B_n = W G_(n)^T, W = (x)_{k != n} A^(k), whose rows are indexed
 * row-major by the multi-index over the modes k != n.  Its rows lie in the
 * column space of W, so l_j(B_n) <= prod_{k != n} l_{j_k}(A^(k)) (Lemma 4.1 at
 * lambda = 0): the product distribution of the other modes' leverage scores is
 * an (R_n / prod_{k != n} R_k)-overestimate, and Alg. 1's sketch applies with
 * B_n in place of K.  m draws use the core sampler's arithmetic over the modes
 * k != n with Philox key (seed, sweep + (n + 1) 2^32) (apart from the core
 * sampler's (seed, sweep)); after the dedupe, with w_u = c_u / (m p_u),
 *     M = sum_u w_u b_u b_u^T + lambda I,   Y = sum_u w_u x_u b_u^T,   A^(n) = Y M^-1,
 * b_u = G_(n) (x)_{k != n} A^(k)[j_k] and x_u the mode-n fiber of X at row u
 * (I_n strided reads).  The fibers and Y are in X's element type (FP32 or
 * FP64) summed in a fixed order; b_u, M and its inverse in FP64.
 *   X               dense tensor (order >= 2)
 *   A_inout[N]      device factors; A_inout[n] is overwritten
 *   core            device FP64 [d], vec(G) row-major
 *   n               the mode, 0 <= n < N
 *   m               draws, 1 <= m < 2^31
 * Errors: EINVAL, ENOTSPD, ECUDA. */
tucker_status tucker_factor_update_sketched(tucker_handle* h, const tucker_tensor* X, const int* R,
                                            void* const* A_inout, const double* core, int n,
                                            double lambda, int64_t m, uint64_t seed,
                                            uint32_t sweep);

/* Sketched factor update of regularised CP-ALS: the extension to L2-regularised
 * CP decompositions that Sec. 6 notes, with the Khatri-Rao design overestimated
 * by Kronecker leverage scores as the remark in Sec. 4 recalls.  The rank-R CP
 * model is X_hat = sum_r a_1[:, r] o ... o a_N[:, r]; the mode-n update is the
 * ridge regression min ||Z_n A^T - X_(n)^T||^2 + lambda ||A||^2 with the design
 * Z_n whose row for the multi-index over the modes k != n (row-major, last
 * fastest) is the Hadamard product of A^(k)[j_k, :].  Z_n's columns are columns
 * of (x)_{k != n} A^(k), so l_j(Z_n) <= prod_{k != n} l_{j_k}(A^(k)) and the
 * product distribution of the other modes' leverage scores is an
 * (R / prod_{k != n} rank A^(k))-overestimate.  The draws, dedupe, weights and
 * normal equations are those of tucker_factor_update_sketched with z_u (the
 * Hadamard row, FP64, modes in increasing order) in place of b_u:
 *     M = sum_u w_u z_u z_u^T + lambda I,   Y = sum_u w_u x_u z_u^T,   A^(n) = Y M^-1.
 *   X               dense tensor (order >= 2), FP32 or FP64
 *   R               CP rank, 1 <= R <= TUCKER_MAX_RANK
 *   A_inout[N]      device factors I_n x R (X's dtype); A_inout[n] is overwritten
 *   n, m, seed, sweep, lambda: as for tucker_factor_update_sketched (Philox key
 *                   word sweep + (n + 1) 2^32)
 * Errors: EINVAL, ENOTSPD, ECUDA. */
tucker_status tucker_cp_factor_update_sketched(tucker_handle* h, const tucker_tensor* X, int R,
                                               void* const* A_inout, int n, double lambda,
                                               int64_t m, uint64_t seed, uint32_t sweep);

/* One sweep of regularised CP-ALS: tucker_cp_factor_update_sketched for the
 * modes n = 0 .. N-1 in turn, m draws each, every update using the factors the
 * earlier ones wrote.  Returns no loss (the library does not form the CP model).
 * Errors: as tucker_cp_factor_update_sketched. */
tucker_status tucker_cp_als_sweep(tucker_handle* h, const tucker_tensor* X, int R,
                                  void* const* A_inout, double lambda, int64_t m, uint64_t seed,
                                  uint32_t sweep);

/* m > 0: the factor updates of later tucker_als_sweep calls on h are
 * tucker_factor_update_sketched with m draws each (key word sweep + (n+1) 2^32);
 * 0 (the default): exact factor updates.  With sketched factor updates the
 * sweep forms the product chain X x_{k<N} A^(k)T once more for its loss.
 * Errors: EINVAL (h NULL, m < 0 or m >= 2^31). */
tucker_status tucker_set_factor_sketch(tucker_handle* h, int64_t m);

/* Overestimate factor of the observed-entry sampler (Sec. 4.2, missing data).
 * With S the observed rows of K, S-bar the missing ones and
 * L = K (K^T K + lambda I)^+ K^T the cross lambda-ridge scores of K, the ridge
 * scores of K restricted to S are a beta_miss-overestimate of the ridge scores
 * of K_S (Thm 4.3 with the lemma on sums of squared cross scores), where
 *     1 / beta_miss = 1 + 1 / (1 - lambda_max(L_{S-bar,S-bar})).
 * Modes:
 *   TUCKER_BETA_BOUND  the corollary to Thm 4.3: lambda_max <= P / (P + lambda),
 *                      P = prod_n ||A^(n)||_2^2 (the largest eigenvalue of each
 *                      A^(n)T A^(n), FP64 Jacobi), so beta_miss >= 1 / (2 + P / lambda);
 *   TUCKER_BETA_EXACT  lambda_max = 1 - nu_min, nu_min the smallest eigenvalue of
 *                      the pencil (K_S^T K_S + lambda I, K^T K + lambda I).  The
 *                      Gram of all observed rows is formed in `prec` (as the exact
 *                      observed-entry update forms it) and whitened with the
 *                      factor eigendecompositions, D^-1/2 Vk^T (G + lambda I) Vk D^-1/2
 *                      (Vk = (x)_n V_n, D = (x)_n ev_n + lambda); nu_min is estimated
 *                      by inverse iteration on an FP64 Cholesky factor (every
 *                      estimate is at or above nu_min) and then certified from
 *                      below: the first nu (1 - tau), tau = 1e-6, 1e-4, 1e-2, 0.1,
 *                      0.5, for which the whitened matrix minus nu I has an FP64
 *                      Cholesky factor.  lambda_max = 1 - that nu is an upper bound
 *                      for the Gram as formed.  d <= 4096.  Overwrites the handle's
 *                      cached factor (a later adjoint call factors again).
 * A dense X has nothing missing: lambda_max = 0, beta_miss = 1.
 * The observed-entry sampler draws from the classical scores of K and rejects
 * unobserved rows; on S its distribution is a beta-overestimate of the ridge
 * scores of K_S with beta = c_min beta_miss, where c_min = min_t c_t over the
 * components with P_t > 0 (by Lemma 4.1 every classical score of K is at most
 * l^lam_i(K) / c_min).  Alg. 1 line 2 with d'_eff = 0 gives
 * beta' = min{beta, 1} / 2 and line 3 the count s.
 *   X, R, A         as for tucker_core_update_sketched
 *   lambda          > 0 (Thm 4.3)
 *   prec            precision of the observed Gram (exact mode only)
 *   eps, delta      in (0, 1): the accuracy and failure probability of s
 *   out_host        filled on success
 * Synchronises.  Errors: EINVAL, ERANK (a zero factor), ENOTSUP (exact mode
 * with d > 4096), ENOTSPD (the whitened Gram has no Cholesky factor), ECUDA. */
typedef enum { TUCKER_BETA_BOUND = 0, TUCKER_BETA_EXACT = 1 } tucker_beta_mode;

typedef struct {
  double lambda_max;    /* upper bound on lambda_max(L_{S-bar,S-bar}) */
  double beta_miss;     /* 1 / (1 + 1 / (1 - lambda_max)); 1 for a dense X */
  double c_min;         /* min_t c_t, c_t = P_t / (P_t + lambda) */
  double beta;          /* c_min * beta_miss */
  double beta_prime;    /* min{beta, 1} / 2 (Alg. 1 line 2, d'_eff = 0) */
  double s;             /* Alg. 1 line 3 at (eps, delta): may exceed any sample count */
  double nu_est;        /* exact mode: the last inverse-iteration estimate of nu_min */
  int iters;            /* exact mode: inverse iterations */
  int certify_tries;    /* exact mode: Cholesky factorisations of the certification */
} tucker_missing_beta_info;

tucker_status tucker_missing_beta(tucker_handle* h, const tucker_tensor* X, const int* R,
                                  const void* const* A, double lambda, tucker_beta_mode mode,
                                  tucker_prec prec, double eps, double delta,
                                  tucker_missing_beta_info* out_host);

/* ---------------------------------------------------------------------------
 * Allocation-free sampling.  The paper has no counterpart to this entry
 * point; it exists for callers that are not allowed to allocate device memory
 * while they run (code working inside a memory pool it does not own, a
 * process that has reserved or capped all GPU memory up front, a real-time
 * loop where a cudaMalloc could block or fail).  Such callers cannot use a
 * tucker_handle, whose workspace grows on demand.
 *
 * tucker_sample_rows_noalloc computes exactly what tucker_sample_rows
 * computes for a dense tensor (same keys, counts, probabilities, n_unique and
 * n_draws) with the same kernels, but all of its scratch lives in one
 * statically sized device array inside libtucker: TUCKER_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that every GPU which loads the library keeps until the process
 * exits.  The caller still provides the inputs (scores) and the outputs (out).
 *   cuda_stream     cudaStream_t to run on (NULL = legacy default stream);
 *                   the current device must be an sm_103 GPU
 *   N, I, R, lev, m, seed, sweep, reg, out: as for tucker_sample_rows; dense
 *                   mode only (no observed-entry mask, which needs a hash table)
 *   err_host        nullable host buffer of err_len bytes for a one-line message
 * Limits: m is bounded by the scratch size - about 2.5e5 draws for order 3;
 * larger m returns TUCKER_ECAPACITY with the bytes needed in err_host.
 * The first successful call on each device looks up the device address of
 * the array (cudaGetSymbolAddress, with that device current) and caches it; a
 * lookup that failed is retried by the next call.  The call synchronises its
 * stream, so it cannot be made while that stream is capturing a CUDA graph.
 * Every call shares the one array, so calls whose
 * work overlaps on the GPU (two streams, two host threads) race and corrupt
 * each other: serialise them.  Each call clears what must start at zero.
 * Synchronises the stream.  Calls no cudaMalloc, cudaFree or other
 * allocating routine.  Errors: EINVAL (also when prod(I_n) >= 4e18, where
 * linear row keys would wrap, as for tucker_sample_rows), ECAPACITY, ERANK,
 * ENOTSUP, ECUDA. */
#define TUCKER_NOALLOC_SCRATCH_BYTES (16u << 20)

tucker_status tucker_sample_rows_noalloc(void* cuda_stream, int N, const int64_t* I, const int* R,
                                         const double* const* lev, int64_t m, uint64_t seed,
                                         uint32_t sweep, tucker_reg reg, tucker_samples* out,
                                         char* err_host, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_H */
