// C ABI entry points of libtucker (declared in include/tucker.h).
//
// Each entry point validates its arguments on the host, sizes one workspace
// arena, and enqueues the kernel pipeline on the handle's stream:
//   sketched core update (Alg. 3 -> Alg. 1):
//     leverage (+ fixed-point CDF) -> sample keys -> sort + run-length dedupe
//     -> gather x and weights -> Gram G and right-hand side h -> + lambda R
//     -> FP64 Cholesky solve (-> FP64 refinement for tensor-core Grams)
//   exact core update (Alg. 2 core line; Lemma 4.1 proof): TTM chain,
//     factor eigendecompositions, diagonal scaling; or the Gram of all
//     observed rows for missing data
//   ALS sweep (Alg. 2), ridge loss, adjoint of the frozen-sketch solve.
#include <float.h>
#include <math.h>
#include <stdarg.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

namespace tk {

// ------------------------------------------------ launchers from other files
tucker_status hash_ensure(tucker_handle* h, const tucker_tensor* X, int* probes_out);
size_t sample_keys_scratch(const FactorSet& F, bool observed);
tucker_status sample_keys(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                          int64_t m, uint64_t seed, uint64_t sweep, int reg,
                          const tucker_tensor* observed, int64_t max_draws,
                          uint64_t* keys_out, int64_t* d_T, int64_t* T_host, Arena& ar);
tucker_status launch_gather(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                            int reg, const uint64_t* keys_u, const uint32_t* counts,
                            const int* d_nu, const int64_t* d_T, const tucker_tensor* X,
                            int64_t cap, uint32_t* const* idx, double* w, double* x, double* p,
                            float* sw32, int* d_nreal, double* D, const double* p_in,
                            double* ptab, bool tables_ready = false);
tucker_status launch_prob_tables(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                                 double* ptab);
tucker_status launch_cdf_from_lev(tucker_handle* h, int N, const int64_t* I,
                                  const double* const* lev, uint64_t* const* cdf,
                                  bool dep = false);
int gram_simt_splits(tucker_handle* h, int d, int64_t cap);
size_t gram_simt_partial_bytes(int d, int nsplit, int is64);
tucker_status launch_gram_simt(tucker_handle* h, const RowSet& s, int use64, int nsplit,
                               void* partial, double* G);
int axpy_splits(tucker_handle* h, int d, int64_t cap);
tucker_status launch_kron_axpy(tucker_handle* h, const RowSet& s, const double* a,
                               const double* b, double coef, int nsplit, double* partial,
                               const double* base, const double* diag, const double* y,
                               double* out);
tucker_status launch_kron_dot(tucker_handle* h, const RowSet& s, const double* g1,
                              const double* g2, double* z1, double* z2);
tucker_status cholesky(tucker_handle* h, double* M, int d);
tucker_status cholesky32(tucker_handle* h, float* M, int d, float* X, float* XC, int* inv_done);
bool chol32_on_cluster(tucker_handle* h, int d);
tucker_status chol_prepare(tucker_handle* h, const double* L, int d, double* LT, double* Linv);
tucker_status chol_prepare32(tucker_handle* h, const float* L, int d, float* LT, float* Linv);
tucker_status chol_solve2(tucker_handle* h, const double* L, const double* LT, const double* Linv,
                          int d, const double* rhs, double* g, double* tmp);
tucker_status chol_solve32(tucker_handle* h, const float* L, const float* LT, const float* Linv,
                           int d, const double* rhs, double* g, double* tmp);
tucker_status launch_to_f32(tucker_handle* h, const double* in, size_t n, float* out);
tucker_status launch_gemv_resid(tucker_handle* h, const double* M, int d, const double* g,
                                const double* hv, double* r);
size_t chol_inv_doubles(int d);
int chol_inverse_fits(int d);
tucker_status chol_inverse32(tucker_handle* h, const float* L, const float* Linv, int d, float* X,
                             float* XC);
tucker_status chol_solve_inv32(tucker_handle* h, const float* X, const float* XC, int d,
                               const double* rhs, double* g, double* tmp);
tucker_status launch_regdiag(tucker_handle* h, double* out, int d, double lambda, const double* D);
tucker_status chol_correct_inv32(tucker_handle* h, const float* X, const float* XC, int d,
                                 double* r, double* g, double* stats, double* tmp, double* part);
tucker_status launch_refine_update(tucker_handle* h, double* g, const double* r, int d,
                                   double* out2);
tucker_status launch_add_diag(tucker_handle* h, double* M, int d, const double* diag);
tucker_status ttm_chain_all(tucker_handle* h, const FactorSet& F, const void* X, double* buf0,
                            double* buf1, double* y);
tucker_status ttm_last(tucker_handle* h, const void* X, int is64, int64_t P, int I, const void* A,
                       int R, double* out, double* sq_partial = nullptr, int sq_cap = 0,
                       double* sq_out = nullptr);
tucker_status ttm_chain_except(tucker_handle* h, const FactorSet& F, const void* X, int n,
                               double* buf0, double* buf1, double* out,
                               const double* ylast = nullptr);
size_t fiber_workspace_bytes(const FactorSet& F, int n, int64_t cap, int splits);
int fiber_splits(int64_t cap);
tucker_status launch_fiber_update(tucker_handle* h, const FactorSet& F, int n, const void* X,
                                  const double* core, const uint64_t* keys,
                                  const uint32_t* counts, const int* d_nu, int64_t cap,
                                  const uint64_t* const* cdf_others, int64_t m, double lambda,
                                  char* ws, size_t ws_bytes, void* A_out, int cp);
tucker_status kron_whiten(tucker_handle* h, const FactorSet& F, double* const* V,
                          double* const* ev, double lambda, const double* M, double* tmp,
                          double* out);
tucker_status vec_normalize(tucker_handle* h, const double* y, int d, double* x, double* norm_out);
tucker_status kron_eig_core(tucker_handle* h, const FactorSet& F, double* const* V,
                            double* const* s, const double* y, double lambda, double* g);
tucker_status residual_sq(tucker_handle* h, const FactorSet& F, const tucker_tensor* X,
                          const double* g, double* buf0, double* buf1, double* partial,
                          int npartial, double* out);
tucker_status sumsq(tucker_handle* h, const void* v, int is64, int64_t n, double* partial,
                    int npartial, double* out);
tucker_status launch_factor_grams(tucker_handle* h, const FactorSet& F, int* d_rank,
                                  double* const* gram);
tucker_status tensor_sumsq(tucker_handle* h, const void* X, int is64, int64_t n, double* partial,
                           int npartial, double* out);
tucker_status kt_x_from_last(tucker_handle* h, const FactorSet& F, const double* B, double* y);
tucker_status kron_quad(tucker_handle* h, const FactorSet& F, double* const* gram, const double* g,
                        const double* y, double* out);
tucker_status factor_solve(tucker_handle* h, const FactorSet& F, int n, double* const* gram,
                           const double* core, const double* B, double lambda, void* A_out,
                           double* Lscratch);
tucker_status launch_adjoint_rows(tucker_handle* h, const FactorSet& F, uint32_t* const* idx,
                                  const double* w, const double* x, const double* zg,
                                  const double* zv, const double* g, const double* v,
                                  const int* n_rows, int64_t cap, double* const* dA, double* dx);
size_t walk_scratch_doubles(int64_t I1, int d, int R1, int64_t cap, int sms);
bool walk_fits(int N, const int* R, int64_t I1);
tucker_status walk_segments(tucker_handle* h, const RowSet& s, int64_t I1, const WalkBuf& wb);
tucker_status walk_dot(tucker_handle* h, const RowSet& s, int64_t I1, const WalkBuf& wb,
                       const double* g1, const double* g2, double* z1, double* z2,
                       bool f32 = false);
tucker_status walk_axpy(tucker_handle* h, const RowSet& s, int64_t I1, const WalkBuf& wb,
                        const double* ca, const double* cb, double coef, const double* base,
                        const double* diag, const double* y, double* out, bool f32 = false);
bool walk_f32_ok(const RowSet& s);
tucker_status launch_decode_rows(tucker_handle* h, const FactorSet& F, const uint64_t* keys,
                                 int64_t n, uint32_t* const* idx, const void* vals, double* x);
int gram_tc_supported(int prec, int d);
size_t gram_tc_workspace(tucker_handle* h, int prec, int d, int sumR, int64_t cap, int N, int R1,
                         int64_t I1);
int gram_tc_grouped_ok(int N, int d, int R1, int64_t I1);
int gram_tc_narrow_ok(int N, int d, int R1, int64_t I1, int64_t cap);
tucker_status launch_gram_tc_narrow(tucker_handle* h, const RowSet& s, int64_t I1, int64_t cap,
                                    char* ws, size_t ws_bytes, double* G);
tucker_status launch_gram_tc_grouped(tucker_handle* h, const RowSet& s, int prec, int64_t cap,
                                     int64_t I1, char* ws, size_t ws_bytes, double* G);
tucker_status launch_gram_tc(tucker_handle* h, const RowSet& s, int prec, int64_t cap, char* ws,
                             size_t ws_bytes, double* G);

tucker_status launch_to_f64(tucker_handle* h, const FactorSet& F, double* const* out);
tucker_status launch_gram_eig(tucker_handle* h, int N, const int* R, const double* const* gram,
                              double* const* evecs, double* const* evals);
int kpcg_fits(int d, int N, const int* R);
int ridge_components(const FactorSet& F, int* K);
size_t ridge_tables_scratch(const FactorSet& F);
size_t ridge_sample_scratch(const FactorSet& F, int64_t m);
tucker_status ridge_tables(tucker_handle* h, const FactorSet& F, double lambda, char* scratch,
                           double* const* usq, double* c, double* d_eff,
                           double* const* V_out, double* const* ev_out);
tucker_status ridge_draw(tucker_handle* h, const FactorSet& F, const double* const* usq,
                         const double* c, int64_t m, uint64_t seed, uint32_t sweep,
                         char* scratch, uint64_t* keys_raw, int64_t* d_T, RidgeState* st);
tucker_status ridge_prob(tucker_handle* h, RidgeState* st, const uint64_t* keys_u,
                         const int* n_unique, int64_t cap, double* prob);
tucker_status launch_kpcg(tucker_handle* h, const float* M, const double* regdiag, int d, int N,
                          const int* R, const double* const* V, const double* const* ev,
                          const double* rhs, double* out, double* upd, double* stats,
                          double* part, float* sg, double* res, double tol, int max_iter,
                          bool dep);
size_t leverage_aux_bytes(int64_t maxI);
static int64_t max_dim(const FactorSet& F) { int64_t m = 1; for (int n = 0; n < F.N; ++n) if (F.I[n] > m) m = F.I[n]; return m; }

// The row set with FP64 factors (converted once per call when they are FP32).
static tucker_status rowset64(tucker_handle* h, const FactorSet& F, const RowSet& rs,
                              double* const* A64, RowSet* out) {
  *out = rs;
  if (F.is64) return TUCKER_OK;
  TK_TRY(launch_to_f64(h, F, A64));
  for (int n = 0; n < F.N; ++n) out->A[n] = A64[n];
  out->is64 = 1;
  return TUCKER_OK;
}

// ---------------------------------------------- FP64 products with sampled rows
// Level walk along the sorted sample when its vectors fit in shared memory,
// else the per-element kernels (same results up to summation order).
static tucker_status rows_dot(tucker_handle* h, const FactorSet& F, const RowSet& rs,
                              const WalkBuf& walk, const double* g1, const double* g2, double* z1,
                              double* z2) {
  if (walk_fits(F.N, F.R, F.I[0])) return walk_dot(h, rs, F.I[0], walk, g1, g2, z1, z2);
  return launch_kron_dot(h, rs, g1, g2, z1, z2);
}

static tucker_status rows_axpy(tucker_handle* h, const FactorSet& F, const RowSet& rs,
                               const WalkBuf& walk, int nsplit, double* part, const double* ca,
                               const double* cb, double coef, const double* base,
                               const double* diag, const double* y, double* out) {
  if (walk_fits(F.N, F.R, F.I[0]))
    return walk_axpy(h, rs, F.I[0], walk, ca, cb, coef, base, diag, y, out);
  return launch_kron_axpy(h, rs, ca, cb, coef, nsplit, part, base, diag, y, out);
}

// Whether a residual may be evaluated with the FP32 walks on the FP32 factors of rs32.
static bool rows_f32_ok(const FactorSet& F, const RowSet* rs32) {
  return rs32 && walk_fits(F.N, F.R, F.I[0]) && walk_f32_ok(*rs32);
}

// ----------------------------------------------------------------- plumbing

tucker_status fail(tucker_handle* h, tucker_status s, const char* fmt, ...) {
  if (h) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h->err, sizeof(h->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

tucker_status ws_reserve(tucker_handle* h, size_t bytes) {
  if (bytes <= h->ws_cap) return TUCKER_OK;
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  if (h->ws) cudaFree(h->ws);
  h->ws = nullptr;
  h->ws_cap = 0;
  size_t want = bytes + bytes / 4 + (1 << 20);
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, TUCKER_ENOMEM, "workspace of %zu bytes", bytes);
    }
    want = bytes;
  }
  h->ws = static_cast<char*>(p);
  h->ws_cap = want;
  return TUCKER_OK;
}

static const char* dev_msg(int code) {
  switch (code) {
    case DEV_NOTSPD: return "Cholesky met a non-positive pivot (matrix not SPD)";
    case DEV_RANK: return "a factor has zero total leverage";
    case DEV_DRAWLIMIT: return "draw limit reached before m accepted";
    case DEV_HASHFULL: return "observed-entry hash table probe limit exceeded";
    default: return "device-side consistency check failed";
  }
}

tucker_status device_status(tucker_handle* h) {
  TK_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                             h->stream));
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  const int code = *h->h_status;
  if (!code) return TUCKER_OK;
  TK_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  return fail(h, (tucker_status)code, "%s", dev_msg(code));
}

tucker_status finish(tucker_handle* h) {
  if (!h->sync_mode) return TUCKER_OK;
  return device_status(h);
}

static tucker_status make_factors(tucker_handle* h, int N, const int64_t* I, const int* R,
                                  tucker_dtype dt, const void* const* A, FactorSet* F) {
  if (N < 1 || N > TUCKER_MAX_ORDER) return fail(h, TUCKER_EINVAL, "order %d out of range", N);
  if (!I || !R) return fail(h, TUCKER_EINVAL, "null dims or ranks");
  if (dt != TUCKER_F32 && dt != TUCKER_F64) return fail(h, TUCKER_EINVAL, "bad dtype");
  memset(F, 0, sizeof(*F));
  F->N = N;
  F->is64 = dt == TUCKER_F64;
  int64_t d = 1;
  double tot = 1.0;
  uint64_t total = 1;
  for (int n = 0; n < N; ++n) {
    if (I[n] < 1 || I[n] > (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "I_%d out of range", n);
    if (R[n] < 1 || R[n] > TUCKER_MAX_RANK) return fail(h, TUCKER_EINVAL, "R_%d out of range", n);
    F->I[n] = I[n];
    F->R[n] = R[n];
    F->A[n] = A ? A[n] : nullptr;
    if (A && !A[n]) return fail(h, TUCKER_EINVAL, "factor %d is NULL", n);
    d *= R[n];
    tot *= double(I[n]);
    total *= (uint64_t)I[n];
  }
  if (d > 8192) return fail(h, TUCKER_EINVAL, "prod(R_n) = %lld exceeds 8192", (long long)d);
  if (tot >= 4.0e18) return fail(h, TUCKER_EINVAL, "prod(I_n) too large");
  F->d = (int)d;
  F->total = total;
  return TUCKER_OK;
}

static tucker_status check_tensor(tucker_handle* h, const tucker_tensor* X, const int* R,
                                  const void* const* A, FactorSet* F) {
  if (!X) return fail(h, TUCKER_EINVAL, "X is NULL");
  TK_TRY(make_factors(h, X->order, X->dims, R, X->dtype, A, F));
  const bool dense = X->dense != nullptr;
  const bool coo = X->keys != nullptr && X->vals != nullptr;
  if (dense == coo) return fail(h, TUCKER_EINVAL, "X must be dense or COO (exactly one)");
  if (coo && X->nnz < 1) return fail(h, TUCKER_EINVAL, "COO tensor with nnz < 1");
  if (coo && (uint64_t)X->nnz > F->total) return fail(h, TUCKER_EINVAL, "nnz > prod(I)");
  return TUCKER_OK;
}

static int bits_for(uint64_t v) {   // bits needed to hold values < v
  int b = 1;
  while (b < 64 && (v - 1) >> b) ++b;
  return b;
}

static void ev_record(tucker_handle* h, bool on, int i) {
  if (on) cudaEventRecord(h->ev[i], h->stream);
}

static double ev_ms(tucker_handle* h, int a, int b) {
  float ms = 0.f;
  cudaEventElapsedTime(&ms, h->ev[a], h->ev[b]);
  return ms;
}

// --------------------------------------------------------- sketch pipeline

constexpr int kMaxRefine = 12;                 // refinement iterations, at most

struct SketchBufs {
  double* lev[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  int* rank;
  uint64_t* keys_raw;
  int64_t* d_T;
  char* sort_scratch;
  size_t sort_bytes;
  uint64_t* keys_u;
  uint32_t* counts;
  int* nu;
  int* nreal;
  uint32_t* idx[TUCKER_MAX_ORDER];
  double *w, *x, *p, *z;
  float* sw32;
  double *D, *h, *g, *r, *axpy_part;
  double* rstat;                      // refinement: ||c_k||^2, ||g_k||^2 per iteration
  double* ptab;                       // per-mode q/Q and Q/q tables of the gather
  WalkBuf walk;
  double* A64[TUCKER_MAX_ORDER];      // FP64 copies of FP32 factors (walk kernels)
  double* fgram[TUCKER_MAX_ORDER];    // A^(n)T A^(n) (R_n x R_n), for the CG preconditioner
  char* gram_ws;
  size_t gram_bytes;
  int axpy_split;
  int simt_split;
};

static void carve_sketch(Arena& ar, tucker_handle* h, const FactorSet& F, int64_t m,
                         int prec, int fixed, SketchBufs* b) {
  for (int n = 0; n < F.N; ++n) {
    b->lev[n] = ar.get<double>(F.I[n]);
    b->cdf[n] = ar.get<uint64_t>(F.I[n]);
  }
  b->rank = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(max_dim(F))));
  for (int n = 0; n < F.N; ++n) b->fgram[n] = ar.get<double>((size_t)F.R[n] * F.R[n]);
  b->keys_raw = fixed ? nullptr : ar.get<uint64_t>(m);
  b->d_T = ar.get<int64_t>(1);
  b->sort_bytes = fixed ? 0 : sort_dedupe_scratch(m);
  b->sort_scratch = fixed ? nullptr : ar.get<char>(b->sort_bytes);
  b->keys_u = fixed ? nullptr : ar.get<uint64_t>(m);
  b->counts = fixed ? nullptr : ar.get<uint32_t>(m);
  b->nu = ar.get<int>(1);
  b->nreal = ar.get<int>(1);
  for (int n = 0; n < F.N; ++n) b->idx[n] = ar.get<uint32_t>(m);
  b->w = ar.get<double>(m);
  b->x = ar.get<double>(m);
  b->p = ar.get<double>(m);
  b->z = ar.get<double>(m);
  b->sw32 = ar.get<float>(m);
  b->D = ar.get<double>(F.d);
  {
    int64_t sumI = 0;
    for (int n = 0; n < F.N; ++n) sumI += F.I[n];
    b->ptab = ar.get<double>(2 * sumI);
  }
  b->h = ar.get<double>(F.d);
  b->g = ar.get<double>(F.d);
  b->r = ar.get<double>(F.d);
  b->rstat = ar.get<double>(2 * kMaxRefine);
  b->axpy_split = axpy_splits(h, F.d, m);
  b->axpy_part = ar.get<double>((size_t)b->axpy_split * F.d);
  b->walk.p = ar.get<double>(walk_scratch_doubles(F.I[0], F.d, F.R[0], m, h->num_sms));
  b->walk.cap = m;
  b->walk.I2 = F.N >= 2 ? F.I[1] : 0;
  for (int n = 0; n < F.N; ++n)
    b->A64[n] = F.is64 ? nullptr : ar.get<double>((size_t)F.I[n] * F.R[n]);
  b->simt_split = gram_simt_splits(h, F.d, m);
  int sumR = 0;
  for (int n = 0; n < F.N; ++n) sumR += F.R[n];
  // room for the FP64 CUDA-core Gram as well: the fallback of solve_robust
  b->gram_bytes = gram_simt_partial_bytes(F.d, b->simt_split, 1);
  if (prec == TUCKER_PREC_TF32 || prec == TUCKER_PREC_BF16)
    b->gram_bytes = std::max(b->gram_bytes,
                             gram_tc_workspace(h, prec, F.d, sumR, m, F.N, F.R[0], F.I[0]));
  b->gram_ws = ar.get<char>(b->gram_bytes);
}

constexpr size_t kPartDoubles = 512;            // per-CTA partial sums of one inverse application

constexpr int kKresSlots = 64;                  // CG solves recorded per call, at most
constexpr size_t kKronDoubles =                 // V_n and ev_n of every mode
    (size_t)TUCKER_MAX_ORDER * (TUCKER_MAX_RANK * TUCKER_MAX_RANK + TUCKER_MAX_RANK);

template <class T>
static T* align16(T* p) {
  return reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(p) + 15) & ~uintptr_t(15));
}

static tucker_status chol_reserve(tucker_handle* h, int d) {
  CholCache& c = h->chol;
  const size_t need = (size_t)d * d;
  const size_t inv = chol_inv_doubles(d);
  const size_t xinv = chol_inverse_fits(d) ? 2 * need : 0;
  // FP64: L, LT, regdiag, tmp, Linv, part, V_n / ev_n, CG records; FP32: L32, LT32,
  // Linv32, the CG product exchange (+ X32, XC32 for small d)
  const size_t bytes = (2 * need + 2 * (size_t)d + inv + 64 + kPartDoubles + kKronDoubles +
                        2 * kKresSlots) * sizeof(double) +
                       (2 * need + inv + 64 + xinv + 2 * (size_t)d + 64) * sizeof(float) + 64;
  if (c.cap < bytes) {
    TK_CUDA(h, cudaStreamSynchronize(h->stream));
    if (c.L) cudaFree(c.L);
    c.L = nullptr;
    c.cap = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, TUCKER_ENOMEM, "Cholesky buffer for d = %d", d);
    }
    c.L = static_cast<double*>(p);
    c.cap = bytes;
  }
  c.LT = c.L + need;
  c.regdiag = c.LT + need;
  c.tmp = c.regdiag + d;
  c.Linv = c.tmp + d;
  c.part = c.Linv + inv + 64;
  double* kb = c.part + kPartDoubles;
  for (int n = 0; n < TUCKER_MAX_ORDER; ++n) {
    c.kv[n] = kb + (size_t)n * TUCKER_MAX_RANK * TUCKER_MAX_RANK;
    c.ke[n] = kb + (size_t)TUCKER_MAX_ORDER * TUCKER_MAX_RANK * TUCKER_MAX_RANK +
              (size_t)n * TUCKER_MAX_RANK;
  }
  c.kres = kb + kKronDoubles;
  c.L32 = align16(reinterpret_cast<float*>(c.kres + 2 * kKresSlots));
  c.LT32 = c.L32 + need;
  c.Linv32 = c.LT32 + need;
  c.sg = align16(c.Linv32 + inv + 64);
  c.X32 = xinv ? align16(c.sg + 2 * (size_t)d) : nullptr;
  c.XC32 = c.X32 ? c.X32 + need : nullptr;
  c.kpcg = 0;
  c.kron_ready = 0;
  c.d = d;
  c.id = 0;
  return TUCKER_OK;
}

// Factor M (= G + diag(regdiag), full and symmetric in the FP64 buffer L)
// with the handle's solver.  FP64: L L^T = M in place; the solves run in FP64
// when the Gram is FP64 (no refinement follows), else in FP32 on the rounded
// factor (they only precondition the FP64 refinement).  Mixed: the FP32 copy
// is factored and L keeps M for the FP64 residual.
// Whether the Kronecker-preconditioned CG solver handles this solve: chosen on
// the handle, a rounded Gram (an FP64 Gram keeps the direct FP64 solve), and
// the d-vectors and V_n fit in shared memory.
static bool kpcg_wanted(tucker_handle* h, const FactorSet& F, int prec) {
  return h->solver == TUCKER_SOLVER_KRON_PCG && prec != TUCKER_PREC_FP64 &&
         kpcg_fits(F.d, F.N, F.R);
}

// Eigendecompositions A^(n)T A^(n) = V_n diag(ev_n) V_n^T of the factor Grams
// (written by the leverage launcher) into the cache, for the CG preconditioner.
// The eigenvalues ev_n to the pinned host buffer h_kev, on the current stream
// (the refinement's first check of the contraction reads them).
static tucker_status kron_ev_to_host(tucker_handle* h) {
  const CholCache& c = h->chol;
  for (int n = 0; n < c.kN; ++n)
    TK_CUDA(h, cudaMemcpyAsync(h->h_kev + n * TUCKER_MAX_RANK, c.ke[n], sizeof(double) * c.kR[n],
                               cudaMemcpyDeviceToHost, h->stream));
  return TUCKER_OK;
}

static tucker_status kron_prepare(tucker_handle* h, const FactorSet& F,
                                  const double* const* fgram) {
  CholCache& c = h->chol;
  TK_TRY(launch_gram_eig(h, F.N, F.R, fgram, c.kv, c.ke));
  c.kN = F.N;
  for (int n = 0; n < F.N; ++n) c.kR[n] = F.R[n];
  c.kron_ready = 1;
  return kron_ev_to_host(h);
}

// Relative residual of each CG solve: below the rounding of the Gram it
// solves with (about 3e-4 relative for BF16 operands, 3e-5 for TF32 on the
// 512^3 workload), so that the FP64 refinement contracts at the Gram's rate.
static double kpcg_tol(int prec) { return prec == TUCKER_PREC_BF16 ? 1e-4 : 1e-5; }
constexpr int kKpcgMaxIter = 50;

// One CG solve with the cached M~ (L32) and preconditioner: out = M~^-1 rhs
// and/or upd += M~^-1 rhs with the norms in stats.  The first solve of a call
// is timed (events 12, 13) when the call records stage times.
static tucker_status kpcg_solve(tucker_handle* h, int d, const double* rhs, double* out,
                                double* upd, double* stats) {
  CholCache& c = h->chol;
  double* res = c.kres_n < kKresSlots ? c.kres + 2 * c.kres_n : nullptr;
  const bool first = c.kres_n == 0;
  ++c.kres_n;
  if (first) ev_record(h, h->timing, 12);
  // a correction's solve follows the residual's kernels on this stream: launched
  // with programmatic dependence on them (the first follows the join of the
  // second stream, and is launched in full order)
  TK_TRY(launch_kpcg(h, c.L32, c.regdiag, d, c.kN, c.kR, c.kv, c.ke, rhs, out, upd, stats,
                     c.part, c.sg, res, c.ktol, kKpcgMaxIter, !first));
  if (first) ev_record(h, h->timing, 13);
  return TUCKER_OK;
}

static tucker_status factorize(tucker_handle* h, double* L, int d, int prec, int solver) {
  CholCache& c = h->chol;
  c.prep64 = c.prep32 = c.inv32 = 0;
  c.kpcg = 0;
  if (solver == TUCKER_SOLVER_KRON_PCG && prec != TUCKER_PREC_FP64 && c.kron_ready &&
      kpcg_fits(d, c.kN, c.kR)) {
    // no factor: the CG solves read the FP32 copy of M (L keeps M in FP64)
    c.mixed = 0;
    ev_record(h, h->timing, 8);
    TK_TRY(launch_to_f32(h, L, (size_t)d * d, c.L32));
    ev_record(h, h->timing, 9);
    c.kpcg = 1;
    c.ktol = kpcg_tol(prec);
    return TUCKER_OK;
  }
  c.mixed = solver == TUCKER_SOLVER_MIXED || solver == TUCKER_SOLVER_KRON_PCG;
  if (c.mixed) {
    TK_TRY(launch_to_f32(h, L, (size_t)d * d, c.L32));
    ev_record(h, h->timing, 8);
    int inv_done = 0;
    TK_TRY(cholesky32(h, c.L32, d, c.X32, c.XC32, &inv_done));
    ev_record(h, h->timing, 9);
    if (inv_done) {                     // the factor's launch also formed X = L^-1
      c.inv32 = 1;
      return TUCKER_OK;
    }
    TK_TRY(chol_prepare32(h, c.L32, d, c.LT32, c.Linv32));
    c.prep32 = 1;
    if (c.X32) {
      TK_TRY(chol_inverse32(h, c.L32, c.Linv32, d, c.X32, c.XC32));
      c.inv32 = 1;
    }
    return TUCKER_OK;
  }
  ev_record(h, h->timing, 8);
  TK_TRY(cholesky(h, L, d));
  ev_record(h, h->timing, 9);
  if (prec == TUCKER_PREC_FP64) {
    TK_TRY(chol_prepare(h, L, d, c.LT, c.Linv));
    c.prep64 = 1;
  } else {
    TK_TRY(launch_to_f32(h, L, (size_t)d * d, c.L32));
    TK_TRY(chol_prepare32(h, c.L32, d, c.LT32, c.Linv32));
    c.prep32 = 1;
    if (c.X32) {
      TK_TRY(chol_inverse32(h, c.L32, c.Linv32, d, c.X32, c.XC32));
      c.inv32 = 1;
    }
  }
  return TUCKER_OK;
}

// g = (L L^T)^-1 rhs with the cached factor (g may alias rhs).  FP32 solves
// when the factor is FP32, or when the Gram precision calls for refinement and
// the rounded copy exists; FP64 otherwise.
static tucker_status chol_solve(tucker_handle* h, int d, const double* rhs, double* g, int prec) {
  CholCache& c = h->chol;
  if (c.kpcg) return kpcg_solve(h, d, rhs, g, nullptr, nullptr);
  if (c.mixed || (c.prep32 && prec != TUCKER_PREC_FP64)) {
    if (c.inv32) return chol_solve_inv32(h, c.X32, c.XC32, d, rhs, g, c.tmp);
    return chol_solve32(h, c.L32, c.LT32, c.Linv32, d, rhs, g, c.tmp);
  }
  if (!c.prep64) {
    TK_TRY(chol_prepare(h, c.L, d, c.LT, c.Linv));
    c.prep64 = 1;
  }
  return chol_solve2(h, c.L, c.LT, c.Linv, d, rhs, g, c.tmp);
}

// G (into L buffer) from the sample, by precision.
static tucker_status build_gram(tucker_handle* h, const FactorSet& F, const RowSet& rs, int prec,
                                int64_t cap, SketchBufs& b, double* G) {
  if (prec == TUCKER_PREC_FP64 || prec == TUCKER_PREC_FP32)
    return launch_gram_simt(h, rs, prec == TUCKER_PREC_FP64, b.simt_split, b.gram_ws, G);
  if (!gram_tc_supported(prec, F.d))
    return fail(h, TUCKER_ENOTSUP, "tensor-core Gram does not support d = %d", F.d);
  // sorted sample: group the Gram by the leading index when that is the smaller job
  if (gram_tc_narrow_ok(F.N, F.d, F.R[0], F.I[0], cap))
    return launch_gram_tc_narrow(h, rs, F.I[0], cap, b.gram_ws, b.gram_bytes, G);
  if (gram_tc_grouped_ok(F.N, F.d, F.R[0], F.I[0]))
    return launch_gram_tc_grouped(h, rs, prec, cap, F.I[0], b.gram_ws, b.gram_bytes, G);
  return launch_gram_tc(h, rs, prec, cap, b.gram_ws, b.gram_bytes, G);
}

// g = M^-1 rhs with the cached factor of M~ (the Gram as built + diag(regdiag)),
// refined in FP64 whenever the factor is not an FP64 factor of M itself:
//   g <- g + M~^-1 (rhs - M g),  M g = sum_u w_u k_u (k_u . g) + regdiag * g
// on the implicit FP64 rows, or the explicit FP64 M when the Gram was FP64
// (mixed solver).  Stops at ||correction|| < tol ||g|| or when the correction
// stops shrinking.
static tucker_status solve_refined(tucker_handle* h, const FactorSet& F, const RowSet& rs,
                                   int prec, SketchBufs& b, const double* rhs, double* g,
                                   int* iters, double* rel, const RowSet* rs32 = nullptr,
                                   bool* converged = nullptr) {
  const int d = F.d;
  TK_TRY(chol_solve(h, d, rhs, g, prec));
  *iters = 0;
  *rel = 0.0;
  if (converged) *converged = true;
  const bool explicit_m = prec == TUCKER_PREC_FP64;
  if (explicit_m && !h->chol.mixed) return TUCKER_OK;
  // stop when the remaining relative error, estimated from the last correction
  // c_k and the contraction rho ~ c_k / c_{k-1}, is below target (c_0 = 1: the
  // first solve), or when the corrections stop shrinking (rounding level).  A
  // BF16 Gram (and a TF32 one under the factor solvers) always takes two
  // corrections, so the first two are enqueued back to back and the host waits
  // once for both.  The first of them only has to be accurate to the Gram's
  // rounding level, so with FP32 factors its residual is evaluated by the FP32
  // walks; every later residual, which sets the accuracy of the result, is FP64.
  const double target = explicit_m ? 1e-13 : 1e-8;
  const int max_iters = (h->chol.mixed || h->chol.kpcg) ? 12 : 8;
  bool reached = false;
  // With the CG solver on a TF32 Gram one FP64 correction reaches the target
  // (the rounded solve is off by about 3e-5 relative; each CG solve stops at 1e-5)
  const int batch =
      (prec == TUCKER_PREC_BF16 || (prec == TUCKER_PREC_TF32 && !h->chol.kpcg)) ? 2 : 1;
  // A single correction c_1 proves convergence only when the contraction is
  // known to be small: along a direction that M resolves but the rounded M~
  // does not (an eigenvalue of M far below M~'s rounding error) both the
  // residual and the correction are scaled down by lambda_min(M) / lambda_min(M~),
  // so c_1 is small while the error is not.  The estimate rho ~ u kappa(K^T K),
  // u the Gram's unit roundoff and kappa from the factor eigenvalues (those of
  // the Kronecker preconditioner), must be at most 0.1 for c_1 alone to decide
  // (with rho ~ c_1 as before); otherwise the contraction is measured from two
  // corrections, and corrections that stop shrinking end the solve unconverged.
  // (h_kev was filled by kron_ev_to_host behind the eigendecompositions, on a
  // stream the solve has joined, so the first host wait below also covers it)
  const bool kev = h->chol.kpcg && h->chol.kron_ready;
  bool trust_first = false;                       // decided at the first wait
  double prev = 1.0;
  int checked = 0;
  for (int it = 0; it < max_iters; ++it) {
    if (explicit_m) {
      TK_TRY(launch_gemv_resid(h, h->chol.L, d, g, rhs, b.r));
    } else if (it == 0 && batch == 2 && rows_f32_ok(F, rs32)) {
      TK_TRY(walk_dot(h, *rs32, F.I[0], b.walk, g, nullptr, b.z, nullptr, true));
      TK_TRY(walk_axpy(h, *rs32, F.I[0], b.walk, b.w, b.z, -1.0, rhs, h->chol.regdiag, g, b.r,
                       true));
    } else {
      TK_TRY(rows_dot(h, F, rs, b.walk, g, nullptr, b.z, nullptr));
      TK_TRY(rows_axpy(h, F, rs, b.walk, b.axpy_split, b.axpy_part, b.w, b.z, -1.0, rhs,
                       h->chol.regdiag, g, b.r));
    }
    CholCache& cc = h->chol;
    if (cc.kpcg) {
      TK_TRY(kpcg_solve(h, d, b.r, nullptr, g, b.rstat + 2 * it));
    } else if ((cc.mixed || (cc.prep32 && prec != TUCKER_PREC_FP64)) && cc.inv32) {
      TK_TRY(chol_correct_inv32(h, cc.X32, cc.XC32, d, b.r, g, b.rstat + 2 * it, cc.tmp, cc.part));
    } else {
      TK_TRY(chol_solve(h, d, b.r, b.r, prec));
      TK_TRY(launch_refine_update(h, g, b.r, d, b.rstat + 2 * it));
    }
    if (it + 1 < batch) continue;                     // the next correction is certain
    double hv[2 * kMaxRefine];
    const int n = it + 1 - checked;
    TK_CUDA(h, cudaMemcpyAsync(hv, b.rstat + 2 * checked, 2 * n * sizeof(double),
                               cudaMemcpyDeviceToHost, h->stream));
    TK_CUDA(h, cudaMemcpyAsync(h->h_status, h->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                               h->stream));
    TK_CUDA(h, cudaStreamSynchronize(h->stream));
    if (*h->h_status) return device_status(h);     // e.g. a factor met a non-positive pivot
    if (checked == 0 && kev) {
      double emax = 1.0, emin = 1.0;
      for (int q = 0; q < h->chol.kN; ++q) {
        double top = 0.0, low = HUGE_VAL;
        for (int k = 0; k < h->chol.kR[q]; ++k) {
          top = fmax(top, h->h_kev[q * TUCKER_MAX_RANK + k]);
          low = fmin(low, h->h_kev[q * TUCKER_MAX_RANK + k]);
        }
        emax *= top;
        emin *= low;
      }
      const double u = prec == TUCKER_PREC_BF16 ? 0x1p-8 : prec == TUCKER_PREC_TF32 ? 0x1p-11
                                                                                   : 0x1p-24;
      const double kappa = emin > 0.0 ? emax / emin : HUGE_VAL;
      trust_first = u * kappa <= 0.1;
      // each CG solve stops at the relative residual ktol, so an error component
      // whose residual share is below ktol (kappa ktol >= 1) is never corrected,
      // whatever the corrections show: the caller solves with a factor instead
      if (kappa * h->chol.ktol > 0.1) {
        *iters = it + 1;
        if (converged) *converged = false;
        return TUCKER_OK;
      }
    }
    bool stop = false;
    for (int k = 0; k < n; ++k) {
      const double rk = hv[2 * k + 1] > 0 ? sqrt(hv[2 * k] / hv[2 * k + 1]) : 0.0;
      const bool first = checked + k == 0;
      const double rho = fmin(rk / prev, 0.5);
      const bool hit = (!first || trust_first) &&
                       (rk == 0.0 || rk * rho / (1.0 - rho) < target || rk < 1e-10);
      reached = reached || hit;
      stop = stop || hit || (checked + k > 0 && rk > 0.5 * prev);
      prev = rk;
      *rel = rk;
    }
    checked = it + 1;
    *iters = it + 1;
    if (stop) break;
  }
  // every path has to meet the target: a refinement that stalls above it (an
  // ill-conditioned matrix that the rounded Gram or the FP32 factor cannot
  // resolve) is reported, and the caller tries a more precise step
  if (converged) *converged = reached;
  return TUCKER_OK;
}

// solve_refined, and when the CG solver did not reach the target (a sketch
// far from the Kronecker Gram), the same solve with the FP32 factor of M~ (the
// mixed solver), from the FP64 M still held in the cache.  A refinement that
// still misses its target returns ENOTSPD (solve_robust then tries a more
// precise Gram and factor).
static tucker_status solve_checked(tucker_handle* h, const FactorSet& F, const RowSet& rs,
                                   int prec, SketchBufs& b, const double* rhs, double* g,
                                   int* iters, double* rel, const RowSet* rs32 = nullptr) {
  bool conv = true;
  TK_TRY(solve_refined(h, F, rs, prec, b, rhs, g, iters, rel, rs32, &conv));
  if (conv) return TUCKER_OK;
  if (h->chol.kpcg) {
    TK_TRY(factorize(h, h->chol.L, F.d, prec, TUCKER_SOLVER_MIXED));
    TK_TRY(solve_refined(h, F, rs, prec, b, rhs, g, iters, rel, rs32, &conv));
    if (conv) return TUCKER_OK;
  }
  return fail(h, TUCKER_ENOTSPD, "the refinement stalled at %.2e above its target: the Gram or "
              "its factor is too coarse for this matrix", *rel);
}

// solve_checked, and when a rounded Gram (TF32, BF16) or an FP32 factor met a
// non-positive pivot (an ill-conditioned Gram with a small lambda: early ALS
// sweeps from a random start), more precise steps in turn, each with an FP64
// Cholesky factor (and the FP64 refinement while the Gram is rounded):
//   TF32 / BF16 Gram: the FP32 and then the FP64 CUDA-core Gram of the same rows;
//   FP32 Gram:        its FP64 factor (FP32-factor solvers), then the FP64 Gram;
//   FP64 Gram:        its FP64 factor (FP32-factor solvers).
// Under the FP32-factor solvers L still holds M, so "its FP64 factor" needs no
// new Gram.  *used: the Gram precision that solved.
static tucker_status solve_robust(tucker_handle* h, const FactorSet& F, const RowSet& rs,
                                  const RowSet& rs64, int prec, SketchBufs& b, int* iters,
                                  double* rel, const RowSet* rs32, int* used) {
  *used = prec;
  tucker_status st = solve_checked(h, F, rs64, prec, b, b.h, b.g, iters, rel, rs32);
  if (st != TUCKER_ENOTSPD) return st;
  const bool fp32_factor = h->solver != TUCKER_SOLVER_FP64_CHOLESKY;
  struct Step { int prec; bool rebuild; } steps[2];
  int ns = 0;
  if (prec == TUCKER_PREC_TF32 || prec == TUCKER_PREC_BF16) {
    steps[ns++] = {TUCKER_PREC_FP32, true};
    steps[ns++] = {TUCKER_PREC_FP64, true};
  } else if (prec == TUCKER_PREC_FP32) {
    if (fp32_factor) steps[ns++] = {TUCKER_PREC_FP32, false};
    steps[ns++] = {TUCKER_PREC_FP64, true};
  } else if (fp32_factor) {
    steps[ns++] = {TUCKER_PREC_FP64, false};
  }
  for (int k = 0; k < ns; ++k) {
    const int lp = steps[k].prec;
    if (steps[k].rebuild) {
      TK_TRY(launch_gram_simt(h, rs, lp == TUCKER_PREC_FP64, b.simt_split, b.gram_ws,
                              h->chol.L));
      TK_TRY(launch_add_diag(h, h->chol.L, F.d, h->chol.regdiag));
    }
    TK_TRY(factorize(h, h->chol.L, F.d, lp, TUCKER_SOLVER_FP64_CHOLESKY));
    st = solve_checked(h, F, rs64, lp, b, b.h, b.g, iters, rel, nullptr);
    if (st == TUCKER_OK && lp == TUCKER_PREC_FP64) st = device_status(h);  // no wait inside
    *used = lp;
    if (st != TUCKER_ENOTSPD) return st;
  }
  return st;
}

// Factor G + diag(regdiag) (G in the FP64 buffer L) and solve for b.h, with
// the more precise steps of solve_robust when the first solve fails.
static tucker_status solve_refine(tucker_handle* h, const FactorSet& F, const RowSet& rs_raw,
                                  const RowSet& rs, int prec, SketchBufs& b, int* iters,
                                  double* rel) {
  TK_TRY(launch_add_diag(h, h->chol.L, F.d, h->chol.regdiag));
  TK_TRY(factorize(h, h->chol.L, F.d, prec, h->solver));
  int used;
  return solve_robust(h, F, rs_raw, rs, prec, b, iters, rel, nullptr, &used);
}

}  // namespace tk

using namespace tk;

// ========================================================== C entry points

extern "C" {

tucker_status tucker_create(tucker_handle** out, void* cuda_stream) {
  if (!out) return TUCKER_EINVAL;
  *out = nullptr;
  tucker_handle* h = new (std::nothrow) tucker_handle();
  if (!h) return TUCKER_ENOMEM;
  h->err[0] = 0;
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  cudaDeviceProp prop;
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaGetDeviceProperties(&prop, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return TUCKER_ECUDA;
  }
  if (prop.major * 10 + prop.minor != 103) {
    delete h;
    return TUCKER_ENOTSUP;
  }
  h->num_sms = prop.multiProcessorCount;
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&h->keep, kAuxDoubles * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&h->h_status, sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&h->h_kev, sizeof(double) * TUCKER_MAX_ORDER * TUCKER_MAX_RANK) !=
          cudaSuccess ||
      cudaMemset(h->d_status, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return TUCKER_ECUDA;
  }
  for (int i = 0; i < 16; ++i) cudaEventCreate(&h->ev[i]);
  if (cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    tucker_destroy(h);
    return TUCKER_ECUDA;
  }
  *out = h;
  return TUCKER_OK;
}

tucker_status tucker_destroy(tucker_handle* h) {
  if (!h) return TUCKER_EINVAL;
  cudaStreamSynchronize(h->stream);
  if (h->ws) cudaFree(h->ws);
  if (h->hash.slot_key) cudaFree(h->hash.slot_key);
  if (h->chol.L) cudaFree(h->chol.L);
  if (h->d_status) cudaFree(h->d_status);
  if (h->keep) cudaFree(h->keep);
  if (h->h_status) cudaFreeHost(h->h_status);
  if (h->h_kev) cudaFreeHost(h->h_kev);
  for (int i = 0; i < 16; ++i) cudaEventDestroy(h->ev[i]);
  if (h->aux) {
    cudaStreamSynchronize(h->aux);
    cudaStreamDestroy(h->aux);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
  return TUCKER_OK;
}

const char* tucker_last_error(const tucker_handle* h) { return h ? h->err : "null handle"; }

tucker_status tucker_set_sync(tucker_handle* h, int synchronous) {
  if (!h) return TUCKER_EINVAL;
  h->sync_mode = synchronous != 0;
  return TUCKER_OK;
}

tucker_status tucker_set_solver(tucker_handle* h, tucker_solver solver) {
  if (!h) return TUCKER_EINVAL;
  if (solver != TUCKER_SOLVER_FP64_CHOLESKY && solver != TUCKER_SOLVER_MIXED &&
      solver != TUCKER_SOLVER_KRON_PCG)
    return fail(h, TUCKER_EINVAL, "unknown solver %d", (int)solver);
  h->solver = solver;
  h->chol.id = 0;
  return TUCKER_OK;
}

tucker_status tucker_sync(tucker_handle* h) {
  if (!h) return TUCKER_EINVAL;
  return device_status(h);
}

tucker_status tucker_leverage_scores(tucker_handle* h, int N, const int64_t* I, const int* R,
                                     tucker_dtype dtype, const void* const* A,
                                     double* const* lev_out, uint64_t* const* cdf_out,
                                     int* rank_out_host) {
  if (!h) return TUCKER_EINVAL;
  if (!A || !lev_out) return fail(h, TUCKER_EINVAL, "null factor or output array");
  FactorSet F;
  TK_TRY(make_factors(h, N, I, R, dtype, A, &F));
  for (int n = 0; n < N; ++n)
    if (!lev_out[n]) return fail(h, TUCKER_EINVAL, "lev_out[%d] is NULL", n);
  Arena sz(nullptr);
  uint64_t* cdf_ws[TUCKER_MAX_ORDER];
  for (int n = 0; n < N; ++n) cdf_ws[n] = sz.get<uint64_t>(F.I[n]);
  int* rk = reinterpret_cast<int*>(sz.get<char>(leverage_aux_bytes(max_dim(F))));
  TK_TRY(ws_reserve(h, sz.off));
  Arena ar(h->ws);
  for (int n = 0; n < N; ++n) {
    uint64_t* c = ar.get<uint64_t>(F.I[n]);
    cdf_ws[n] = (cdf_out && cdf_out[n]) ? cdf_out[n] : c;
  }
  rk = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(max_dim(F))));
  TK_TRY(launch_leverage(h, F, lev_out, cdf_ws, rk, nullptr, nullptr, nullptr));
  if (rank_out_host) {
    TK_CUDA(h, cudaMemcpyAsync(rank_out_host, rk, sizeof(int) * N, cudaMemcpyDeviceToHost, h->stream));
    return device_status(h);
  }
  return finish(h);
}

tucker_status tucker_sample_rows(tucker_handle* h, int N, const int64_t* I, const int* R,
                                 const double* const* lev, int64_t m, uint64_t seed,
                                 uint32_t sweep, tucker_reg reg, const tucker_tensor* observed,
                                 int64_t max_draws, tucker_samples* out) {
  if (!h) return TUCKER_EINVAL;
  if (!lev || !out || !out->keys || !out->counts || !out->prob)
    return fail(h, TUCKER_EINVAL, "null scores or output arrays");
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
  if (out->capacity < m) return fail(h, TUCKER_ECAPACITY, "capacity %lld < m %lld",
                                     (long long)out->capacity, (long long)m);
  if (reg != TUCKER_REG_EXACT && reg != TUCKER_REG_AUGMENTED)
    return fail(h, TUCKER_EINVAL, "bad reg mode");
  FactorSet F;
  TK_TRY(make_factors(h, N, I, R, TUCKER_F64, nullptr, &F));
  if (observed) {
    if (!observed->keys || !observed->vals || observed->dense || observed->order != N)
      return fail(h, TUCKER_EINVAL, "observed must be a COO tensor of the same order");
    for (int n = 0; n < N; ++n)
      if (observed->dims[n] != I[n]) return fail(h, TUCKER_EINVAL, "observed dims differ");
  }
  for (int n = 0; n < N; ++n) if (!lev[n]) return fail(h, TUCKER_EINVAL, "lev[%d] NULL", n);
  auto carve = [&](Arena& ar, uint64_t** cdf, uint64_t** raw, int64_t** dT, char** ss, int** nu,
                   int** nreal, uint32_t** idx, double** w, double** x, double** D) {
    for (int n = 0; n < N; ++n) cdf[n] = ar.get<uint64_t>(F.I[n]);
    *raw = ar.get<uint64_t>(m);
    *dT = ar.get<int64_t>(1);
    *ss = ar.get<char>(sort_dedupe_scratch(m));
    *nu = ar.get<int>(1);
    *nreal = ar.get<int>(1);
    for (int n = 0; n < N; ++n) idx[n] = ar.get<uint32_t>(m);
    *w = ar.get<double>(m);
    *x = ar.get<double>(m);
    *D = ar.get<double>(F.d);
  };
  uint64_t* cdf[TUCKER_MAX_ORDER];
  uint64_t* raw;
  int64_t* dT;
  char* ss;
  int *nu, *nreal;
  uint32_t* idx[TUCKER_MAX_ORDER];
  double *w, *x, *D;
  Arena sz(nullptr);
  carve(sz, cdf, &raw, &dT, &ss, &nu, &nreal, idx, &w, &x, &D);
  // the missing-mode sampler carves its round buffers after these
  size_t extra = sample_keys_scratch(F, observed != nullptr);
  TK_TRY(ws_reserve(h, sz.off + extra));
  Arena ar(h->ws);
  carve(ar, cdf, &raw, &dT, &ss, &nu, &nreal, idx, &w, &x, &D);
  TK_TRY(launch_cdf_from_lev(h, N, I, lev, cdf));
  TK_TRY(device_status(h));
  int64_t T = 0;
  TK_TRY(sample_keys(h, F, cdf, m, seed, sweep, reg, observed, max_draws, raw, dT, &T, ar));
  const uint64_t key_range = F.total + (reg == TUCKER_REG_AUGMENTED ? (uint64_t)F.d : 0);
  TK_TRY(sort_dedupe(h, raw, m, bits_for(key_range), out->keys, out->counts, nu, ss,
                     sort_dedupe_scratch(m)));
  tucker_tensor none;
  memset(&none, 0, sizeof(none));
  none.order = N;
  none.dtype = TUCKER_F64;
  TK_TRY(launch_gather(h, F, cdf, reg, out->keys, out->counts, nu, dT, &none, m, idx, w, x,
                       out->prob, nullptr, nreal, D, nullptr, nullptr));
  int nuh = 0;
  TK_CUDA(h, cudaMemcpyAsync(&nuh, nu, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  TK_TRY(device_status(h));
  out->n_unique = nuh;
  out->n_draws = T;
  return TUCKER_OK;
}

// Alg. 1 line 3: s = ceil(4 d / beta' max{420 ln(4 d / delta), 1 / (delta eps)}).
static int64_t paper_s(int d, double eps, double delta, double beta_prime = 0.5) {
  double s = 4.0 * d / beta_prime * fmax(420.0 * log(4.0 * d / delta), 1.0 / (delta * eps));
  return (int64_t)ceil(s);
}

// beta' of Eq. beta_prime (Lemma beta_overestimate) for the exact lambda-ridge
// scores of K as the overestimate: beta = 1, ||l-hat||_1 = d_eff, and d_eff
// itself as the lower bound d'_eff; both terms of the minimum equal
// d / (d_eff + d min{1, d - d_eff}).
static double ridge_beta_prime(int d, double d_eff) {
  const double mlt = fmin(1.0, (double)d - d_eff);
  const double a = 1.0 * d / d_eff / (1.0 + d * mlt / d_eff);
  const double b = 1.0 / (d_eff / d + mlt);
  return fmin(a, b);
}

// Buffers of the lambda-ridge sampler inside the sketch arena.
struct RidgeBufs {
  double* usq[TUCKER_MAX_ORDER];
  double* c;
  double* d_eff;
  double* p;
  char* tab_scratch;
  char* samp_scratch;
};

static void carve_ridge(Arena& ar, const FactorSet& F, int64_t cap, RidgeBufs* r) {
  int K[TUCKER_MAX_ORDER];
  const int dK = ridge_components(F, K);
  for (int n = 0; n < F.N; ++n) r->usq[n] = ar.get<double>((size_t)K[n] * F.I[n]);
  r->c = ar.get<double>(dK);
  r->d_eff = ar.get<double>(1);
  r->p = ar.get<double>(cap);
  r->tab_scratch = ar.get<char>(ridge_tables_scratch(F));
  r->samp_scratch = ar.get<char>(ridge_sample_scratch(F, cap));
}

tucker_status tucker_core_update_sketched(tucker_handle* h, const tucker_tensor* X, const int* R,
                                          const void* const* A, double lambda, int64_t m,
                                          double eps, double delta, uint64_t seed, uint32_t sweep,
                                          tucker_reg reg, tucker_prec prec,
                                          const tucker_samples* fixed, double* core_out,
                                          tucker_stats* stats) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, A, &F));
  if (!A) return fail(h, TUCKER_EINVAL, "factors NULL");
  if (!core_out) return fail(h, TUCKER_EINVAL, "core_out NULL");
  if (!(lambda >= 0.0) || (reg == TUCKER_REG_AUGMENTED && !(lambda > 0.0)))
    return fail(h, TUCKER_EINVAL, "lambda must be >= 0 (> 0 in augmented mode)");
  if (reg != TUCKER_REG_EXACT && reg != TUCKER_REG_AUGMENTED && reg != TUCKER_REG_RIDGE)
    return fail(h, TUCKER_EINVAL, "reg");
  if (prec < TUCKER_PREC_FP64 || prec > TUCKER_PREC_BF16) return fail(h, TUCKER_EINVAL, "prec");
  const bool ridge = reg == TUCKER_REG_RIDGE && !fixed;
  if (ridge && !X->dense) return fail(h, TUCKER_EINVAL, "ridge sampling needs a dense X");
  // a frozen sample carries its probabilities: the ridge mode then is the exact one
  const int greg = reg == TUCKER_REG_RIDGE ? TUCKER_REG_EXACT : reg;
  int64_t cap;
  if (ridge && m == 0) {
    // Alg. 1 line 3 with beta' of Eq. beta_prime for the exact ridge scores: d_eff first
    if (!(eps > 0 && eps < 1 && delta > 0 && delta < 1))
      return fail(h, TUCKER_EINVAL, "eps, delta must be in (0,1) when m = 0");
    Arena sz0(nullptr);
    RidgeBufs r0;
    carve_ridge(sz0, F, 1, &r0);
    TK_TRY(ws_reserve(h, sz0.off));
    Arena ar0(h->ws);
    carve_ridge(ar0, F, 1, &r0);
    TK_TRY(ridge_tables(h, F, lambda, r0.tab_scratch, r0.usq, r0.c, r0.d_eff, nullptr, nullptr));
    double deff = 0.0;
    TK_CUDA(h, cudaMemcpyAsync(&deff, r0.d_eff, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TK_TRY(device_status(h));
    if (!(deff > 0.0)) return fail(h, TUCKER_ERANK, "all ridge weights are zero");
    m = paper_s(F.d, eps, delta, ridge_beta_prime(F.d, deff));
  }
  if (fixed) {
    if (!fixed->keys || !fixed->counts || !fixed->prob || fixed->n_unique < 1 ||
        fixed->n_unique > fixed->capacity || fixed->n_draws < 1)
      return fail(h, TUCKER_EINVAL, "fixed sample is incomplete");
    cap = fixed->n_unique;
  } else {
    if (m == 0) {
      if (!(eps > 0 && eps < 1 && delta > 0 && delta < 1))
        return fail(h, TUCKER_EINVAL, "eps, delta must be in (0,1) when m = 0");
      if (X->dense) {
        m = paper_s(F.d, eps, delta);
      } else {
        // observed entries: beta' from the Sec. 4.2 corollary bound and c_min
        tucker_missing_beta_info bi;
        TK_TRY(tucker_missing_beta(h, X, R, A, lambda, TUCKER_BETA_BOUND, prec, eps, delta, &bi));
        if (!(bi.s < (double)(int64_t(1) << 31)))
          return fail(h, TUCKER_EINVAL,
                      "Alg. 1 line 3 with the missing-data bound gives s = %.3g rows (beta' = %.3g); "
                      "pass m > 0, e.g. from tucker_missing_beta's exact mode", bi.s, bi.beta_prime);
        m = (int64_t)bi.s;
      }
    }
    if (m < 1 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
    cap = m;
  }
  if (reg == TUCKER_REG_AUGMENTED && F.total + (uint64_t)F.d < F.total)
    return fail(h, TUCKER_EINVAL, "key range overflow");
  const bool timing = stats != nullptr;
  const int64_t launches0 = h->launches;
  struct TimingFlag {
    tucker_handle* h;
    ~TimingFlag() { h->timing = 0; }
  } timing_guard{h};
  h->timing = timing;
  SketchBufs b;
  memset(&b, 0, sizeof(b));
  RidgeBufs rb;
  memset(&rb, 0, sizeof(rb));
  Arena sz(nullptr);
  carve_sketch(sz, h, F, cap, prec, fixed != nullptr, &b);
  if (ridge) carve_ridge(sz, F, cap, &rb);
  size_t extra = fixed ? 0 : sample_keys_scratch(F, !X->dense);
  TK_TRY(ws_reserve(h, sz.off + extra));
  TK_TRY(chol_reserve(h, F.d));
  Arena ar(h->ws);
  carve_sketch(ar, h, F, cap, prec, fixed != nullptr, &b);
  if (ridge) carve_ridge(ar, F, cap, &rb);
  ev_record(h, timing, 0);
  int64_t T = 0;
  const uint64_t* keys_u;
  const uint32_t* counts;
  const double* p_in = nullptr;
  bool tables_ready = false;
  const bool kpcg = kpcg_wanted(h, F, prec);
  h->chol.kres_n = 0;
  h->chol.kron_ready = 0;
  if (ridge) {
    // lambda-ridge leverage of K (Lemma 4.1): the factor eigenpairs (also the CG
    // preconditioner's), the column tables and mixture weights, m draws, dedupe,
    // and the probabilities of the distinct rows
    TK_TRY(ridge_tables(h, F, lambda, rb.tab_scratch, rb.usq, rb.c, rb.d_eff,
                        kpcg ? h->chol.kv : nullptr, kpcg ? h->chol.ke : nullptr));
    if (kpcg) {
      h->chol.kN = F.N;
      for (int n = 0; n < F.N; ++n) h->chol.kR[n] = F.R[n];
      h->chol.kron_ready = 1;
      TK_TRY(kron_ev_to_host(h));
    }
    ev_record(h, timing, 1);
    RidgeState rst;
    TK_TRY(ridge_draw(h, F, rb.usq, rb.c, m, seed, sweep, rb.samp_scratch, b.keys_raw, b.d_T,
                      &rst));
    T = m;
    ev_record(h, timing, 2);
    TK_TRY(sort_dedupe(h, b.keys_raw, m, bits_for(F.total), b.keys_u, b.counts, b.nu,
                       b.sort_scratch, b.sort_bytes));
    TK_TRY(ridge_prob(h, &rst, b.keys_u, b.nu, cap, rb.p));
    keys_u = b.keys_u;
    counts = b.counts;
    p_in = rb.p;
  } else if (!fixed) {
    TK_TRY(launch_leverage(h, F, b.lev, b.cdf, b.rank, nullptr, nullptr,
                           kpcg ? b.fgram : nullptr));
    ev_record(h, timing, 1);
    // the gather's probability tables need only the CDFs: built on the second
    // stream beside the sampling and the dedupe, joined before the gather
    TK_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
    TK_CUDA(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    {
      cudaStream_t main_stream = h->stream;
      h->stream = h->aux;
      tucker_status st = launch_prob_tables(h, F, b.cdf, b.ptab);
      if (st == TUCKER_OK) st = cudaEventRecord(h->ev_join, h->aux) == cudaSuccess ? TUCKER_OK
                                                                               : TUCKER_ECUDA;
      // the CG preconditioner's eigendecompositions of the factor Grams, behind the
      // tables on the second stream (joined before the solve, with the right-hand side)
      if (st == TUCKER_OK && kpcg) st = kron_prepare(h, F, b.fgram);
      h->stream = main_stream;
      if (st == TUCKER_ECUDA && !h->err[0]) return fail(h, st, "cudaEventRecord on the second stream");
      TK_TRY(st);
    }
    tables_ready = true;
    TK_TRY(sample_keys(h, F, b.cdf, m, seed, sweep, reg, X->dense ? nullptr : X, 0, b.keys_raw,
                       b.d_T, &T, ar));
    ev_record(h, timing, 2);
    const uint64_t key_range = F.total + (reg == TUCKER_REG_AUGMENTED ? (uint64_t)F.d : 0);
    TK_TRY(sort_dedupe(h, b.keys_raw, m, bits_for(key_range), b.keys_u, b.counts, b.nu,
                       b.sort_scratch, b.sort_bytes));
    keys_u = b.keys_u;
    counts = b.counts;
  } else {
    ev_record(h, timing, 1);
    ev_record(h, timing, 2);
    int nuh = (int)fixed->n_unique;
    T = fixed->n_draws;
    TK_CUDA(h, cudaMemcpyAsync(b.nu, &nuh, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    TK_CUDA(h, cudaMemcpyAsync(b.d_T, &fixed->n_draws, sizeof(int64_t), cudaMemcpyHostToDevice,
                               h->stream));
    keys_u = fixed->keys;
    counts = fixed->counts;
    p_in = fixed->prob;
    if (kpcg) {
      TK_TRY(launch_leverage(h, F, b.lev, b.cdf, b.rank, nullptr, nullptr, b.fgram));
      TK_TRY(kron_prepare(h, F, b.fgram));
    }
    if (!X->dense) { int pr; TK_TRY(hash_ensure(h, X, &pr)); }
    TK_CUDA(h, cudaStreamSynchronize(h->stream));   // host values above are stack-held
  }
  ev_record(h, timing, 3);
  if (tables_ready) TK_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  TK_TRY(launch_gather(h, F, b.cdf, greg, keys_u, counts, b.nu, b.d_T, X, cap, b.idx, b.w, b.x,
                       b.p, b.sw32, b.nreal, b.D, p_in, b.ptab, tables_ready));
  ev_record(h, timing, 4);
  RowSet rs = make_rowset(F, b.idx, b.w, b.nreal);
  RowSet rs64;
  double* G = h->chol.L;
  // the FP64 factor copies, the walk tables and the right-hand side h = K_S^T W x
  // do not depend on the Gram; when the factorisation occupies one thread-block
  // cluster (mixed solver, small d) they run on the second stream beside the
  // Gram and the factorisation and are joined before the solve (a grid-wide
  // factorisation needs every SM, so there everything stays in order)
  const bool beside = (h->solver == TUCKER_SOLVER_MIXED && chol32_on_cluster(h, F.d)) || kpcg;
  auto rhs_chain = [&]() -> tucker_status {
    TK_TRY(rowset64(h, F, rs, b.A64, &rs64));
    TK_TRY(walk_segments(h, rs, F.I[0], b.walk));
    return rows_axpy(h, F, rs64, b.walk, b.axpy_split, b.axpy_part, b.w, b.x, 1.0, nullptr,
                     nullptr, nullptr, b.h);
  };
  if (beside) {
    TK_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
    TK_CUDA(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    cudaStream_t main_stream = h->stream;
    h->stream = h->aux;
    const tucker_status st = rhs_chain();
    h->stream = main_stream;
    TK_TRY(st);
    TK_CUDA(h, cudaEventRecord(h->ev_join, h->aux));
    TK_TRY(build_gram(h, F, rs, prec, cap, b, G));
  } else {
    TK_TRY(build_gram(h, F, rs, prec, cap, b, G));
    TK_TRY(rhs_chain());
  }
  TK_TRY(launch_regdiag(h, h->chol.regdiag, F.d, lambda,
                        reg == TUCKER_REG_AUGMENTED ? b.D : nullptr));
  ev_record(h, timing, 5);
  int iters = 0;
  double rel = 0.0;
  TK_TRY(launch_add_diag(h, h->chol.L, F.d, h->chol.regdiag));
  TK_TRY(factorize(h, h->chol.L, F.d, prec, h->solver));
  if (beside) TK_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
  int prec_used = prec;
  TK_TRY(solve_robust(h, F, rs, rs64, prec, b, &iters, &rel, &rs, &prec_used));
  TK_CUDA(h, cudaMemcpyAsync(core_out, b.g, sizeof(double) * F.d, cudaMemcpyDeviceToDevice,
                             h->stream));
  ev_record(h, timing, 6);
  h->chol.id = h->next_solve_id++;
  if (timing) {
    tucker_status st = device_status(h);
    memset(stats, 0, sizeof(*stats));
    stats->ms_leverage = ev_ms(h, 0, 1);
    stats->ms_sample = ev_ms(h, 1, 2);
    stats->ms_dedupe = ev_ms(h, 2, 3);
    stats->ms_gather = ev_ms(h, 3, 4);
    stats->ms_gram = ev_ms(h, 4, 5);
    stats->ms_solve = ev_ms(h, 5, 6);
    stats->ms_total = ev_ms(h, 0, 6);
    int nuh = 0, nrh = 0;
    cudaMemcpy(&nuh, b.nu, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemcpy(&nrh, b.nreal, sizeof(int), cudaMemcpyDeviceToHost);
    stats->n_unique = nuh;
    stats->n_real = nrh;
    stats->n_draws = T;
    stats->refine_iters = iters;
    stats->refine_rel = rel;
    stats->solve_id = h->chol.id;
    stats->launches = h->launches - launches0;
    stats->ms_factor = ev_ms(h, 8, 9);
    stats->ms_gram_kernel = ev_ms(h, 10, 11);
    stats->gram_prec_used = prec_used;
    if (h->chol.kres_n > 0) {             // CG solves ran (negative: the factor took over)
      stats->ms_inner = ev_ms(h, 12, 13);
      double kr[2 * kKresSlots];
      const int nk = std::min(h->chol.kres_n, kKresSlots);
      cudaMemcpy(kr, h->chol.kres, 2 * nk * sizeof(double), cudaMemcpyDeviceToHost);
      for (int k = 0; k < nk; ++k) stats->inner_iters += (int64_t)kr[2 * k];
      if (!h->chol.kpcg) stats->inner_iters = -stats->inner_iters;
    }
    if (st != TUCKER_OK) h->chol.id = 0;
    return st;
  }
  tucker_status st = finish(h);
  if (st != TUCKER_OK) h->chol.id = 0;
  return st;
}

tucker_status tucker_core_update_exact(tucker_handle* h, const tucker_tensor* X, const int* R,
                                       const void* const* A, double lambda, tucker_prec prec,
                                       double* core_out) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, A, &F));
  if (!A || !core_out) return fail(h, TUCKER_EINVAL, "null factors or core_out");
  if (!(lambda >= 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be >= 0");
  if (X->dense) {
    const int N = F.N;
    const int64_t inter = (int64_t)(F.total / (uint64_t)F.I[N - 1]) * F.R[N - 1];
    auto carve = [&](Arena& ar, double** lev, uint64_t** cdf, double** V, double** s, int** rk,
                     double** b0, double** b1, double** y) {
      for (int n = 0; n < N; ++n) {
        lev[n] = ar.get<double>(F.I[n]);
        cdf[n] = ar.get<uint64_t>(F.I[n]);
        V[n] = ar.get<double>(F.R[n] * F.R[n]);
        s[n] = ar.get<double>(F.R[n]);
      }
      *rk = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(max_dim(F))));
      *b0 = ar.get<double>(inter);
      *b1 = ar.get<double>(inter);
      *y = ar.get<double>(F.d);
    };
    double *lev[TUCKER_MAX_ORDER], *V[TUCKER_MAX_ORDER], *s[TUCKER_MAX_ORDER];
    uint64_t* cdf[TUCKER_MAX_ORDER];
    int* rk;
    double *b0, *b1, *y;
    Arena sz(nullptr);
    carve(sz, lev, cdf, V, s, &rk, &b0, &b1, &y);
    TK_TRY(ws_reserve(h, sz.off));
    Arena ar(h->ws);
    carve(ar, lev, cdf, V, s, &rk, &b0, &b1, &y);
    // the factor eigendecompositions (a latency-bound FP64 Jacobi on a few SMs)
    // on the second stream, beside the pass over X; joined before the core solve
    TK_CUDA(h, cudaEventRecord(h->ev_fork, h->stream));
    TK_CUDA(h, cudaStreamWaitEvent(h->aux, h->ev_fork, 0));
    {
      cudaStream_t main_stream = h->stream;
      h->stream = h->aux;
      tucker_status st = launch_leverage(h, F, lev, cdf, rk, V, s, nullptr);
      if (st == TUCKER_OK && cudaEventRecord(h->ev_join, h->aux) != cudaSuccess) st = TUCKER_ECUDA;
      h->stream = main_stream;
      if (st == TUCKER_ECUDA && !h->err[0]) return fail(h, st, "cudaEventRecord on the second stream");
      TK_TRY(st);
    }
    TK_TRY(ttm_chain_all(h, F, X->dense, b0, b1, y));
    TK_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_join, 0));
    TK_TRY(kron_eig_core(h, F, V, s, y, lambda, core_out));
    return finish(h);
  }
  // missing entries: Gram of all observed rows, FP64 Cholesky (+ refinement)
  const int64_t nnz = X->nnz;
  if (nnz >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "nnz must be < 2^31");
  SketchBufs b;
  memset(&b, 0, sizeof(b));
  Arena sz(nullptr);
  carve_sketch(sz, h, F, nnz, prec, 1, &b);
  TK_TRY(ws_reserve(h, sz.off));
  TK_TRY(chol_reserve(h, F.d));
  Arena ar(h->ws);
  carve_sketch(ar, h, F, nnz, prec, 1, &b);
  int nn = (int)nnz;
  TK_CUDA(h, cudaMemcpyAsync(b.nreal, &nn, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  TK_TRY(launch_decode_rows(h, F, X->keys, nnz, b.idx, X->vals, b.x));
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  RowSet rs = make_rowset(F, b.idx, nullptr, b.nreal);
  // unit weights: w = 1 for every observed row (the fill kernel's 32-bit
  // grid-stride index covers 2^30 entries per launch)
  for (int64_t off = 0; off < nnz; off += int64_t(1) << 30)
    TK_TRY(launch_regdiag(h, b.w + off, (int)std::min<int64_t>(nnz - off, int64_t(1) << 30), 1.0,
                          nullptr));
  rs.w = b.w;
  RowSet rs64;
  TK_TRY(rowset64(h, F, rs, b.A64, &rs64));
  double* G = h->chol.L;
  TK_TRY(walk_segments(h, rs, F.I[0], b.walk));
  TK_TRY(build_gram(h, F, rs, prec, nnz, b, G));
  TK_TRY(rows_axpy(h, F, rs64, b.walk, b.axpy_split, b.axpy_part, b.w, b.x, 1.0, nullptr, nullptr,
                   nullptr, b.h));
  TK_TRY(launch_regdiag(h, h->chol.regdiag, F.d, lambda, nullptr));
  h->chol.kres_n = 0;
  h->chol.kron_ready = 0;
  if (kpcg_wanted(h, F, prec)) {
    TK_TRY(launch_leverage(h, F, b.lev, b.cdf, b.rank, nullptr, nullptr, b.fgram));
    TK_TRY(kron_prepare(h, F, b.fgram));
  }
  int iters;
  double rel;
  TK_TRY(solve_refine(h, F, rs, rs64, prec, b, &iters, &rel));
  TK_CUDA(h, cudaMemcpyAsync(core_out, b.g, sizeof(double) * F.d, cudaMemcpyDeviceToDevice,
                             h->stream));
  return finish(h);
}

// ------------------------------------------------ missing-data beta (Sec. 4.2)
struct FactorEigs {
  double* lev[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  double* V[TUCKER_MAX_ORDER];
  double* ev[TUCKER_MAX_ORDER];
  int* rk;
};

static void carve_eigs(Arena& ar, const FactorSet& F, FactorEigs* e) {
  for (int n = 0; n < F.N; ++n) {
    e->lev[n] = ar.get<double>(F.I[n]);
    e->cdf[n] = ar.get<uint64_t>(F.I[n]);
    e->V[n] = ar.get<double>(F.R[n] * F.R[n]);
    e->ev[n] = ar.get<double>(F.R[n]);
  }
  e->rk = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(max_dim(F))));
}

// Alg. 1 line 3 as a real number (it may exceed any integer type).
static double alg1_count(int d, double eps, double delta, double beta_prime) {
  return ceil(4.0 * d / beta_prime * fmax(420.0 * log(4.0 * d / delta), 1.0 / (delta * eps)));
}

tucker_status tucker_missing_beta(tucker_handle* h, const tucker_tensor* X, const int* R,
                                  const void* const* A, double lambda, tucker_beta_mode mode,
                                  tucker_prec prec, double eps, double delta,
                                  tucker_missing_beta_info* out) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, A, &F));
  if (!A || !out) return fail(h, TUCKER_EINVAL, "null factors or out");
  if (!(lambda > 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be > 0 (Thm 4.3)");
  if (!(eps > 0 && eps < 1 && delta > 0 && delta < 1))
    return fail(h, TUCKER_EINVAL, "eps, delta must be in (0,1)");
  if (mode != TUCKER_BETA_BOUND && mode != TUCKER_BETA_EXACT) return fail(h, TUCKER_EINVAL, "mode");
  if (prec < TUCKER_PREC_FP64 || prec > TUCKER_PREC_BF16) return fail(h, TUCKER_EINVAL, "prec");
  const bool gram = mode == TUCKER_BETA_EXACT && !X->dense;
  const int d = F.d;
  if (gram && d > 4096) return fail(h, TUCKER_ENOTSUP, "exact missing-data beta needs d <= 4096");
  if (gram && X->nnz >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "nnz must be < 2^31");
  memset(out, 0, sizeof(*out));
  FactorEigs e;
  SketchBufs b;
  memset(&b, 0, sizeof(b));
  double *T1 = nullptr, *C = nullptr, *vx = nullptr, *vy = nullptr, *nrm = nullptr, *dg = nullptr;
  auto carve = [&](Arena& ar) {
    carve_eigs(ar, F, &e);
    if (!gram) return;
    carve_sketch(ar, h, F, X->nnz, prec, 1, &b);
    T1 = ar.get<double>((size_t)d * d);
    C = ar.get<double>((size_t)d * d);
    vx = ar.get<double>(d);
    vy = ar.get<double>(d);
    dg = ar.get<double>(d);
    nrm = ar.get<double>(1);
  };
  Arena sz(nullptr);
  carve(sz);
  TK_TRY(ws_reserve(h, sz.off));
  if (gram) TK_TRY(chol_reserve(h, d));
  Arena ar(h->ws);
  carve(ar);
  // factor eigenpairs (FP64 Jacobi of A^(n)T A^(n)), eigenvalues to the host
  TK_TRY(launch_leverage(h, F, e.lev, e.cdf, e.rk, e.V, e.ev, nullptr));
  double evh[TUCKER_MAX_ORDER][TUCKER_MAX_RANK];
  for (int n = 0; n < F.N; ++n)
    TK_CUDA(h, cudaMemcpyAsync(evh[n], e.ev[n], sizeof(double) * F.R[n], cudaMemcpyDeviceToHost,
                               h->stream));
  TK_TRY(device_status(h));
  // P_max = prod_n ||A^(n)||_2^2; c_min = P_min / (P_min + lambda) with P_min the
  // product of the smallest eigenvalues above the pseudo-inverse cutoff
  double pmax = 1.0, pmin = 1.0;
  for (int n = 0; n < F.N; ++n) {
    double top = 0.0;
    for (int k = 0; k < F.R[n]; ++k) top = fmax(top, evh[n][k]);
    const double cut = (double)std::max<int64_t>(F.I[n], F.R[n]) * DBL_EPSILON * top;
    double lo = top;
    for (int k = 0; k < F.R[n]; ++k)
      if (evh[n][k] > cut) lo = fmin(lo, evh[n][k]);
    pmax *= top;
    pmin *= lo;
  }
  if (!(pmax > 0.0) || !(pmin > 0.0)) return fail(h, TUCKER_ERANK, "a factor matrix is zero");
  out->c_min = pmin / (pmin + lambda);
  double lmax = 0.0;
  if (X->dense) {
    lmax = 0.0;                                   // nothing missing: beta_miss = 1
  } else if (mode == TUCKER_BETA_BOUND) {
    lmax = pmax / (pmax + lambda);                // the corollary to Thm 4.3
  } else {
    // K_S^T K_S over all observed rows, whitened: C = D^-1/2 Vk^T (G + lambda I) Vk D^-1/2
    h->chol.id = 0;                               // the cached factor is overwritten
    h->chol.kron_ready = 0;
    const int64_t nnz = X->nnz;
    int nn = (int)nnz;
    TK_CUDA(h, cudaMemcpyAsync(b.nreal, &nn, sizeof(int), cudaMemcpyHostToDevice, h->stream));
    TK_TRY(launch_decode_rows(h, F, X->keys, nnz, b.idx, X->vals, b.x));
    TK_CUDA(h, cudaStreamSynchronize(h->stream));
    RowSet rs = make_rowset(F, b.idx, nullptr, b.nreal);
    for (int64_t off = 0; off < nnz; off += int64_t(1) << 30)
      TK_TRY(launch_regdiag(h, b.w + off, (int)std::min<int64_t>(nnz - off, int64_t(1) << 30), 1.0,
                            nullptr));
    rs.w = b.w;
    double* G = h->chol.L;
    TK_TRY(walk_segments(h, rs, F.I[0], b.walk));
    TK_TRY(build_gram(h, F, rs, prec, nnz, b, G));
    TK_TRY(kron_whiten(h, F, e.V, e.ev, lambda, G, T1, C));
    // nu_min by inverse iteration: ||C^-1 x|| <= 1 / nu_min for unit x, so every
    // estimate 1 / ||C^-1 x_k|| is at or above nu_min and they decrease towards it
    TK_CUDA(h, cudaMemcpyAsync(G, C, sizeof(double) * d * d, cudaMemcpyDeviceToDevice, h->stream));
    TK_TRY(cholesky(h, G, d));
    TK_TRY(device_status(h));
    TK_TRY(chol_prepare(h, G, d, h->chol.LT, h->chol.Linv));
    std::vector<double> x0(d);
    for (int i = 0; i < d; ++i)                   // a fixed vector with no zero entry
      x0[i] = 1.0 + (double)((uint32_t)(i + 1) * 2654435761u >> 22) / 1024.0;
    TK_CUDA(h, cudaMemcpyAsync(vy, x0.data(), sizeof(double) * d, cudaMemcpyHostToDevice,
                               h->stream));
    TK_TRY(vec_normalize(h, vy, d, vx, nrm));
    double nu = HUGE_VAL;
    int it = 0;
    while (it < 200) {
      TK_TRY(chol_solve2(h, G, h->chol.LT, h->chol.Linv, d, vx, vy, h->chol.tmp));
      TK_TRY(vec_normalize(h, vy, d, vx, nrm));
      double nv = 0.0;
      TK_CUDA(h, cudaMemcpyAsync(&nv, nrm, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      TK_TRY(device_status(h));
      ++it;
      if (!(nv > 0.0)) return fail(h, TUCKER_EINTERNAL, "inverse iteration lost its vector");
      const double nn_ = 1.0 / nv;
      const bool conv = fabs(nu - nn_) <= 1e-12 * nn_;
      nu = nn_;
      if (conv) break;
    }
    out->nu_est = nu;
    out->iters = it;
    // certify nu_lo <= nu_min: C - nu_lo I has an FP64 Cholesky factor
    double nu_lo = 0.0;
    const double taus[] = {1e-6, 1e-4, 1e-2, 1e-1, 0.5};
    for (double tau : taus) {
      const double lo = nu * (1.0 - tau);
      TK_CUDA(h, cudaMemcpyAsync(G, C, sizeof(double) * d * d, cudaMemcpyDeviceToDevice,
                                 h->stream));
      TK_TRY(launch_regdiag(h, dg, d, -lo, nullptr));
      TK_TRY(launch_add_diag(h, G, d, dg));
      TK_TRY(cholesky(h, G, d));
      ++out->certify_tries;
      const tucker_status st = device_status(h);
      if (st == TUCKER_OK) {
        nu_lo = lo;
        break;
      }
      if (st != TUCKER_ENOTSPD) return st;
    }
    lmax = fmax(0.0, 1.0 - nu_lo);
  }
  out->lambda_max = lmax;
  out->beta_miss = X->dense ? 1.0 : (lmax < 1.0 ? 1.0 / (1.0 + 1.0 / (1.0 - lmax)) : 0.0);
  out->beta = out->c_min * out->beta_miss;
  out->beta_prime = fmin(out->beta, 1.0) / 2.0;
  out->s = out->beta_prime > 0.0 ? alg1_count(d, eps, delta, out->beta_prime) : HUGE_VAL;
  return TUCKER_OK;
}

tucker_status tucker_ridge_loss(tucker_handle* h, const tucker_tensor* X, const int* R,
                                const void* const* A, double lambda, const double* g,
                                double* loss_out_host) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, A, &F));
  if (!A || !g || !loss_out_host) return fail(h, TUCKER_EINVAL, "null argument");
  const int N = F.N;
  const int64_t rows = (int64_t)(F.total / (uint64_t)F.I[N - 1]) * F.R[N - 1];
  const int np = h->num_sms * 8;
  Arena sz(nullptr);
  sz.get<double>(rows); sz.get<double>(rows); sz.get<double>(np); sz.get<double>(4);
  TK_TRY(ws_reserve(h, sz.off));
  Arena ar(h->ws);
  double* b0 = ar.get<double>(rows);
  double* b1 = ar.get<double>(rows);
  double* part = ar.get<double>(np);
  double* res = ar.get<double>(4);
  TK_TRY(residual_sq(h, F, X, g, b0, b1, part, np, res));
  TK_TRY(sumsq(h, g, 1, F.d, part, np, res + 1));
  double hv[2];
  TK_CUDA(h, cudaMemcpyAsync(hv, res, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  TK_TRY(device_status(h));
  *loss_out_host = hv[0] + lambda * hv[1];
  return TUCKER_OK;
}

// ------------------------------------------------ sketched factor update
// Rows of the mode-n factor design B_n drawn from the product of the leverage
// scores of A^(k), k != n (the core sampler over those modes, Philox key word
// sweep + (n + 1) 2^32), deduplicated, and the weighted normal equations of
// the mode-n fibers (launch_fiber_update).
struct FsBufs {
  double* lev[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  int* rk;
  uint64_t* raw;
  int64_t* d_T;
  char* sort;
  size_t sort_bytes;
  uint64_t* keys_u;
  uint32_t* counts;
  int* nu;
  char* fws;
  size_t fws_bytes;
};

static FactorSet others_of(const FactorSet& F, int n) {
  FactorSet o;
  memset(&o, 0, sizeof(o));
  o.is64 = F.is64;
  o.d = F.d / F.R[n];
  o.total = F.total / (uint64_t)F.I[n];
  for (int k = 0; k < F.N; ++k) {
    if (k == n) continue;
    o.I[o.N] = F.I[k];
    o.R[o.N] = F.R[k];
    o.A[o.N] = F.A[k];
    ++o.N;
  }
  return o;
}

static void carve_fs(Arena& ar, const FactorSet& F, int n, int64_t m, FsBufs* b) {
  const FactorSet o = others_of(F, n);
  for (int k = 0; k < o.N; ++k) {
    b->lev[k] = ar.get<double>(o.I[k]);
    b->cdf[k] = ar.get<uint64_t>(o.I[k]);
  }
  b->rk = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(max_dim(o))));
  b->raw = ar.get<uint64_t>(m);
  b->d_T = ar.get<int64_t>(1);
  b->sort_bytes = sort_dedupe_scratch(m);
  b->sort = ar.get<char>(b->sort_bytes);
  b->keys_u = ar.get<uint64_t>(m);
  b->counts = ar.get<uint32_t>(m);
  b->nu = ar.get<int>(1);
  b->fws_bytes = fiber_workspace_bytes(F, n, m, fiber_splits(m));
  b->fws = ar.get<char>(b->fws_bytes);
}

static size_t fs_bytes(const FactorSet& F, int n, int64_t m) {
  Arena sz(nullptr);
  FsBufs b;
  carve_fs(sz, F, n, m, &b);
  return sz.off + sample_keys_scratch(others_of(F, n), false) + 4096;
}

static tucker_status factor_sketch_impl(tucker_handle* h, const FactorSet& F, const void* Xd,
                                        void* const* A, const double* core, int n, double lambda,
                                        int64_t m, uint64_t seed, uint32_t sweep, Arena& ar) {
  FsBufs b;
  carve_fs(ar, F, n, m, &b);
  const FactorSet o = others_of(F, n);
  TK_TRY(launch_leverage(h, o, b.lev, b.cdf, b.rk, nullptr, nullptr, nullptr));
  int64_t T_host = 0;
  TK_TRY(sample_keys(h, o, b.cdf, m, seed, (uint64_t)sweep + ((uint64_t)(n + 1) << 32),
                     TUCKER_REG_EXACT, nullptr, 0, b.raw, b.d_T, &T_host, ar));
  TK_TRY(sort_dedupe(h, b.raw, m, bits_for(o.total), b.keys_u, b.counts, b.nu, b.sort,
                     b.sort_bytes));
  return launch_fiber_update(h, F, n, Xd, core, b.keys_u, b.counts, b.nu, m, b.cdf, m, lambda,
                             b.fws, b.fws_bytes, A[n], core == nullptr);
}

tucker_status tucker_factor_update_sketched(tucker_handle* h, const tucker_tensor* X, const int* R,
                                            void* const* A_inout, const double* core, int n,
                                            double lambda, int64_t m, uint64_t seed,
                                            uint32_t sweep) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, (const void* const*)A_inout, &F));
  if (!X->dense) return fail(h, TUCKER_EINVAL, "the sketched factor update needs a dense X");
  if (!A_inout || !core) return fail(h, TUCKER_EINVAL, "null factors or core");
  if (F.N < 2) return fail(h, TUCKER_EINVAL, "order must be >= 2");
  if (n < 0 || n >= F.N) return fail(h, TUCKER_EINVAL, "mode %d out of range", n);
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
  if (!(lambda >= 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be >= 0");
  TK_TRY(ws_reserve(h, fs_bytes(F, n, m)));
  Arena ar(h->ws);
  TK_TRY(factor_sketch_impl(h, F, X->dense, A_inout, core, n, lambda, m, seed, sweep, ar));
  return finish(h);
}

// ----------------------------------------------- CP-ALS (Sec. 6's extension)
// The factor set of a rank-R CP model: every R_n = R.  d is not a Kronecker
// dimension here (the CP design has R columns), so prod R_n is not bounded.
static tucker_status cp_factors(tucker_handle* h, const tucker_tensor* X, int R,
                                void* const* A, FactorSet* F) {
  if (!X) return fail(h, TUCKER_EINVAL, "X is NULL");
  if (!X->dense) return fail(h, TUCKER_EINVAL, "the CP update needs a dense X");
  const int N = X->order;
  if (N < 2 || N > TUCKER_MAX_ORDER) return fail(h, TUCKER_EINVAL, "order %d out of range", N);
  if (R < 1 || R > TUCKER_MAX_RANK) return fail(h, TUCKER_EINVAL, "CP rank %d out of range", R);
  if (X->dtype != TUCKER_F32 && X->dtype != TUCKER_F64) return fail(h, TUCKER_EINVAL, "bad dtype");
  if (!A) return fail(h, TUCKER_EINVAL, "null factors");
  memset(F, 0, sizeof(*F));
  F->N = N;
  F->is64 = X->dtype == TUCKER_F64;
  double tot = 1.0;
  uint64_t total = 1;
  for (int n = 0; n < N; ++n) {
    if (X->dims[n] < 1 || X->dims[n] > (int64_t(1) << 31))
      return fail(h, TUCKER_EINVAL, "I_%d out of range", n);
    if (!A[n]) return fail(h, TUCKER_EINVAL, "factor %d is NULL", n);
    F->I[n] = X->dims[n];
    F->R[n] = R;
    F->A[n] = A[n];
    tot *= double(X->dims[n]);
    total *= (uint64_t)X->dims[n];
  }
  if (tot >= 4.0e18) return fail(h, TUCKER_EINVAL, "prod(I_n) too large");
  F->d = R;
  F->total = total;
  return TUCKER_OK;
}

tucker_status tucker_cp_factor_update_sketched(tucker_handle* h, const tucker_tensor* X, int R,
                                               void* const* A_inout, int n, double lambda,
                                               int64_t m, uint64_t seed, uint32_t sweep) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(cp_factors(h, X, R, A_inout, &F));
  if (n < 0 || n >= F.N) return fail(h, TUCKER_EINVAL, "mode %d out of range", n);
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
  if (!(lambda >= 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be >= 0");
  TK_TRY(ws_reserve(h, fs_bytes(F, n, m)));
  Arena ar(h->ws);
  TK_TRY(factor_sketch_impl(h, F, X->dense, A_inout, nullptr, n, lambda, m, seed, sweep, ar));
  return finish(h);
}

tucker_status tucker_cp_als_sweep(tucker_handle* h, const tucker_tensor* X, int R,
                                  void* const* A_inout, double lambda, int64_t m, uint64_t seed,
                                  uint32_t sweep) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(cp_factors(h, X, R, A_inout, &F));
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
  if (!(lambda >= 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be >= 0");
  size_t need = 0;
  for (int n = 0; n < F.N; ++n) need = std::max(need, fs_bytes(F, n, m));
  TK_TRY(ws_reserve(h, need));
  for (int n = 0; n < F.N; ++n) {
    Arena ar(h->ws);
    TK_TRY(factor_sketch_impl(h, F, X->dense, A_inout, nullptr, n, lambda, m, seed, sweep, ar));
  }
  return finish(h);
}

tucker_status tucker_set_factor_sketch(tucker_handle* h, int64_t m) {
  if (!h) return TUCKER_EINVAL;
  if (m < 0 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
  h->factor_m = m;
  return TUCKER_OK;
}

tucker_status tucker_als_sweep(tucker_handle* h, const tucker_tensor* X, const int* R,
                               void* const* A_inout, double* core_inout, double lambda,
                               int sketched, int64_t m, uint64_t seed, uint32_t sweep,
                               tucker_reg reg, tucker_prec prec, double* loss_out_host,
                               double* rmse_out_host) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, (const void* const*)A_inout, &F));
  if (!X->dense) return fail(h, TUCKER_EINVAL, "ALS sweep needs a dense X");
  if (!A_inout || !core_inout) return fail(h, TUCKER_EINVAL, "null factors or core");
  if (!(lambda >= 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be >= 0");
  if (F.N < 2) return fail(h, TUCKER_EINVAL, "ALS needs order >= 2");
  const int N = F.N;
  // largest intermediate of the mode-n product chains
  int64_t inter = 0;
  for (int n = 0; n < N; ++n) {
    int first = (n != N - 1) ? N - 1 : N - 2;
    int64_t e = (int64_t)(F.total / (uint64_t)F.I[first]) * F.R[first];
    if (e > inter) inter = e;
  }
  const int np = h->num_sms * 8;
  double* Ls = nullptr;                           // the R_n x R_n factor of a factor update
  double* Ylast = nullptr;                        // X x_N A^(N)T, shared by modes 1..N-1
  auto carve = [&](Arena& ar, double** lev, uint64_t** cdf, double** gram, int** rk, double** b0,
                   double** b1, double** B, double** part, double** res) {
    Ls = ar.get<double>(TUCKER_MAX_RANK * TUCKER_MAX_RANK);
    Ylast = N >= 3 ? ar.get<double>(inter) : nullptr;
    for (int n = 0; n < N; ++n) {
      lev[n] = ar.get<double>(F.I[n]);
      cdf[n] = ar.get<uint64_t>(F.I[n]);
      gram[n] = ar.get<double>(F.R[n] * F.R[n]);
    }
    *rk = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(max_dim(F))));
    *b0 = ar.get<double>(inter);
    *b1 = ar.get<double>(inter);
    *B = ar.get<double>(inter);
    *part = ar.get<double>(np);
    *res = ar.get<double>(3 + N);
  };
  double *lev[TUCKER_MAX_ORDER], *gram[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  int* rk;
  double *b0, *b1, *B, *part, *res;
  Arena sz(nullptr);
  carve(sz, lev, cdf, gram, &rk, &b0, &b1, &B, &part, &res);
  const int64_t mf = h->factor_m;                 // > 0: sketched factor updates
  size_t fsb = 0;
  if (mf > 0)
    for (int n = 0; n < N; ++n) fsb = std::max(fsb, fs_bytes(F, n, mf));
  TK_TRY(ws_reserve(h, sz.off + fsb + 256));
  Arena ar(h->ws);
  carve(ar, lev, cdf, gram, &rk, &b0, &b1, &B, &part, &res);
  const bool want_loss = loss_out_host || rmse_out_host;
  bool xx_done = false;                           // ||X||^2 formed with the shared product
  for (int n = 0; n < N; ++n) {
    if (mf > 0) {
      Arena fa(h->ws + ((ar.off + 255) & ~size_t(255)));
      TK_TRY(factor_sketch_impl(h, F, X->dense, A_inout, core_inout, n, lambda, mf, seed, sweep,
                                fa));
      continue;
    }
    TK_TRY(launch_factor_grams(h, F, rk, gram));
    // the chains of modes 1..N-1 start with X x_N A^(N)T, and A^(N) changes only
    // in the last update: one pass over X serves them all (N >= 3)
    const bool shared = Ylast && n < N - 1;
    if (shared && n == 0) {                       // with ||X||^2 for the loss, same pass
      int64_t P = 1;
      for (int k = 0; k < N - 1; ++k) P *= F.I[k];
      TK_TRY(ttm_last(h, X->dense, F.is64, P, (int)F.I[N - 1], F.A[N - 1], F.R[N - 1], Ylast,
                      want_loss ? part : nullptr, np, h->keep + F.d));
      xx_done = want_loss;
    }
    TK_TRY(ttm_chain_except(h, F, X->dense, n, b0, b1, B, shared ? Ylast : nullptr));
    TK_TRY(factor_solve(h, F, n, gram, core_inout, B, lambda, A_inout[n], Ls));
  }
  // the loss by the Gram identity needs y = K^T vec(X) for the new factors: the last
  // product chain B = X x_{k<N} A^(k)T (formed here when the factor updates were
  // sketched), times the new A^(N); and ||X||^2 (one pass)
  if (want_loss) {
    if (mf > 0) TK_TRY(ttm_chain_except(h, F, X->dense, N - 1, b0, b1, B));
    TK_TRY(kt_x_from_last(h, F, B, h->keep));
    if (!xx_done)
      TK_TRY(tensor_sumsq(h, X->dense, F.is64, (int64_t)F.total, part, np, h->keep + F.d));
  }
  TK_TRY(device_status(h));
  tucker_status st;
  if (sketched)
    st = tucker_core_update_sketched(h, X, R, (const void* const*)A_inout, lambda, m, 0.1, 0.1,
                                     seed, sweep, reg, prec, nullptr, core_inout, nullptr);
  else
    st = tucker_core_update_exact(h, X, R, (const void* const*)A_inout, lambda, prec, core_inout);
  if (st != TUCKER_OK) return st;
  if (loss_out_host || rmse_out_host) {
    // workspace may have been regrown by the core update: carve again
    Arena sz2(nullptr);
    carve(sz2, lev, cdf, gram, &rk, &b0, &b1, &B, &part, &res);
    TK_TRY(ws_reserve(h, sz2.off));
    Arena ar2(h->ws);
    carve(ar2, lev, cdf, gram, &rk, &b0, &b1, &B, &part, &res);
    // L = ||X||^2 - 2 g.y + g.(x_n A^(n)T A^(n)) g + lambda (||g||^2 + sum_n ||A^(n)||^2)
    // (the objective of Sec. 2 expanded; FP64), with the Grams of the new factors
    TK_TRY(launch_factor_grams(h, F, rk, gram));
    TK_TRY(kron_quad(h, F, gram, core_inout, h->keep, res));
    for (int n = 0; n < N; ++n)
      TK_TRY(sumsq(h, A_inout[n], F.is64, F.I[n] * F.R[n], part, np, res + 3 + n));
    double hv[3 + TUCKER_MAX_ORDER], xx = 0.0;
    TK_CUDA(h, cudaMemcpyAsync(hv, res, (3 + N) * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    TK_CUDA(h, cudaMemcpyAsync(&xx, h->keep + F.d, sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
    TK_TRY(device_status(h));
    const double resid = xx - 2.0 * hv[1] + hv[0];
    double reg_sum = hv[2];
    for (int n = 0; n < N; ++n) reg_sum += hv[3 + n];
    if (loss_out_host) *loss_out_host = resid + lambda * reg_sum;
    if (rmse_out_host) *rmse_out_host = sqrt(fmax(resid, 0.0) / (double)F.total);
  }
  return TUCKER_OK;
}

tucker_status tucker_sketched_gram(tucker_handle* h, const tucker_tensor* X, const int* R,
                                   const void* const* A, tucker_prec prec,
                                   const tucker_samples* samples, double* G_out, double* h_out) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, A, &F));
  if (!A || !samples || !G_out) return fail(h, TUCKER_EINVAL, "null argument");
  if (!samples->keys || !samples->counts || !samples->prob || samples->n_unique < 1 ||
      samples->n_draws < 1)
    return fail(h, TUCKER_EINVAL, "incomplete sample");
  if (prec < TUCKER_PREC_FP64 || prec > TUCKER_PREC_BF16) return fail(h, TUCKER_EINVAL, "prec");
  const int64_t cap = samples->n_unique;
  SketchBufs b;
  memset(&b, 0, sizeof(b));
  Arena sz(nullptr);
  carve_sketch(sz, h, F, cap, prec, 1, &b);
  TK_TRY(ws_reserve(h, sz.off));
  Arena ar(h->ws);
  carve_sketch(ar, h, F, cap, prec, 1, &b);
  int nuh = (int)cap;
  int64_t T = samples->n_draws;
  TK_CUDA(h, cudaMemcpyAsync(b.nu, &nuh, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  TK_CUDA(h, cudaMemcpyAsync(b.d_T, &T, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  if (!X->dense) { int pr; TK_TRY(hash_ensure(h, X, &pr)); }
  TK_TRY(launch_gather(h, F, b.cdf, TUCKER_REG_EXACT, samples->keys, samples->counts, b.nu,
                       b.d_T, X, cap, b.idx, b.w, b.x, b.p, b.sw32, b.nreal, b.D, samples->prob,
                       nullptr));
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  RowSet rs = make_rowset(F, b.idx, b.w, b.nreal);
  RowSet rs64;
  TK_TRY(rowset64(h, F, rs, b.A64, &rs64));
  TK_TRY(walk_segments(h, rs, F.I[0], b.walk));
  TK_TRY(build_gram(h, F, rs, prec, cap, b, G_out));
  if (h_out)
    TK_TRY(rows_axpy(h, F, rs64, b.walk, b.axpy_split, b.axpy_part, b.w, b.x, 1.0, nullptr, nullptr,
                     nullptr, h_out));
  return finish(h);
}

tucker_status tucker_core_solve_adjoint(tucker_handle* h, const tucker_tensor* X, const int* R,
                                        const void* const* A, double lambda, tucker_reg reg,
                                        tucker_prec prec, const tucker_samples* samples,
                                        uint64_t solve_id, const double* g, const double* gbar,
                                        double* const* dA_out, double* dx_out) {
  if (!h) return TUCKER_EINVAL;
  FactorSet F;
  TK_TRY(check_tensor(h, X, R, A, &F));
  if (!A || !samples || !g || !gbar || !dA_out || !dx_out)
    return fail(h, TUCKER_EINVAL, "null argument");
  if (!samples->keys || !samples->counts || !samples->prob || samples->n_unique < 1 ||
      samples->n_draws < 1)
    return fail(h, TUCKER_EINVAL, "incomplete sample");
  for (int n = 0; n < F.N; ++n) if (!dA_out[n]) return fail(h, TUCKER_EINVAL, "dA_out NULL");
  const int64_t cap = samples->n_unique;
  SketchBufs b;
  memset(&b, 0, sizeof(b));
  Arena sz(nullptr);
  carve_sketch(sz, h, F, cap, prec, 1, &b);
  double* v = sz.get<double>(F.d);
  double* zv = sz.get<double>(cap);
  TK_TRY(ws_reserve(h, sz.off));
  const bool reuse = solve_id != 0 && solve_id == h->chol.id && h->chol.d == F.d;
  if (!reuse) TK_TRY(chol_reserve(h, F.d));
  Arena ar(h->ws);
  carve_sketch(ar, h, F, cap, prec, 1, &b);
  v = ar.get<double>(F.d);
  zv = ar.get<double>(cap);
  int nuh = (int)cap;
  int64_t T = samples->n_draws;
  TK_CUDA(h, cudaMemcpyAsync(b.nu, &nuh, sizeof(int), cudaMemcpyHostToDevice, h->stream));
  TK_CUDA(h, cudaMemcpyAsync(b.d_T, &T, sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  if (!X->dense) { int pr; TK_TRY(hash_ensure(h, X, &pr)); }
  const int greg = reg == TUCKER_REG_RIDGE ? TUCKER_REG_EXACT : reg;   // p comes with the sample
  TK_TRY(launch_gather(h, F, b.cdf, greg, samples->keys, samples->counts, b.nu, b.d_T, X, cap,
                       b.idx, b.w, b.x, b.p, b.sw32, b.nreal, b.D, samples->prob, nullptr));
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  RowSet rs = make_rowset(F, b.idx, b.w, b.nreal);
  RowSet rs64;
  TK_TRY(rowset64(h, F, rs, b.A64, &rs64));
  TK_TRY(walk_segments(h, rs, F.I[0], b.walk));
  h->chol.kres_n = 0;
  if (!reuse) {
    h->chol.kron_ready = 0;
    if (kpcg_wanted(h, F, prec)) {
      TK_TRY(launch_leverage(h, F, b.lev, b.cdf, b.rank, nullptr, nullptr, b.fgram));
      TK_TRY(kron_prepare(h, F, b.fgram));
    }
    TK_TRY(build_gram(h, F, rs, prec, cap, b, h->chol.L));
    TK_TRY(launch_regdiag(h, h->chol.regdiag, F.d, lambda,
                          reg == TUCKER_REG_AUGMENTED ? b.D : nullptr));
    TK_TRY(launch_add_diag(h, h->chol.L, F.d, h->chol.regdiag));
    TK_TRY(factorize(h, h->chol.L, F.d, prec, h->solver));
    h->chol.id = h->next_solve_id++;
  }
  int iters;
  double rel;
  TK_TRY(solve_checked(h, F, rs64, prec, b, gbar, v, &iters, &rel));
  TK_TRY(rows_dot(h, F, rs64, b.walk, g, v, b.z, zv));
  TK_CUDA(h, cudaMemsetAsync(dx_out, 0, sizeof(double) * cap, h->stream));
  TK_TRY(launch_adjoint_rows(h, F, b.idx, b.w, b.x, b.z, zv, g, v, b.nreal, cap, dA_out, dx_out));
  return finish(h);
}

tucker_status tucker_ridge_tables(tucker_handle* h, int N, const int64_t* I, const int* R,
                                  tucker_dtype dtype, const void* const* A, double lambda,
                                  double* const* usq_out, double* c_out, int* K_out_host,
                                  double* d_eff_out_host) {
  if (!h) return TUCKER_EINVAL;
  if (!A || !usq_out || !c_out) return fail(h, TUCKER_EINVAL, "null factors or outputs");
  if (!(lambda >= 0.0)) return fail(h, TUCKER_EINVAL, "lambda must be >= 0");
  FactorSet F;
  TK_TRY(make_factors(h, N, I, R, dtype, A, &F));
  for (int n = 0; n < N; ++n)
    if (!usq_out[n]) return fail(h, TUCKER_EINVAL, "usq_out[%d] is NULL", n);
  Arena sz(nullptr);
  double* deff = sz.get<double>(1);
  char* scratch = sz.get<char>(ridge_tables_scratch(F));
  TK_TRY(ws_reserve(h, sz.off));
  Arena ar(h->ws);
  deff = ar.get<double>(1);
  scratch = ar.get<char>(ridge_tables_scratch(F));
  TK_TRY(ridge_tables(h, F, lambda, scratch, usq_out, c_out, deff, nullptr, nullptr));
  if (K_out_host) ridge_components(F, K_out_host);
  if (d_eff_out_host) {
    TK_CUDA(h, cudaMemcpyAsync(d_eff_out_host, deff, sizeof(double), cudaMemcpyDeviceToHost,
                               h->stream));
    return device_status(h);
  }
  return finish(h);
}

tucker_status tucker_sample_rows_ridge(tucker_handle* h, int N, const int64_t* I, const int* K,
                                       const double* const* usq, const double* c, int64_t m,
                                       uint64_t seed, uint32_t sweep, tucker_samples* out) {
  if (!h) return TUCKER_EINVAL;
  if (!usq || !c || !out || !out->keys || !out->counts || !out->prob)
    return fail(h, TUCKER_EINVAL, "null tables or output arrays");
  if (m < 1 || m >= (int64_t(1) << 31)) return fail(h, TUCKER_EINVAL, "m out of range");
  if (out->capacity < m) return fail(h, TUCKER_ECAPACITY, "capacity %lld < m %lld",
                                     (long long)out->capacity, (long long)m);
  FactorSet F;
  TK_TRY(make_factors(h, N, I, K, TUCKER_F64, nullptr, &F));
  for (int n = 0; n < N; ++n) {
    if (!usq[n]) return fail(h, TUCKER_EINVAL, "usq[%d] is NULL", n);
    if (K[n] > I[n]) return fail(h, TUCKER_EINVAL, "K_%d > I_%d", n, n);
  }
  Arena sz(nullptr);
  auto carve = [&](Arena& ar, uint64_t** raw, int64_t** dT, char** ss, int** nu, char** rs) {
    *raw = ar.get<uint64_t>(m);
    *dT = ar.get<int64_t>(1);
    *ss = ar.get<char>(sort_dedupe_scratch(m));
    *nu = ar.get<int>(1);
    *rs = ar.get<char>(ridge_sample_scratch(F, m));
  };
  uint64_t* raw;
  int64_t* dT;
  char *ss, *rs;
  int* nu;
  carve(sz, &raw, &dT, &ss, &nu, &rs);
  TK_TRY(ws_reserve(h, sz.off));
  Arena ar(h->ws);
  carve(ar, &raw, &dT, &ss, &nu, &rs);
  RidgeState st;
  TK_TRY(ridge_draw(h, F, usq, c, m, seed, sweep, rs, raw, dT, &st));
  TK_TRY(sort_dedupe(h, raw, m, bits_for(F.total), out->keys, out->counts, nu, ss,
                     sort_dedupe_scratch(m)));
  TK_TRY(ridge_prob(h, &st, out->keys, nu, m, out->prob));
  int nuh = 0;
  TK_CUDA(h, cudaMemcpyAsync(&nuh, nu, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  TK_TRY(device_status(h));
  out->n_unique = nuh;
  out->n_draws = m;
  return TUCKER_OK;
}

}  // extern "C"
