// Sampling rows of K from its lambda-ridge leverage distribution
// l^lam(K) / d_eff(K) (Lemma 4.1 with lambda > 0; Eq. d_eff_def), and the
// sample count of Alg. 1 line 3 with beta' from Eq. beta_prime.
//
// Lemma 4.1: with the thin SVDs A^(n) = U^(n) S^(n) V^(n)T,
//     l^lam_i(K) = sum_t c_t prod_n (u^(n)_{i_n t_n})^2,   c_t = P_t / (P_t + lam),
//     P_t = prod_n s^2_{t_n}(A^(n)),   d_eff(K) = sum_t c_t
// (every column of U^(n) has unit norm).  So l^lam(K) / d_eff(K) is a mixture
// over the components t, with weights c_t / d_eff, of the product
// distributions prod_n (u^(n)_{. t_n})^2: a draw picks t, then one row index
// per mode from column t_n of U^(n).  Drawing this way is this library's
// design; the paper draws from the classical product (Alg. 3).
//
// Tables (tucker_ridge_tables): U^(n) comes from the eigendecomposition of
// A^(n)T A^(n) = V diag(ev) V^T (the leverage kernels' Jacobi), u_{i t} =
// (a_i . v_t) / sqrt(ev_t), with the eigenpairs sorted by decreasing ev (the
// SVD's order) and K_n = min(I_n, R_n) components per mode; a squared singular
// value at or below max(I_n, R_n) 2^-52 times the largest counts as zero (the
// pseudo-inverse rule of the leverage scores), and its column is written as 0.
//
// Sampler arithmetic (the product sampler's, extended): fixed-point weights
// q = floor(clamp(x, 0, 1) 2^32) of c_t (component CDF, row-major over t) and
// of each column of squares (one CDF per (n, t_n)); a draw t takes the
// component from word 0 of Philox stream 3 and the row index of mode n from
// word n % 4 of stream n / 4, each by min{i : C_i > floor(u Q / 2^64)}.  The
// probability of a drawn row is
//     p = sum_t (q^c_t / Q^c) prod_n (q^(n,t_n)_{i_n} / Q^(n,t_n)),
// summed over t in row-major order and multiplied in mode order, each ratio
// one FP64 division (the CPU oracle's order, so p is bit-identical).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace tk {

constexpr int RG_THREADS = 256;

// ---------------------------------------------------------------- tables
struct RidgeTabArgs {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  int R[TUCKER_MAX_ORDER];
  int K[TUCKER_MAX_ORDER];                 // components: min(I_n, R_n)
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  const double* evecs[TUCKER_MAX_ORDER];   // R x R, evecs[a * R + k] = component a of vector k
  const double* evals[TUCKER_MAX_ORDER];   // R
  int* perm;                               // [N][TUCKER_MAX_RANK]: k-th largest eigenpair
  double* s2;                              // [N][TUCKER_MAX_RANK]: sorted, cut squared values
  double* usq[TUCKER_MAX_ORDER];           // K_n x I_n (column t contiguous)
  double* c;                               // prod K_n, row-major over t
  double* d_eff;                           // 1
  double lambda;
  int dK;                                  // prod K_n
};

// One warp per mode: rank the eigenvalues (decreasing, ties by index) and cut.
__global__ void k_ridge_sort(RidgeTabArgs a) {
  const int n = blockIdx.x, lane = threadIdx.x;
  const int R = a.R[n];
  const double* ev = a.evals[n];
  double top = 0.0;
  for (int k = 0; k < R; ++k) top = fmax(top, ev[k]);
  const double tol = double(a.I[n] > R ? a.I[n] : R) * 2.220446049250313e-16 * top;
  for (int k = lane; k < R; k += 32) {
    const double e = ev[k];
    int rank = 0;
    for (int j = 0; j < R; ++j) rank += ev[j] > e || (ev[j] == e && j < k);
    a.perm[n * TUCKER_MAX_RANK + rank] = k;
    if (rank < a.K[n]) a.s2[n * TUCKER_MAX_RANK + rank] = e > tol ? e : 0.0;
  }
}

__device__ __forceinline__ double fac_at(const void* A, int is64, int64_t i, int R, int r) {
  return is64 ? static_cast<const double*>(A)[i * R + r]
              : (double)static_cast<const float*>(A)[i * R + r];
}

// usq[n][k][i] = (a_i . v_{perm k})^2 / s2_k for the K_n leading components.
__global__ void k_ridge_usq(RidgeTabArgs a) {
  const int n = blockIdx.y;
  const int R = a.R[n], K = a.K[n];
  const int64_t I = a.I[n];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < K; ++k) {
      const double s2 = a.s2[n * TUCKER_MAX_RANK + k];
      double v = 0.0;
      if (s2 > 0.0) {
        const int t = a.perm[n * TUCKER_MAX_RANK + k];
        double dot = 0.0;
        for (int r = 0; r < R; ++r)
          dot = fma(fac_at(a.A[n], a.is64, i, R, r), a.evecs[n][r * R + t], dot);
        v = dot * dot / s2;
      }
      a.usq[n][(size_t)k * I + i] = v;
    }
  }
}

// c_t = P_t / (P_t + lam), P_t = ((1 s2_1[t_1]) s2_2[t_2]) ..., and d_eff = sum c_t.
__global__ void __launch_bounds__(RG_THREADS) k_ridge_c(RidgeTabArgs a) {
  __shared__ double part[RG_THREADS / 32];
  double acc = 0.0;
  for (int t = threadIdx.x; t < a.dK; t += RG_THREADS) {
    int rem = t, tn[TUCKER_MAX_ORDER];
    for (int n = a.N - 1; n >= 0; --n) { tn[n] = rem % a.K[n]; rem /= a.K[n]; }
    double P = 1.0;
    for (int n = 0; n < a.N; ++n) P = __dmul_rn(P, a.s2[n * TUCKER_MAX_RANK + tn[n]]);
    const double c = P > 0.0 ? P / (P + a.lambda) : 0.0;
    a.c[t] = c;
    acc += c;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < RG_THREADS / 32; ++k) s += part[k];
    *a.d_eff = s;
  }
}

// ---------------------------------------------------------------- sampler
__device__ __forceinline__ uint64_t fixed_q(double x) {
  return (uint64_t)__double2ull_rz(fmin(fmax(x, 0.0), 1.0) * 4294967296.0);
}

// Inclusive prefix sums of fixed-point weights: blockIdx.x < sum_n K_n are
// the columns (mode-major), the last CTA is the component CDF.
__global__ void __launch_bounds__(RG_THREADS) k_ridge_cdfs(RidgeSampArgs a) {
  __shared__ int64_t scan_tmp[32];
  int col = blockIdx.x, n = 0;
  const double* src;
  uint64_t* dst;
  int64_t len;
  while (n < a.N && col >= a.K[n]) { col -= a.K[n]; ++n; }
  if (n < a.N) {
    len = a.I[n];
    src = a.usq[n] + (size_t)col * len;
    dst = a.colcdf[n] + (size_t)col * len;
  } else {
    len = a.dK;
    src = a.c;
    dst = a.ccdf;
  }
  uint64_t carry = 0;
  for (int64_t base = 0; base < len; base += RG_THREADS) {
    const int64_t i = base + threadIdx.x;
    const uint64_t q = i < len ? fixed_q(src[i]) : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan((int64_t)q, scan_tmp, &tot);
    if (i < len) dst[i] = carry + (uint64_t)ex + q;
    carry += (uint64_t)tot;
  }
  if (threadIdx.x == 0 && n == a.N && carry == 0) set_status(a.status, DEV_RANK);
}

// The ratio tables of the probabilities: rc[t] = q^c_t / Q^c, and
// rrow[n][i][t] = q^(n,t)_i / Q^(n,t) (FP64 divisions of the integers).
__global__ void k_ridge_ratios(RidgeSampArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const double Qc = (double)a.ccdf[a.dK - 1];
  for (int64_t t = g; t < a.dK; t += stride) {
    const uint64_t q = a.ccdf[t] - (t ? a.ccdf[t - 1] : 0);
    a.rc[t] = (double)q / Qc;
  }
  for (int n = 0; n < a.N; ++n) {
    const int64_t I = a.I[n];
    const int K = a.K[n];
    for (int64_t e = g; e < I * K; e += stride) {
      const int64_t i = e / K;
      const int t = (int)(e - i * K);
      const uint64_t* C = a.colcdf[n] + (size_t)t * I;
      const uint64_t Q = C[I - 1];
      const uint64_t q = C[i] - (i ? C[i - 1] : 0);
      a.rrow[n][e] = Q ? (double)q / (double)Q : 0.0;
    }
  }
}

__global__ void k_ridge_draw(RidgeSampArgs a) {
  const uint64_t Qc = a.ccdf[a.dK - 1];
  if (a.T_out && blockIdx.x == 0 && threadIdx.x == 0) *a.T_out = a.m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const U64x4 w3 = philox4x64_10((uint64_t)t, 3, 0, 0, a.seed, a.sweep);
    int comp = upper_bound_u64(a.ccdf, a.dK, __umul64hi(w3.v[0], Qc));
    int tn[TUCKER_MAX_ORDER];
    for (int n = a.N - 1; n >= 0; --n) { tn[n] = comp % a.K[n]; comp /= a.K[n]; }
    uint64_t key = 0;
    U64x4 w = philox4x64_10((uint64_t)t, 0, 0, 0, a.seed, a.sweep);
    for (int n = 0; n < a.N; ++n) {
      if (n == 4) w = philox4x64_10((uint64_t)t, 1, 0, 0, a.seed, a.sweep);
      const int In = (int)a.I[n];
      const uint64_t* C = a.colcdf[n] + (size_t)tn[n] * In;
      const int i = upper_bound_u64(C, In, __umul64hi(w.v[n & 3], C[In - 1]));
      key = key * (uint64_t)In + (uint64_t)i;
    }
    a.keys_out[t] = key;
  }
}

// p of each distinct row: the sum over components in row-major order.
__global__ void k_ridge_prob(RidgeSampArgs a) {
  const int nu = *a.n_unique;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
    uint64_t key = a.keys_u[u];
    int64_t idx[TUCKER_MAX_ORDER];
    for (int n = a.N - 1; n >= 0; --n) {
      idx[n] = (int64_t)(key % (uint64_t)a.I[n]);
      key /= (uint64_t)a.I[n];
    }
    const double* row[TUCKER_MAX_ORDER];
    for (int n = 0; n < a.N; ++n) row[n] = a.rrow[n] + (size_t)idx[n] * a.K[n];
    int tn[TUCKER_MAX_ORDER] = {};
    double p = 0.0;
    for (int t = 0; t < a.dK; ++t) {
      const double r0 = a.rc[t];
      if (r0 != 0.0) {                                // rounded products and sum, never fused
        double f = r0;
        for (int n = 0; n < a.N; ++n) f = __dmul_rn(f, row[n][tn[n]]);
        p = __dadd_rn(p, f);
      }
      for (int n = a.N - 1; n >= 0; --n) {             // row-major odometer over t
        if (++tn[n] < a.K[n]) break;
        tn[n] = 0;
      }
    }
    a.prob[u] = p;
  }
}

// ---------------------------------------------------------------- launchers
tucker_status launch_leverage(tucker_handle* h, const FactorSet& F, double* const* lev,
                              uint64_t* const* cdf, int* d_rank, double* const* evecs,
                              double* const* evals, double* const* gram_out);
size_t leverage_aux_bytes(int64_t maxI);

int ridge_components(const FactorSet& F, int* K) {
  int dK = 1;
  for (int n = 0; n < F.N; ++n) {
    K[n] = (int)(F.I[n] < F.R[n] ? F.I[n] : F.R[n]);
    dK *= K[n];
  }
  return dK;
}

// Device bytes of ridge_tables' scratch (beyond its outputs).
size_t ridge_tables_scratch(const FactorSet& F) {
  int64_t maxI = 1, sumI = 0;
  for (int n = 0; n < F.N; ++n) {
    if (F.I[n] > maxI) maxI = F.I[n];
    sumI += F.I[n];
  }
  return (size_t)(sumI + 2 * TUCKER_MAX_ORDER * (TUCKER_MAX_RANK * TUCKER_MAX_RANK + TUCKER_MAX_RANK)) *
             sizeof(double) +
         sumI * sizeof(uint64_t) + leverage_aux_bytes(maxI) +
         2 * TUCKER_MAX_ORDER * TUCKER_MAX_RANK * 8 + 4096;
}

// usq[n] (K_n x I_n), c (prod K_n) and d_eff (device double) of the factors.
tucker_status ridge_tables(tucker_handle* h, const FactorSet& F, double lambda, char* scratch,
                           double* const* usq, double* c, double* d_eff,
                           double* const* V_out = nullptr, double* const* ev_out = nullptr) {
  Arena ar(scratch);
  double* lev[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  double* V[TUCKER_MAX_ORDER];
  double* ev[TUCKER_MAX_ORDER];
  int64_t maxI = 1;
  for (int n = 0; n < F.N; ++n) {
    lev[n] = ar.get<double>(F.I[n]);
    cdf[n] = ar.get<uint64_t>(F.I[n]);
    V[n] = V_out ? V_out[n] : ar.get<double>((size_t)F.R[n] * F.R[n]);
    ev[n] = ev_out ? ev_out[n] : ar.get<double>(F.R[n]);
    if (F.I[n] > maxI) maxI = F.I[n];
  }
  int* rk = reinterpret_cast<int*>(ar.get<char>(leverage_aux_bytes(maxI)));
  RidgeTabArgs a;
  memset(&a, 0, sizeof(a));
  a.perm = reinterpret_cast<int*>(ar.get<char>(TUCKER_MAX_ORDER * TUCKER_MAX_RANK * sizeof(int)));
  a.s2 = ar.get<double>(TUCKER_MAX_ORDER * TUCKER_MAX_RANK);
  TK_TRY(launch_leverage(h, F, lev, cdf, rk, V, ev, nullptr));
  a.N = F.N;
  a.is64 = F.is64;
  a.lambda = lambda;
  a.d_eff = d_eff;
  a.c = c;
  a.dK = ridge_components(F, a.K);
  int64_t maxI2 = 1;
  for (int n = 0; n < F.N; ++n) {
    a.I[n] = F.I[n];
    a.R[n] = F.R[n];
    a.A[n] = F.A[n];
    a.evecs[n] = V[n];
    a.evals[n] = ev[n];
    a.usq[n] = usq[n];
    if (F.I[n] > maxI2) maxI2 = F.I[n];
  }
  TK_COUNT(h);
  k_ridge_sort<<<F.N, 32, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  int gx = (int)((maxI2 + 255) / 256);
  if (gx > 64) gx = 64;
  TK_COUNT(h);
  k_ridge_usq<<<dim3(gx, F.N), 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_ridge_c<<<1, RG_THREADS, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// Device bytes of the sampler's scratch for m draws (tables, CDFs, raw keys).
size_t ridge_sample_scratch(const FactorSet& F, int64_t m) {
  int K[TUCKER_MAX_ORDER];
  const int dK = ridge_components(F, K);
  size_t b = (size_t)dK * 16 + (size_t)m * 8 + 4096;
  for (int n = 0; n < F.N; ++n) b += (size_t)F.I[n] * K[n] * 16 + 512;
  return b;
}

// m draws into keys_raw (T = m); the CDF and ratio tables are carved from scratch.
tucker_status ridge_draw(tucker_handle* h, const FactorSet& F, const double* const* usq,
                         const double* c, int64_t m, uint64_t seed, uint32_t sweep,
                         char* scratch, uint64_t* keys_raw, int64_t* d_T, RidgeState* st) {
  Arena ar(scratch);
  RidgeSampArgs& a = st->a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  a.dK = ridge_components(F, a.K);
  int ncols = 0;
  for (int n = 0; n < F.N; ++n) {
    a.I[n] = F.I[n];
    a.usq[n] = usq[n];
    a.colcdf[n] = ar.get<uint64_t>((size_t)F.I[n] * a.K[n]);
    a.rrow[n] = ar.get<double>((size_t)F.I[n] * a.K[n]);
    ncols += a.K[n];
  }
  a.c = c;
  a.ccdf = ar.get<uint64_t>(a.dK);
  a.rc = ar.get<double>(a.dK);
  a.seed = seed;
  a.sweep = sweep;
  a.m = m;
  a.keys_out = keys_raw;
  a.T_out = d_T;
  a.status = h->d_status;
  TK_COUNT(h);
  k_ridge_cdfs<<<ncols + 1, RG_THREADS, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_ridge_ratios<<<h->num_sms, 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  int gx = (int)std::min<int64_t>((m + 255) / 256, (int64_t)h->num_sms * 8);
  if (gx < 1) gx = 1;
  TK_COUNT(h);
  k_ridge_draw<<<gx, 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// Probabilities of the n_unique (device count) sorted distinct keys.
tucker_status ridge_prob(tucker_handle* h, RidgeState* st, const uint64_t* keys_u,
                         const int* n_unique, int64_t cap, double* prob) {
  RidgeSampArgs a = st->a;
  a.keys_u = keys_u;
  a.n_unique = n_unique;
  a.prob = prob;
  int gx = (int)std::min<int64_t>((cap + 127) / 128, (int64_t)h->num_sms * 16);
  if (gx < 1) gx = 1;
  TK_COUNT(h);
  k_ridge_prob<<<gx, 128, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
