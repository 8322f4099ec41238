// Per-factor leverage scores (Alg. 3 line 1; Eq. ridge_leverage_score_def at
// lambda = 0) and the fixed-point CDF used by the product-distribution sampler.
//
// One CTA per mode n:
//   1. Gram G_n = A^(n)T A^(n) in FP64 (warp per Gram entry, lanes over rows);
//   2. cyclic Jacobi eigendecomposition G_n = V diag(ev) V^T with the
//      round-robin (tournament) ordering, so R/2 disjoint rotations run in
//      parallel per step; at most 40 sweeps;
//   3. l_i = sum_{k: ev_k > tol} (a_i . v_k)^2 / ev_k, tol = max(I,R) 2^-52 ev_max
//      (the pseudo-inverse of the Gram, eigenvalues below tol taken as zero);
//   4. q_i = floor(clamp(l_i,0,1) 2^32) and C = inclusive prefix sum (uint64).
#include "common.cuh"

namespace tk {

struct LevArgs {
  FactorSet F;
  double* lev[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  double* evecs[TUCKER_MAX_ORDER];   // nullable: R x R, V[a][k] row-major
  double* evals[TUCKER_MAX_ORDER];   // nullable: R
  double* gram[TUCKER_MAX_ORDER];    // nullable: R x R Gram before diagonalisation
  int* rank;                          // device int[N]
  int* status;
};

constexpr int LEV_THREADS = 256;

__global__ void __launch_bounds__(LEV_THREADS) k_leverage(LevArgs a) {
  extern __shared__ double sm[];
  const int n = blockIdx.x;
  const int R = a.F.R[n];
  const int Rp = R + (R & 1);                 // even size for the tournament
  const int64_t I = a.F.I[n];
  const void* A = a.F.A[n];
  const int is64 = a.F.is64;
  double* G = sm;                             // Rp x Rp
  double* V = G + Rp * Rp;                    // Rp x Rp
  double* cs = V + Rp * Rp;                   // Rp/2 cos
  double* sn = cs + Rp / 2;                   // Rp/2 sin
  int* pp = reinterpret_cast<int*>(sn + Rp / 2);
  int* qq = pp + Rp / 2;
  double* red = reinterpret_cast<double*>(qq + Rp / 2 + 2);  // 64 doubles
  __shared__ int64_t scan_tmp[32];
  __shared__ int s_done;

  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;

  // 1. Gram (upper triangle, mirrored), padded entries zero.
  for (int e = tid; e < Rp * Rp; e += blockDim.x) {
    G[e] = 0.0;
    V[e] = (e / Rp == e % Rp) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int npairs = R * (R + 1) / 2;
  for (int pidx = wid; pidx < npairs; pidx += nw) {
    // decode pidx -> (r, c) with r <= c
    int r = 0, rem = pidx;
    while (rem >= R - r) { rem -= R - r; ++r; }
    int c = r + rem;
    double s = 0.0;
    for (int64_t i = lane; i < I; i += 32)
      s += load_as_double(A, i * R + r, is64) * load_as_double(A, i * R + c, is64);
    s = warp_sum(s);
    if (lane == 0) { G[r * Rp + c] = s; G[c * Rp + r] = s; }
  }
  __syncthreads();
  if (a.gram[n])
    for (int e = tid; e < R * R; e += blockDim.x) a.gram[n][e] = G[(e / R) * Rp + e % R];

  // 2. Jacobi sweeps.
  const int half = Rp / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    // convergence test: off-diagonal mass vs diagonal mass
    double off = 0.0, dia = 0.0;
    for (int e = tid; e < Rp * Rp; e += blockDim.x) {
      double v = G[e] * G[e];
      if (e / Rp == e % Rp) dia += v; else off += v;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (lane == 0) { red[wid] = off; red[32 + wid] = dia; }
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, g = 0.0;
      for (int w = 0; w < nw; ++w) { o += red[w]; g += red[32 + w]; }
      s_done = (o <= 1e-30 * g) || Rp <= 1;
    }
    __syncthreads();
    if (s_done) break;
    for (int step = 0; step < Rp - 1; ++step) {
      if (tid < half) {
        // circle method: slot 0 fixed, slots 1..Rp-1 rotate by `step`
        int k = tid;
        int s0 = k, s1 = Rp - 1 - k;
        int p = s0 == 0 ? 0 : ((s0 - 1 + step) % (Rp - 1)) + 1;
        int q = ((s1 - 1 + step) % (Rp - 1)) + 1;
        if (p > q) { int t = p; p = q; q = t; }
        double apq = G[p * Rp + q], app = G[p * Rp + p], aqq = G[q * Rp + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0 && fabs(apq) > 1e-300) {
          double theta = (aqq - app) / (2.0 * apq);
          double t;
          if (fabs(theta) > 1e150) t = 0.5 / theta;
          else t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        cs[k] = c; sn[k] = s; pp[k] = p; qq[k] = q;
      }
      __syncthreads();
      for (int e = tid; e < half * Rp; e += blockDim.x) {      // rows p, q
        int k = e / Rp, j = e % Rp;
        int p = pp[k], q = qq[k];
        double c = cs[k], s = sn[k];
        double gp = G[p * Rp + j], gq = G[q * Rp + j];
        G[p * Rp + j] = c * gp - s * gq;
        G[q * Rp + j] = s * gp + c * gq;
      }
      __syncthreads();
      for (int e = tid; e < half * Rp; e += blockDim.x) {      // columns p, q (and V)
        int k = e / Rp, i = e % Rp;
        int p = pp[k], q = qq[k];
        double c = cs[k], s = sn[k];
        double gp = G[i * Rp + p], gq = G[i * Rp + q];
        G[i * Rp + p] = c * gp - s * gq;
        G[i * Rp + q] = s * gp + c * gq;
        double vp = V[i * Rp + p], vq = V[i * Rp + q];
        V[i * Rp + p] = c * vp - s * vq;
        V[i * Rp + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }

  // 3. eigenvalues, tolerance, rank
  if (tid == 0) {
    double emax = 0.0;
    for (int k = 0; k < R; ++k) emax = fmax(emax, G[k * Rp + k]);
    double tol = double(I > R ? I : R) * 2.220446049250313e-16 * emax;
    int rk = 0;
    for (int k = 0; k < R; ++k) rk += G[k * Rp + k] > tol;
    red[0] = tol;
    a.rank[n] = rk;
  }
  __syncthreads();
  const double tol = red[0];
  if (a.evecs[n])
    for (int e = tid; e < R * R; e += blockDim.x) a.evecs[n][e] = V[(e / R) * Rp + e % R];
  if (a.evals[n])
    for (int k = tid; k < R; k += blockDim.x) a.evals[n][k] = G[k * Rp + k];

  // 4. scores, fixed point, inclusive prefix sum in chunks of blockDim
  uint64_t carry = 0;
  for (int64_t base = 0; base < I; base += blockDim.x) {
    int64_t i = base + tid;
    uint64_t q = 0;
    if (i < I) {
      double l = 0.0;
      for (int k = 0; k < R; ++k) {
        double ev = G[k * Rp + k];
        if (!(ev > tol)) continue;
        double pr = 0.0;
        for (int r = 0; r < R; ++r) pr += load_as_double(A, i * R + r, is64) * V[r * Rp + k];
        l += pr * pr / ev;
      }
      a.lev[n][i] = l;
      double v = fmin(fmax(l, 0.0), 1.0) * 4294967296.0;
      q = (uint64_t)__double2ull_rz(v);
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan((int64_t)q, scan_tmp, &tot);
    if (i < I) a.cdf[n][i] = carry + (uint64_t)ex + q;
    carry += (uint64_t)tot;
  }
  if (tid == 0 && carry == 0) set_status(a.status, DEV_RANK);
}

// q_i = floor(clamp(l_i,0,1) 2^32) and inclusive prefix sums from given scores
// (the sampler's integer CDF), one CTA per mode.
struct CdfArgs {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  const double* lev[TUCKER_MAX_ORDER];
  uint64_t* cdf[TUCKER_MAX_ORDER];
  int* status;
};

__global__ void __launch_bounds__(LEV_THREADS) k_cdf_from_lev(CdfArgs a) {
  __shared__ int64_t scan_tmp[32];
  const int n = blockIdx.x;
  const int64_t I = a.I[n];
  uint64_t carry = 0;
  for (int64_t base = 0; base < I; base += blockDim.x) {
    const int64_t i = base + threadIdx.x;
    uint64_t q = 0;
    if (i < I) {
      double v = fmin(fmax(a.lev[n][i], 0.0), 1.0) * 4294967296.0;
      q = (uint64_t)__double2ull_rz(v);
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan((int64_t)q, scan_tmp, &tot);
    if (i < I) a.cdf[n][i] = carry + (uint64_t)ex + q;
    carry += (uint64_t)tot;
  }
  if (threadIdx.x == 0 && carry == 0) set_status(a.status, DEV_RANK);
}

tucker_status launch_cdf_from_lev(tucker_handle* h, int N, const int64_t* I,
                                  const double* const* lev, uint64_t* const* cdf) {
  CdfArgs a;
  memset(&a, 0, sizeof(a));
  a.N = N;
  for (int n = 0; n < N; ++n) { a.I[n] = I[n]; a.lev[n] = lev[n]; a.cdf[n] = cdf[n]; }
  a.status = h->d_status;
  TK_COUNT(h);
  k_cdf_from_lev<<<N, LEV_THREADS, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

tucker_status launch_leverage(tucker_handle* h, const FactorSet& F, double* const* lev,
                              uint64_t* const* cdf, int* d_rank, double* const* evecs,
                              double* const* evals, double* const* gram_out) {
  LevArgs a;
  memset(&a, 0, sizeof(a));
  a.F = F;
  int maxRp = 0;
  for (int n = 0; n < F.N; ++n) {
    a.lev[n] = lev[n];
    a.cdf[n] = cdf[n];
    a.evecs[n] = evecs ? evecs[n] : nullptr;
    a.evals[n] = evals ? evals[n] : nullptr;
    a.gram[n] = gram_out ? gram_out[n] : nullptr;
    int Rp = F.R[n] + (F.R[n] & 1);
    if (Rp > maxRp) maxRp = Rp;
  }
  a.rank = d_rank;
  a.status = h->d_status;
  size_t smem = size_t(2 * maxRp * maxRp + maxRp) * sizeof(double) +
                size_t(maxRp + 2) * sizeof(int) + 64 * sizeof(double) + 64;
  TK_CUDA(h, cudaFuncSetAttribute(k_leverage, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_COUNT(h);
  k_leverage<<<F.N, LEV_THREADS, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
