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
#include <algorithm>

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
  double* gpart[TUCKER_MAX_ORDER];    // [nchunk][R(R+1)/2] partial Grams
  int nchunk;
  int rows_per;                       // factor rows per partial Gram
  double* W[TUCKER_MAX_ORDER];        // R x R outputs of k_leverage_eig
};

// Partial Gram of rows [chunk * rows_per, ...) of every mode (grid: chunk x mode).
// Row tile staged in shared memory as FP64; thread -> (pair, row phase), then
// a fixed-order reduction over the phases.
// Rows per partial Gram: small factors are cut finer so that more CTAs share them.
static int gram_rows_per(int64_t maxI) { return maxI <= 8192 ? 64 : 256; }
__global__ void __launch_bounds__(256) k_gram_partial(LevArgs a) {
  extern __shared__ double st[];                      // rows_per x R, then 256 partials
  const int n = blockIdx.y, ch = blockIdx.x;
  const int R = a.F.R[n];
  const int64_t I = a.F.I[n];
  const int RP = a.rows_per;
  const int64_t i0 = (int64_t)ch * RP;
  const int npairs = R * (R + 1) / 2;
  double* red = st + RP * R;
  const int rows = (int)(i0 < I ? ((I - i0) < RP ? (I - i0) : RP) : 0);
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x)
    st[e] = load_as_double(a.F.A[n], i0 * R + e, a.F.is64);
  __syncthreads();
  const int phases = npairs >= 256 ? 1 : 256 / npairs;
  for (int base = 0; base < npairs; base += 256 / phases) {
    const int pidx = base + threadIdx.x / phases, ph = threadIdx.x % phases;
    double v = 0.0;
    if (pidx < npairs && threadIdx.x / phases < 256 / phases) {
      int r = 0, rem = pidx;
      while (rem >= R - r) { rem -= R - r; ++r; }
      const int c = r + rem;
      for (int i = ph; i < rows; i += phases) v = fma(st[i * R + r], st[i * R + c], v);
    }
    red[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 256 / phases) {
      const int pi = base + threadIdx.x;
      if (pi < npairs) {
        double sum = 0.0;
        for (int q = 0; q < phases; ++q) sum += red[threadIdx.x * phases + q];
        a.gpart[n][(size_t)ch * npairs + pi] = sum;
      }
    }
    __syncthreads();
  }
}

constexpr int LEV_THREADS = 256;

// Cyclic Jacobi eigendecomposition of the symmetric Rp x Rp matrix G (Rp even)
// in shared memory by one warp, with the round-robin (tournament) ordering so
// that Rp/2 disjoint rotations run in parallel per step; at most 40 sweeps.
// V must hold the identity on entry.  On return G is diagonal to FP64 rounding
// (eigenvalue k in G[k][k]) and V[i][k] is component i of eigenvector k.
// cs, sn, pp, qq: Rp/2 entries each of shared scratch.
__device__ void jacobi_eig_warp(double* G, double* V, int Rp, double* cs, double* sn, int* pp,
                                int* qq, int lane) {
  const int half = Rp / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int e = lane; e < Rp * Rp; e += 32) {
      const double v = G[e] * G[e];
      if (e / Rp == e % Rp) dia += v; else off += v;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (off <= 1e-28 * dia || Rp <= 1) break;
    for (int step = 0; step < Rp - 1; ++step) {
      for (int k = lane; k < half; k += 32) {
        // circle method: slot 0 fixed, slots 1..Rp-1 rotate by `step`
        const int s1 = Rp - 1 - k;
        int p = k == 0 ? 0 : ((k - 1 + step) % (Rp - 1)) + 1;
        int q = ((s1 - 1 + step) % (Rp - 1)) + 1;
        if (p > q) { const int t = p; p = q; q = t; }
        const double apq = G[p * Rp + q], app = G[p * Rp + p], aqq = G[q * Rp + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-16 * fabs(app + aqq) && fabs(apq) > 1e-300) {
          // tangent of the rotation angle in FP32 (an approximate annihilation
          // is enough for Jacobi); (c, s) formed in FP64 so that the
          // rotation is orthogonal to FP64 rounding
          const double num = aqq - app, den = 2.0 * apq;
          const bool in32 = fabs(den) > 1e-30 && fabs(den) < 1e30 && fabs(num) < 1e30;
          const float theta = in32 ? (float)num / (float)den : (float)(num / den);
          float tf;
          if (fabsf(theta) > 1e18f) tf = 0.5f / theta;
          else tf = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
          const double t = (double)tf;
          const double q2 = fma(t, t, 1.0);
          const double y = rsqrt(q2);
          c = y;
          s = t * y;
        }
        cs[k] = c; sn[k] = s; pp[k] = p; qq[k] = q;
      }
      __syncwarp();
      for (int e = lane; e < half * Rp; e += 32) {      // rows p, q
        const int k = e / Rp, j = e % Rp;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double gp = G[p * Rp + j], gq = G[q * Rp + j];
        G[p * Rp + j] = c * gp - s * gq;
        G[q * Rp + j] = s * gp + c * gq;
      }
      __syncwarp();
      for (int e = lane; e < half * Rp; e += 32) {      // columns p, q (and V)
        const int k = e / Rp, i = e % Rp;
        const int p = pp[k], q = qq[k];
        const double c = cs[k], s = sn[k];
        const double gp = G[i * Rp + p], gq = G[i * Rp + q];
        G[i * Rp + p] = c * gp - s * gq;
        G[i * Rp + q] = s * gp + c * gq;
        const double vp = V[i * Rp + p], vq = V[i * Rp + q];
        V[i * Rp + p] = c * vp - s * vq;
        V[i * Rp + q] = s * vp + c * vq;
      }
      __syncwarp();
    }
  }
}

// Per mode: Gram (all warps), Jacobi eigendecomposition (warp 0, warp-
// synchronous), and W = V diag(ev^-1/2) with the columns of eigenvalues
// <= tol zeroed, so that l_i = || a_i W ||^2 = a_i G^+ a_i^T.
// The body of k_leverage_eig for mode n, given the chunk partial Grams
// gparts[ch * npairs + pidx] (global or shared memory); sm: the eigensolver's
// scratch (2 Rp^2 + Rp doubles and Rp + 2 ints).  Every thread of the CTA calls
// it; warp 0 does the factorisation.  W goes to a.W[n] (global).
__device__ void lev_factor_W(const LevArgs& a, int n, const double* gparts, double* sm) {
  double* const* Wout = a.W;
  const int R = a.F.R[n];
  const int Rp = R + (R & 1);                 // even size for the tournament
  const int64_t I = a.F.I[n];
  double* G = sm;                             // Rp x Rp
  double* V = G + Rp * Rp;                    // Rp x Rp
  double* cs = V + Rp * Rp;                   // Rp/2 cos
  double* sn = cs + Rp / 2;                   // Rp/2 sin
  int* pp = reinterpret_cast<int*>(sn + Rp / 2);
  int* qq = pp + Rp / 2;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;

  for (int e = tid; e < Rp * Rp; e += blockDim.x) {
    G[e] = 0.0;
    V[e] = (e / Rp == e % Rp) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Gram = sum of the per-chunk partial Grams (fixed order)
  (void)nw; (void)wid;
  const int npairs = R * (R + 1) / 2;
  for (int pidx = tid; pidx < npairs; pidx += blockDim.x) {
    int r = 0, rem = pidx;
    while (rem >= R - r) { rem -= R - r; ++r; }
    const int c = r + rem;
    double v = 0.0;
    for (int ch = 0; ch < a.nchunk; ++ch) v += gparts[(size_t)ch * npairs + pidx];
    G[r * Rp + c] = v;
    G[c * Rp + r] = v;
  }
  (void)I;
  __syncthreads();
  if (a.gram[n])
    for (int e = tid; e < R * R; e += blockDim.x) a.gram[n][e] = G[(e / R) * Rp + e % R];
  // Fast path when only the scores are wanted: G = L L^T and W = L^-T (so that
  // || a_i W ||^2 = a_i G^-1 a_i^T), taken only if it certifies full rank under
  // the pseudo-inverse tolerance: 1 / ||L^-1||_F^2 <= lambda_min, and
  // lambda_max <= trace(G), so lambda_min > max(I, R) eps trace(G) implies that
  // no eigenvalue is dropped.  Otherwise the Jacobi eigendecomposition below.
  if (wid == 0 && !a.evecs[n] && !a.evals[n] && R <= 32) {
    double tr = 0.0;
    for (int i = lane; i < R; i += 32) tr += G[i * Rp + i];
    tr = warp_sum(tr);
    bool ok = true;
    for (int j = 0; j < R && ok; ++j) {                  // lane i owns row i (i < R <= 32)
      const double p = G[j * Rp + j];
      ok = p > 0.0 && p <= 1.7976931348623157e308;
      if (!ok) break;
      const double y = rsqrt(p);
      if (lane > j && lane < R) G[lane * Rp + j] *= y;
      __syncwarp();
      if (lane == j) G[j * Rp + j] = p * y;
      if (lane > j && lane < R) {
        const double lij = G[lane * Rp + j];
        for (int c = j + 1; c <= lane; ++c) G[lane * Rp + c] = fma(-lij, G[c * Rp + j], G[lane * Rp + c]);
      }
      __syncwarp();
    }
    ok = __all_sync(0xffffffffu, ok);
    if (ok) {
      // column c = lane of L^-1 by forward substitution (V holds L^-1)
      double fro = 0.0;
      if (lane < R) {
        for (int i = 0; i < R; ++i) {
          double v = (i == lane) ? 1.0 : 0.0;
          for (int jj = lane; jj < i; ++jj) v = fma(-G[i * Rp + jj], V[jj * Rp + lane], v);
          v = i < lane ? 0.0 : v / G[i * Rp + i];
          V[i * Rp + lane] = v;
          fro = fma(v, v, fro);
        }
      }
      fro = warp_sum(fro);
      const double tol = double(I > R ? I : R) * 2.220446049250313e-16 * tr;
      ok = fro > 0.0 && 1.0 / fro > tol;
      if (ok) {
        for (int e = lane; e < R * R; e += 32) {
          const int r = e / R, k = e % R;
          Wout[n][e] = V[k * Rp + r];                  // W = L^-T
        }
        if (lane == 0) a.rank[n] = R;
      }
    }
    if (ok) return;                                    // warp 0 only; the other warps are done
    // restore G from the partial Grams and V = I for the eigendecomposition
    for (int pidx = lane; pidx < npairs; pidx += 32) {
      int r = 0, rem = pidx;
      while (rem >= R - r) { rem -= R - r; ++r; }
      const int c = r + rem;
      double v = 0.0;
      for (int ch = 0; ch < a.nchunk; ++ch) v += gparts[(size_t)ch * npairs + pidx];
      G[r * Rp + c] = v;
      G[c * Rp + r] = v;
    }
    for (int e = lane; e < Rp * Rp; e += 32) V[e] = (e / Rp == e % Rp) ? 1.0 : 0.0;
    __syncwarp();
  }
  if (wid == 0) {
    jacobi_eig_warp(G, V, Rp, cs, sn, pp, qq, lane);
    // eigenvalues, tolerance, rank, W
    double emax = 0.0;
    for (int k = 0; k < R; ++k) emax = fmax(emax, G[k * Rp + k]);
    const double tol = double(I > R ? I : R) * 2.220446049250313e-16 * emax;
    int rk = 0;
    for (int k = 0; k < R; ++k) rk += G[k * Rp + k] > tol;
    if (lane == 0) a.rank[n] = rk;
    for (int e = lane; e < R * R; e += 32) {
      const int r = e / R, k = e % R;
      const double ev = G[k * Rp + k];
      Wout[n][e] = ev > tol ? V[r * Rp + k] / sqrt(ev) : 0.0;
      if (a.evecs[n]) a.evecs[n][e] = V[r * Rp + k];
    }
    if (a.evals[n])
      for (int k = lane; k < R; k += 32) a.evals[n][k] = G[k * Rp + k];
  }
}


__global__ void __launch_bounds__(LEV_THREADS) k_leverage_eig(LevArgs a) {
  pdl_wait();
  extern __shared__ double sm[];
  lev_factor_W(a, blockIdx.x, a.gpart[blockIdx.x], sm);
}

// l_i = || a_i W ||^2 for every row of every mode (grid y = mode).
struct LevRowArgs {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  int R[TUCKER_MAX_ORDER];
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  const double* W[TUCKER_MAX_ORDER];
  double* lev[TUCKER_MAX_ORDER];
};

// FP64 runs at under two multiply-adds per clock per SM on this GPU, so the
// I_n R_n^2 multiply-adds are spread thinly: thread (row, k) forms (a_i W)_k,
// and the R_n partial squares of a row are added in order of k through shared
// memory (the same order as a single thread's loop over k).
__global__ void __launch_bounds__(256) k_leverage_rows(LevRowArgs a) {
  pdl_wait();
  extern __shared__ double Ws[];
  const int n = blockIdx.y;
  const int R = a.R[n];
  double* pk = Ws + R * R;                                     // [rows per pass][R]
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Ws[e] = a.W[n][e];
  __syncthreads();
  const int rpp = blockDim.x / R;                              // rows per pass
  const int rl = threadIdx.x / R, k = threadIdx.x - rl * R;
  for (int64_t i0 = (int64_t)blockIdx.x * rpp; i0 < a.I[n]; i0 += (int64_t)gridDim.x * rpp) {
    const int64_t i = i0 + rl;
    if (rl < rpp && i < a.I[n]) {
      double p = 0.0;
      for (int r = 0; r < R; ++r) p = fma(load_as_double(a.A[n], i * R + r, a.is64), Ws[r * R + k], p);
      pk[rl * R + k] = p;
    }
    __syncthreads();
    if (threadIdx.x < rpp && i0 + threadIdx.x < a.I[n]) {
      double l = 0.0;
      for (int kk = 0; kk < R; ++kk) {
        const double p = pk[threadIdx.x * R + kk];
        l = fma(p, p, l);
      }
      a.lev[n][i0 + threadIdx.x] = l;
    }
    __syncthreads();
  }
}

tucker_status launch_cdf_from_lev(tucker_handle* h, int N, const int64_t* I,
                                  const double* const* lev, uint64_t* const* cdf,
                                  bool dep = false);

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
  pdl_wait();
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

// dep: the previous operation on the stream is this library's leverage kernel, so
// the launch may depend on it programmatically (otherwise it is launched in full
// order: the scores come from the caller, behind a memset of the status word)
tucker_status launch_cdf_from_lev(tucker_handle* h, int N, const int64_t* I,
                                  const double* const* lev, uint64_t* const* cdf, bool dep) {
  CdfArgs a;
  memset(&a, 0, sizeof(a));
  a.N = N;
  for (int n = 0; n < N; ++n) { a.I[n] = I[n]; a.lev[n] = lev[n]; a.cdf[n] = cdf[n]; }
  a.status = h->d_status;
  if (dep) {
    TK_CUDA(h, launch_dep(h, k_cdf_from_lev, N, LEV_THREADS, 0, a));
  } else {
    TK_COUNT(h);
    k_cdf_from_lev<<<N, LEV_THREADS, 0, h->stream>>>(a);
    TK_LAUNCH(h);
  }
  return TUCKER_OK;
}

tucker_status launch_leverage(tucker_handle* h, const FactorSet& F, double* const* lev,
                              uint64_t* const* cdf, int* d_rank, double* const* evecs,
                              double* const* evals, double* const* gram_out) {
  LevArgs a;
  memset(&a, 0, sizeof(a));
  a.F = F;
  int maxRp = 0, maxR = 0;
  int64_t maxI = 1;
  for (int n = 0; n < F.N; ++n) {
    a.lev[n] = lev[n];
    a.cdf[n] = cdf[n];
    a.evecs[n] = evecs ? evecs[n] : nullptr;
    a.evals[n] = evals ? evals[n] : nullptr;
    a.gram[n] = gram_out ? gram_out[n] : nullptr;
    const int Rp = F.R[n] + (F.R[n] & 1);
    if (Rp > maxRp) maxRp = Rp;
    if (F.R[n] > maxR) maxR = F.R[n];
    if (F.I[n] > maxI) maxI = F.I[n];
  }
  a.rank = d_rank;
  a.status = h->d_status;
  // W matrices live in the rank buffer's neighbourhood: use the handle's
  // small device scratch after the rank ints (d_rank is carved with room).
  double* Wbuf = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(d_rank + 2 * TUCKER_MAX_ORDER + 64) & ~uintptr_t(255));
  double* W[TUCKER_MAX_ORDER];
  LevRowArgs ra;
  memset(&ra, 0, sizeof(ra));
  ra.N = F.N;
  ra.is64 = F.is64;
  for (int n = 0; n < F.N; ++n) {
    W[n] = Wbuf + (size_t)n * TUCKER_MAX_RANK * TUCKER_MAX_RANK;
    ra.I[n] = F.I[n]; ra.R[n] = F.R[n]; ra.A[n] = F.A[n]; ra.W[n] = W[n]; ra.lev[n] = lev[n];
  }
  for (int n = 0; n < F.N; ++n) a.W[n] = W[n];             // by value: no host copy
  double** Wdev = reinterpret_cast<double**>(Wbuf + (size_t)TUCKER_MAX_ORDER * TUCKER_MAX_RANK * TUCKER_MAX_RANK);
  // partial Grams behind the W matrices
  double* gp = reinterpret_cast<double*>(Wdev + TUCKER_MAX_ORDER);
  a.rows_per = gram_rows_per(maxI);
  a.nchunk = (int)((maxI + a.rows_per - 1) / a.rows_per);
  for (int n = 0; n < F.N; ++n) {
    a.gpart[n] = gp;
    gp += (size_t)a.nchunk * (F.R[n] * (F.R[n] + 1) / 2);
  }
  const size_t gsm = (size_t)(a.rows_per * maxR + 256) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)gsm));
  TK_COUNT(h);
  k_gram_partial<<<dim3(a.nchunk, F.N), 256, gsm, h->stream>>>(a);
  TK_LAUNCH(h);
  const size_t smem = size_t(2 * maxRp * maxRp + maxRp) * sizeof(double) +
                      size_t(maxRp + 2) * sizeof(int) + 64;
  TK_CUDA(h, cudaFuncSetAttribute(k_leverage_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_CUDA(h, launch_dep(h, k_leverage_eig, F.N, LEV_THREADS, smem, a));
  const int rpp = maxR <= 256 ? 256 / maxR : 1;                 // rows per CTA pass
  int gx = (int)((maxI + rpp - 1) / rpp);
  if (gx > 4 * h->num_sms / F.N) gx = 4 * h->num_sms / F.N;
  if (gx < 1) gx = 1;
  TK_CUDA(h, launch_dep(h, k_leverage_rows, dim3(gx, F.N), 256,
                        (size_t)(maxR * maxR + 256) * sizeof(double), ra));
  return launch_cdf_from_lev(h, F.N, F.I, lev, cdf, true);
}

// gram[n] = A^(n)T A^(n) (full, row-major) from the chunk partials, summed in
// chunk order (the same order as the leverage kernels' Gram).
__global__ void k_gram_sum(LevArgs a) {
  const int n = blockIdx.x;
  const int R = a.F.R[n];
  const int npairs = R * (R + 1) / 2;
  for (int pidx = threadIdx.x; pidx < npairs; pidx += blockDim.x) {
    int r = 0, rem = pidx;
    while (rem >= R - r) { rem -= R - r; ++r; }
    const int c = r + rem;
    double v = 0.0;
    for (int ch = 0; ch < a.nchunk; ++ch) v += a.gpart[n][(size_t)ch * npairs + pidx];
    a.gram[n][r * R + c] = v;
    a.gram[n][c * R + r] = v;
  }
}

// The factor Grams alone (the ALS factor updates and the loss need no scores):
// two launches instead of the leverage pipeline's four.  d_rank: the scratch
// the leverage launcher uses (leverage_aux_bytes).
tucker_status launch_factor_grams(tucker_handle* h, const FactorSet& F, int* d_rank,
                                  double* const* gram) {
  LevArgs a;
  memset(&a, 0, sizeof(a));
  a.F = F;
  int maxR = 0;
  int64_t maxI = 1;
  for (int n = 0; n < F.N; ++n) {
    a.gram[n] = gram[n];
    if (F.R[n] > maxR) maxR = F.R[n];
    if (F.I[n] > maxI) maxI = F.I[n];
  }
  // the same carve as launch_leverage: W matrices, then the pointer table, then partials
  double* Wbuf = reinterpret_cast<double*>(reinterpret_cast<uintptr_t>(d_rank + 2 * TUCKER_MAX_ORDER + 64) & ~uintptr_t(255));
  double** Wdev = reinterpret_cast<double**>(Wbuf + (size_t)TUCKER_MAX_ORDER * TUCKER_MAX_RANK * TUCKER_MAX_RANK);
  double* gp = reinterpret_cast<double*>(Wdev + TUCKER_MAX_ORDER);
  a.rows_per = gram_rows_per(maxI);
  a.nchunk = (int)((maxI + a.rows_per - 1) / a.rows_per);
  for (int n = 0; n < F.N; ++n) {
    a.gpart[n] = gp;
    gp += (size_t)a.nchunk * (F.R[n] * (F.R[n] + 1) / 2);
  }
  const size_t gsm = (size_t)(a.rows_per * maxR + 256) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_gram_partial, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)gsm));
  TK_COUNT(h);
  k_gram_partial<<<dim3(a.nchunk, F.N), 256, gsm, h->stream>>>(a);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_gram_sum<<<F.N, 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// Device bytes the leverage launcher needs behind its rank pointer.
size_t leverage_aux_bytes(int64_t maxI) {
  const int rp = gram_rows_per(maxI);
  const size_t nchunk = (size_t)((maxI + rp - 1) / rp);
  return (2 * TUCKER_MAX_ORDER + 64) * sizeof(int) + 256 +
         (size_t)TUCKER_MAX_ORDER * TUCKER_MAX_RANK * TUCKER_MAX_RANK * sizeof(double) +
         TUCKER_MAX_ORDER * sizeof(double*) + 64 +
         nchunk * TUCKER_MAX_ORDER * (TUCKER_MAX_RANK * (TUCKER_MAX_RANK + 1) / 2) * sizeof(double);
}

// Eigendecompositions of given R_n x R_n Grams (one CTA per mode, warp 0
// works): the preconditioner of the CG ridge solver needs A^(n)T A^(n) =
// V_n diag(ev_n) V_n^T of every factor.  gram[n] is row-major FP64 (as written
// by the leverage launcher's gram output); evecs[n][r * R + k] = V_n[r][k],
// evals[n][k] = ev_n[k].
struct GramEigArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  const double* gram[TUCKER_MAX_ORDER];
  double* evecs[TUCKER_MAX_ORDER];
  double* evals[TUCKER_MAX_ORDER];
};

// FP32 cyclic Jacobi by one warp (the same tournament ordering as
// jacobi_eig_warp): the preconditioner is applied in FP32, so its V_n and ev_n
// need FP32 accuracy only, and on this GPU a dependent FP64 operation costs
// tens of cycles (the FP64 eigendecomposition of three 8 x 8 Grams took about
// 70 us, the FP32 one a few).  Stops when the off-diagonal mass is below
// 1e-12 of the diagonal's (off-diagonal entries about 1e-6 of the diagonal, the
// level FP32 rotations reach; a tighter test never passes and runs every
// sweep), at most 40 sweeps.
__device__ void jacobi_eig_warp_f32(float* G, float* V, int Rp, float* cs, float* sn, int* pp,
                                    int* qq, int lane) {
  const int half = Rp / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    float off = 0.f, dia = 0.f;
    for (int e = lane; e < Rp * Rp; e += 32) {
      const float v = G[e] * G[e];
      if (e / Rp == e % Rp) dia += v; else off += v;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if (!(off > 1e-12f * dia) || Rp <= 1) break;
    for (int step = 0; step < Rp - 1; ++step) {
      for (int k = lane; k < half; k += 32) {
        const int s1 = Rp - 1 - k;
        int p = k == 0 ? 0 : ((k - 1 + step) % (Rp - 1)) + 1;
        int q = ((s1 - 1 + step) % (Rp - 1)) + 1;
        if (p > q) { const int t = p; p = q; q = t; }
        const float apq = G[p * Rp + q], app = G[p * Rp + p], aqq = G[q * Rp + q];
        float c = 1.f, sv = 0.f;
        if (fabsf(apq) > 1e-8f * fabsf(app + aqq) && fabsf(apq) > 1e-30f) {
          const float theta = (aqq - app) / (2.f * apq);
          const float t = fabsf(theta) > 1e18f
                              ? 0.5f / theta
                              : copysignf(1.f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
          c = rsqrtf(fmaf(t, t, 1.f));
          sv = t * c;
        }
        cs[k] = c; sn[k] = sv; pp[k] = p; qq[k] = q;
      }
      __syncwarp();
      for (int e = lane; e < half * Rp; e += 32) {      // rows p, q
        const int k = e / Rp, j = e % Rp;
        const int p = pp[k], q = qq[k];
        const float c = cs[k], sv = sn[k];
        const float gp = G[p * Rp + j], gq = G[q * Rp + j];
        G[p * Rp + j] = c * gp - sv * gq;
        G[q * Rp + j] = sv * gp + c * gq;
      }
      __syncwarp();
      for (int e = lane; e < half * Rp; e += 32) {      // columns p, q (and V)
        const int k = e / Rp, i = e % Rp;
        const int p = pp[k], q = qq[k];
        const float c = cs[k], sv = sn[k];
        const float gp = G[i * Rp + p], gq = G[i * Rp + q];
        G[i * Rp + p] = c * gp - sv * gq;
        G[i * Rp + q] = sv * gp + c * gq;
        const float vp = V[i * Rp + p], vq = V[i * Rp + q];
        V[i * Rp + p] = c * vp - sv * vq;
        V[i * Rp + q] = sv * vp + c * vq;
      }
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(32) k_gram_eig(GramEigArgs a) {
  extern __shared__ float smf[];
  const int n = blockIdx.x;
  const int R = a.R[n];
  const int Rp = R + (R & 1);
  float* G = smf;
  float* V = G + Rp * Rp;
  float* cs = V + Rp * Rp;
  float* sn = cs + Rp / 2;
  int* pp = reinterpret_cast<int*>(sn + Rp / 2);
  int* qq = pp + Rp / 2;
  const int lane = threadIdx.x;
  for (int e = lane; e < Rp * Rp; e += 32) {
    const int r = e / Rp, c = e % Rp;
    G[e] = (r < R && c < R) ? (float)a.gram[n][r * R + c] : 0.f;
    V[e] = (r == c) ? 1.f : 0.f;
  }
  __syncwarp();
  jacobi_eig_warp_f32(G, V, Rp, cs, sn, pp, qq, lane);
  for (int e = lane; e < R * R; e += 32) {
    const int r = e / R, k = e % R;
    a.evecs[n][e] = (double)V[r * Rp + k];
  }
  for (int k = lane; k < R; k += 32) a.evals[n][k] = (double)G[k * Rp + k];
}

tucker_status launch_gram_eig(tucker_handle* h, int N, const int* R, const double* const* gram,
                              double* const* evecs, double* const* evals) {
  GramEigArgs a;
  memset(&a, 0, sizeof(a));
  a.N = N;
  int maxRp = 0;
  for (int n = 0; n < N; ++n) {
    a.R[n] = R[n];
    a.gram[n] = gram[n];
    a.evecs[n] = evecs[n];
    a.evals[n] = evals[n];
    const int Rp = R[n] + (R[n] & 1);
    if (Rp > maxRp) maxRp = Rp;
  }
  const size_t smem = size_t(2 * maxRp * maxRp + maxRp) * sizeof(float) +
                      size_t(maxRp + 2) * sizeof(int) + 64;
  TK_CUDA(h, cudaFuncSetAttribute(k_gram_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_COUNT(h);
  k_gram_eig<<<N, 32, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk

