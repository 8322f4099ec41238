// Factor update of regularised Tucker ALS (Alg. 2 inner loop) for dense X.
//
// Mode n, every row i of A^(n) solves  argmin_y ||y K_n - b_i||^2 + lambda ||y||^2
// with K_n = G_(n) W^T, W = (x)_{k != n} A^(k), b_i row i of X_(n).  In closed form
//     A^(n) = B G_(n)^T (G_(n) H G_(n)^T + lambda I)^-1,
// B = (X x_{k != n} A^(k)T)_(n) (computed by the n-mode product chain) and
// H = (x)_{k != n} A^(k)T A^(k), applied to the core mode by mode.
// k_factor_lhs (one CTA) forms the R_n x R_n system, factors it (Cholesky,
// FP64) and inverts it; k_factor_rows gives each warp rows of A^(n): it forms a
// row's right-hand side with its lanes over the core entries and applies the
// inverse.
#include "common.cuh"

namespace tk {

struct FactorSolveArgs {
  int N, n;
  int R[TUCKER_MAX_ORDER];
  const double* gram[TUCKER_MAX_ORDER];   // R_k x R_k Grams
  const double* core;                      // d
  const double* B;                         // (pre, I_n, post) FP64
  int64_t In;
  double lambda;
  void* A_out;                             // I_n x R_n, dtype
  int is64;
  int d;
  int* status;
};

constexpr int FS_THREADS = 256;
constexpr int FS_ROWS = 32;                  // rows per CTA of the row kernel: four per warp

// The R_n x R_n system of mode n, lhs = G_(n) H G_(n)^T + lambda I with
// H = (x)_{k != n} A^(k)T A^(k) applied to the core mode by mode, its Cholesky
// factor L (by warp 0 with lane i owning row i when R_n <= 32, else by thread
// 0) and the inverse L^-T L^-1 into Lout (row-major).  One CTA.
__global__ void __launch_bounds__(FS_THREADS) k_factor_lhs(FactorSolveArgs a, double* Lout) {
  extern __shared__ double sm[];
  const int d = a.d, Rn = a.R[a.n];
  double* c0 = sm;                 // core
  double* c1 = c0 + d;             // core x_{k != n} gram_k
  double* c2 = c1 + d;
  double* Lm = c2 + d;             // Rn x Rn
  for (int i = threadIdx.x; i < d; i += blockDim.x) c1[i] = c0[i] = a.core[i];
  __syncthreads();
  int pre = 1;
  for (int k = 0; k < a.N; ++k) {
    const int Rk = a.R[k];
    const int post = d / (pre * Rk);
    if (k != a.n) {
      for (int t = threadIdx.x; t < d; t += blockDim.x) {
        const int q = t % post, r = (t / post) % Rk, p = t / (post * Rk);
        double acc = 0.0;
        for (int j = 0; j < Rk; ++j) acc = fma(c1[(p * Rk + j) * post + q], a.gram[k][j * Rk + r], acc);
        c2[t] = acc;
      }
      __syncthreads();
      for (int t = threadIdx.x; t < d; t += blockDim.x) c1[t] = c2[t];
      __syncthreads();
    }
    pre *= Rk;
  }
  int preN = 1;
  for (int k = 0; k < a.n; ++k) preN *= a.R[k];
  const int postN = d / (preN * Rn);
  const int P = preN * postN;
  // lhs[x][y] = sum_P core[(p,x,q)] c1[(p,y,q)] + lambda delta, four threads per entry
  for (int e4 = threadIdx.x; e4 < 4 * Rn * Rn; e4 += blockDim.x) {
    const int e = e4 >> 2, part = e4 & 3;
    const int x = e / Rn, y = e % Rn;
    double acc = 0.0;
    for (int pq = part; pq < P; pq += 4) {
      const int p = pq / postN, q = pq % postN;
      acc = fma(c0[(p * Rn + x) * postN + q], c1[(p * Rn + y) * postN + q], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    if (part == 0) Lm[e] = acc + (x == y ? a.lambda : 0.0);
  }
  __syncthreads();
  if (Rn <= 32) {
    if (threadIdx.x < 32) {                          // lane i owns row i
      const int lane = threadIdx.x;
      for (int j = 0; j < Rn; ++j) {
        double piv = Lm[j * Rn + j];
        if (!(piv > 0.0)) { if (lane == 0) set_status(a.status, DEV_NOTSPD); piv = 1.0; }
        const double djj = sqrt(piv);
        __syncwarp();
        if (lane == j) Lm[j * Rn + j] = djj;
        if (lane > j && lane < Rn) Lm[lane * Rn + j] /= djj;
        __syncwarp();
        if (lane > j && lane < Rn) {
          const double lij = Lm[lane * Rn + j];
          for (int c = j + 1; c <= lane; ++c) Lm[lane * Rn + c] -= lij * Lm[c * Rn + j];
        }
        __syncwarp();
      }
    }
  } else if (threadIdx.x == 0) {
    for (int j = 0; j < Rn; ++j) {
      double v = Lm[j * Rn + j];
      for (int k = 0; k < j; ++k) v -= Lm[j * Rn + k] * Lm[j * Rn + k];
      if (!(v > 0.0)) { set_status(a.status, DEV_NOTSPD); v = 1.0; }
      const double djj = sqrt(v);
      Lm[j * Rn + j] = djj;
      for (int i = j + 1; i < Rn; ++i) {
        double w = Lm[i * Rn + j];
        for (int k = 0; k < j; ++k) w -= Lm[i * Rn + k] * Lm[j * Rn + k];
        Lm[i * Rn + j] = w / djj;
      }
    }
  }
  __syncthreads();
  // Minv = L^-T L^-1 (the inverse of the system), column j by thread j: the
  // rows then need R_n independent dot products instead of two dependent
  // triangular solves each
  for (int j = threadIdx.x; j < Rn; j += blockDim.x) {
    double z[TUCKER_MAX_RANK];
    for (int x = 0; x < Rn; ++x) {                   // L z = e_j
      double v = x == j ? 1.0 : 0.0;
      for (int k = 0; k < x; ++k) v -= Lm[x * Rn + k] * z[k];
      z[x] = v / Lm[x * Rn + x];
    }
    for (int x = Rn - 1; x >= 0; --x) {              // L^T w = z
      double v = z[x];
      for (int k = x + 1; k < Rn; ++k) v -= Lm[k * Rn + x] * z[k];
      z[x] = v / Lm[x * Rn + x];
    }
    for (int x = 0; x < Rn; ++x) Lout[x * Rn + j] = z[x];
  }
}

// Rows of the new A^(n): warp per row, rhs_x = sum_pq B[p][i][q] core[p][x][q]
// with the lanes over pq, then a = Minv rhs with the lanes over x.
__global__ void __launch_bounds__(FS_THREADS) k_factor_rows(FactorSolveArgs a, const double* Lg) {
  extern __shared__ double sm[];
  const int d = a.d, Rn = a.R[a.n];
  double* c0 = sm;
  double* Lm = c0 + d;
  for (int i = threadIdx.x; i < d; i += blockDim.x) c0[i] = a.core[i];
  for (int e = threadIdx.x; e < Rn * Rn; e += blockDim.x) Lm[e] = Lg[e];
  __syncthreads();
  int preN = 1;
  for (int k = 0; k < a.n; ++k) preN *= a.R[k];
  const int postN = d / (preN * Rn);
  const int P = preN * postN;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int rr = wid; rr < FS_ROWS; rr += FS_THREADS / 32) {
    const int64_t i = (int64_t)blockIdx.x * FS_ROWS + rr;
    if (i >= a.In) break;
    double y[TUCKER_MAX_RANK];
    for (int x = 0; x < Rn; ++x) y[x] = 0.0;
    for (int pq = lane; pq < P; pq += 32) {
      const int p = pq / postN, q = pq % postN;
      const double b = a.B[((int64_t)p * a.In + i) * postN + q];
      for (int x = 0; x < Rn; ++x) y[x] = fma(b, c0[(p * Rn + x) * postN + q], y[x]);
    }
    for (int x = 0; x < Rn; ++x) y[x] = warp_sum(y[x]);       // every lane holds the rhs
    for (int x = lane; x < Rn; x += 32) {           // a_x = sum_k Minv[x][k] rhs_k
      double v = 0.0;
      for (int k = 0; k < Rn; ++k) v = fma(Lm[x * Rn + k], y[k], v);
      if (a.is64) static_cast<double*>(a.A_out)[i * Rn + x] = v;
      else static_cast<float*>(a.A_out)[i * Rn + x] = (float)v;
    }
  }
}

tucker_status factor_solve(tucker_handle* h, const FactorSet& F, int n, double* const* gram,
                           const double* core, const double* B, double lambda, void* A_out,
                           double* Lscratch) {
  FactorSolveArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N; a.n = n;
  for (int k = 0; k < F.N; ++k) { a.R[k] = F.R[k]; a.gram[k] = gram[k]; }
  a.core = core; a.B = B; a.In = F.I[n]; a.lambda = lambda; a.A_out = A_out;
  a.is64 = F.is64; a.d = F.d; a.status = h->d_status;
  const size_t smem = (size_t)(3 * F.d + F.R[n] * F.R[n]) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_factor_lhs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_COUNT(h);
  k_factor_lhs<<<1, FS_THREADS, smem, h->stream>>>(a, Lscratch);
  TK_LAUNCH(h);
  const size_t smem2 = (size_t)(F.d + F.R[n] * F.R[n]) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_factor_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem2));
  TK_COUNT(h);
  k_factor_rows<<<ceil_div(F.I[n], FS_ROWS), FS_THREADS, smem2, h->stream>>>(a, Lscratch);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
