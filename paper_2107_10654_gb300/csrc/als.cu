// Factor update of regularised Tucker ALS (Alg. 2 inner loop) for dense X.
//
// Mode n, every row i of A^(n) solves  argmin_y ||y K_n - b_i||^2 + lambda ||y||^2
// with K_n = G_(n) W^T, W = (x)_{k != n} A^(k), b_i row i of X_(n).  In closed form
//     A^(n) = B G_(n)^T (G_(n) H G_(n)^T + lambda I)^-1,
// B = (X x_{k != n} A^(k)T)_(n) (computed by the n-mode product chain) and
// H = (x)_{k != n} A^(k)T A^(k), applied to the core mode by mode.
// One CTA per block of rows: it forms the R_n x R_n system in shared memory,
// factors it (Cholesky, FP64) and solves one right-hand side per row.
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

constexpr int FS_ROWS = 128;

__global__ void __launch_bounds__(FS_ROWS) k_factor_solve(FactorSolveArgs a) {
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
  // lhs[x][y] = sum_P core[(p,x,q)] c1[(p,y,q)] + lambda delta
  for (int e = threadIdx.x; e < Rn * Rn; e += blockDim.x) {
    const int x = e / Rn, y = e % Rn;
    double acc = 0.0;
    for (int pq = 0; pq < P; ++pq) {
      const int p = pq / postN, q = pq % postN;
      acc = fma(c0[(p * Rn + x) * postN + q], c1[(p * Rn + y) * postN + q], acc);
    }
    Lm[e] = acc + (x == y ? a.lambda : 0.0);
  }
  __syncthreads();
  if (threadIdx.x == 0) {                // Cholesky of the small SPD system
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
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.In) return;
  double y[TUCKER_MAX_RANK];
  for (int x = 0; x < Rn; ++x) {
    double acc = 0.0;
    for (int pq = 0; pq < P; ++pq) {
      const int p = pq / postN, q = pq % postN;
      acc = fma(a.B[((int64_t)p * a.In + i) * postN + q], c0[(p * Rn + x) * postN + q], acc);
    }
    y[x] = acc;
  }
  for (int x = 0; x < Rn; ++x) {            // L z = rhs
    double v = y[x];
    for (int k = 0; k < x; ++k) v -= Lm[x * Rn + k] * y[k];
    y[x] = v / Lm[x * Rn + x];
  }
  for (int x = Rn - 1; x >= 0; --x) {       // L^T a = z
    double v = y[x];
    for (int k = x + 1; k < Rn; ++k) v -= Lm[k * Rn + x] * y[k];
    y[x] = v / Lm[x * Rn + x];
  }
  for (int x = 0; x < Rn; ++x) {
    if (a.is64) static_cast<double*>(a.A_out)[i * Rn + x] = y[x];
    else static_cast<float*>(a.A_out)[i * Rn + x] = (float)y[x];
  }
}

tucker_status factor_solve(tucker_handle* h, const FactorSet& F, int n, double* const* gram,
                           const double* core, const double* B, double lambda, void* A_out) {
  FactorSolveArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N; a.n = n;
  for (int k = 0; k < F.N; ++k) { a.R[k] = F.R[k]; a.gram[k] = gram[k]; }
  a.core = core; a.B = B; a.In = F.I[n]; a.lambda = lambda; a.A_out = A_out;
  a.is64 = F.is64; a.d = F.d; a.status = h->d_status;
  const size_t smem = (size_t)(3 * F.d + F.R[n] * F.R[n]) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_factor_solve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_COUNT(h);
  k_factor_solve<<<ceil_div(F.I[n], FS_ROWS), FS_ROWS, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
