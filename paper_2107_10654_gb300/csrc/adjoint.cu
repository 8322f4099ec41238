// Adjoint of the sketched solve with the sample held fixed.
//
// Forward: M = sum_u w_u k_u k_u^T + diag(regdiag), h = sum_u w_u x_u k_u, g = M^-1 h.
// For a cotangent gbar and v = M^-1 gbar (a transposed solve with the same
// Cholesky factor, M being symmetric):
//     dx_u          = w_u (k_u . v)
//     dk_u          = w_u ((x_u - k_u . g) v - (k_u . v) g)
//     dA^(n)[i_n,:] += contraction of dk_u with the other factor rows:
//                      dA^(n)[i_n, r_n] += sum_{r : r_n} dk_u[r] prod_{m != n} A^(m)[i_m, r_m]
// One CTA per sampled row (grid-stride): dk_u is formed in shared memory,
// the N contractions accumulate in shared memory, then FP64 atomics add the
// row contributions into dA^(n).
#include "common.cuh"

namespace tk {

struct AdjArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  int stride[TUCKER_MAX_ORDER];
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  int d;
  const uint32_t* idx[TUCKER_MAX_ORDER];
  const double* w;
  const double* x;
  const double* zg;       // k_u . g
  const double* zv;       // k_u . v
  const double* g;
  const double* v;
  const int* n_rows;
  double* dA[TUCKER_MAX_ORDER];
  double* dx;
};

__global__ void __launch_bounds__(256) k_adjoint_rows(AdjArgs a) {
  extern __shared__ double sm[];
  int off[TUCKER_MAX_ORDER], sumR = 0;
  for (int n = 0; n < a.N; ++n) { off[n] = sumR; sumR += a.R[n]; }
  double* rows = sm;               // sumR factor values of this sample
  double* acc = rows + sumR;       // sumR accumulators
  const int nrows = *a.n_rows;
  for (int u = blockIdx.x; u < nrows; u += gridDim.x) {
    for (int q = threadIdx.x; q < sumR; q += blockDim.x) {
      int n = 0;
      while (n + 1 < a.N && q >= off[n + 1]) ++n;
      rows[q] = load_as_double(a.A[n], (int64_t)a.idx[n][u] * a.R[n] + (q - off[n]), a.is64);
      acc[q] = 0.0;
    }
    __syncthreads();
    const double w = a.w[u], cx = a.x[u] - a.zg[u], cv = a.zv[u];
    if (threadIdx.x == 0) a.dx[u] = w * cv;
    for (int r = threadIdx.x; r < a.d; r += blockDim.x) {
      const double dk = w * (cx * a.v[r] - cv * a.g[r]);
      int rn[TUCKER_MAX_ORDER];
      for (int n = 0; n < a.N; ++n) rn[n] = (r / a.stride[n]) % a.R[n];
      for (int n = 0; n < a.N; ++n) {
        double prod = dk;
        for (int m = 0; m < a.N; ++m)
          if (m != n) prod *= rows[off[m] + rn[m]];
        atomicAdd(&acc[off[n] + rn[n]], prod);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < sumR; q += blockDim.x) {
      int n = 0;
      while (n + 1 < a.N && q >= off[n + 1]) ++n;
      atomicAdd(&a.dA[n][(int64_t)a.idx[n][u] * a.R[n] + (q - off[n])], acc[q]);
    }
    __syncthreads();
  }
}

__global__ void k_zero(double* p, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) p[i] = 0.0;
}

tucker_status launch_adjoint_rows(tucker_handle* h, const FactorSet& F, uint32_t* const* idx,
                                  const double* w, const double* x, const double* zg,
                                  const double* zv, const double* g, const double* v,
                                  const int* n_rows, int64_t cap, double* const* dA, double* dx) {
  AdjArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N; a.is64 = F.is64; a.d = F.d;
  int st = 1, sumR = 0;
  for (int n = F.N - 1; n >= 0; --n) { a.stride[n] = st; st *= F.R[n]; }
  for (int n = 0; n < F.N; ++n) {
    a.R[n] = F.R[n]; a.A[n] = F.A[n]; a.idx[n] = idx[n]; a.dA[n] = dA[n];
    sumR += F.R[n];
    TK_COUNT(h);
    k_zero<<<64, 256, 0, h->stream>>>(dA[n], F.I[n] * F.R[n]);
  }
  a.w = w; a.x = x; a.zg = zg; a.zv = zv; a.g = g; a.v = v; a.n_rows = n_rows; a.dx = dx;
  int grid = (int)(cap < h->num_sms * 8 ? cap : h->num_sms * 8);
  if (grid < 1) grid = 1;
  TK_COUNT(h);
  k_adjoint_rows<<<grid, 256, 2 * sumR * sizeof(double), h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
