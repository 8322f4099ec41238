// Ridge solve of the (sketched or exact) normal equations (Eq. problem_def;
// Appendix B, proof of Thm 4.2): M = G + diag(regdiag), M = L L^T by a blocked
// right-looking FP64 Cholesky, then L y = h and L^T g = y.
//
// Cholesky step for panel k (width CB):
//   k_potrf_diag     factor the CB x CB diagonal block in shared memory; a
//                    non-positive or NaN pivot records TUCKER_ENOTSPD and all
//                    later kernels return immediately (no trap, no hang);
//   k_trsm_panel     rows below: A[i, k:k+CB] <- A[i, k:k+CB] L_kk^-T;
//   k_syrk_trailing  A[i, j] -= A[i, k:k+CB] . A[j, k:k+CB] on the lower trailing
//                    triangle, 64x64 tiles, FP64 FMA.
// L overwrites the lower triangle of M (row-major, d x d).
#include "common.cuh"

namespace tk {

constexpr int CB = 32;      // panel width
constexpr int CT = 64;      // trailing tile

__global__ void k_add_diag(double* M, int d, const double* diag) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
    M[(size_t)i * d + i] += diag[i];
}

__global__ void k_fill(double* v, int n, double val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = val;
}

// regdiag[j] = lambda (exact) or lambda * D[j] (augmented)
__global__ void k_regdiag(double* out, int d, double lambda, const double* D) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
    out[i] = D ? lambda * D[i] : lambda;
}

__global__ void __launch_bounds__(256) k_potrf_diag(double* M, int d, int k, int* status) {
  __shared__ double a[CB][CB + 1];
  __shared__ int bad;
  if (*status) return;
  const int nb = min(CB, d - k);
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    int i = e / CB, j = e % CB;
    a[i][j] = (i < nb && j < nb) ? M[(size_t)(k + i) * d + k + j] : 0.0;
  }
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (threadIdx.x == 0) {
      double p = a[j][j];
      if (!(p > 0.0)) { bad = 1; set_status(status, DEV_NOTSPD); }
      a[j][j] = sqrt(fmax(p, 0.0));
    }
    __syncthreads();
    if (bad) return;
    const double djj = a[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) a[i][j] /= djj;
    __syncthreads();
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      int i = e / nb, c = e % nb;
      if (c > j && i >= c) a[i][c] -= a[i][j] * a[c][j];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    int i = e / nb, j = e % nb;
    if (j <= i) M[(size_t)(k + i) * d + k + j] = a[i][j];
  }
}

__global__ void __launch_bounds__(128) k_trsm_panel(double* M, int d, int k, const int* status) {
  __shared__ double L[CB][CB + 1];
  if (*status) return;
  const int nb = min(CB, d - k);
  for (int e = threadIdx.x; e < CB * CB; e += blockDim.x) {
    int i = e / CB, j = e % CB;
    L[i][j] = (i < nb && j < nb && j <= i) ? M[(size_t)(k + i) * d + k + j] : 0.0;
  }
  __syncthreads();
  const int row = k + nb + blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d) return;
  double x[CB];
  double* mrow = M + (size_t)row * d + k;
#pragma unroll
  for (int c = 0; c < CB; ++c) x[c] = c < nb ? mrow[c] : 0.0;
#pragma unroll
  for (int c = 0; c < CB; ++c) {
    if (c >= nb) break;
    double v = x[c];
#pragma unroll
    for (int cc = 0; cc < CB; ++cc)
      if (cc < c) v -= x[cc] * L[c][cc];
    x[c] = v / L[c][c];
  }
#pragma unroll
  for (int c = 0; c < CB; ++c) if (c < nb) mrow[c] = x[c];
}

__global__ void __launch_bounds__(256) k_syrk_trailing(double* M, int d, int k, const int* status) {
  __shared__ double Pa[CT][CB + 1];
  __shared__ double Pb[CT][CB + 1];
  if (*status) return;
  const int s = k + CB;                       // trailing start
  const int Tt = (d - s + CT - 1) / CT;
  int ti = 0, rem = blockIdx.x;               // lower-triangle tile (ti >= tj)
  while (rem > ti) { rem -= ti + 1; ++ti; }
  const int tj = rem;
  if (ti >= Tt) return;
  const int r0 = s + ti * CT, c0 = s + tj * CT;
  for (int e = threadIdx.x; e < CT * CB; e += blockDim.x) {
    int i = e / CB, c = e % CB;
    Pa[i][c] = (r0 + i < d) ? M[(size_t)(r0 + i) * d + k + c] : 0.0;
    Pb[i][c] = (c0 + i < d) ? M[(size_t)(c0 + i) * d + k + c] : 0.0;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
#pragma unroll 8
  for (int c = 0; c < CB; ++c) {
    double a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) { a[i] = Pa[ty * 4 + i][c]; b[i] = Pb[tx * 4 + i][c]; }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = r0 + ty * 4 + i;
    if (r >= d) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < d && c <= r) M[(size_t)r * d + c] -= acc[i][j];
    }
  }
}

tucker_status cholesky(tucker_handle* h, double* M, int d) {
  for (int k = 0; k < d; k += CB) {
    TK_COUNT(h);
    k_potrf_diag<<<1, 256, 0, h->stream>>>(M, d, k, h->d_status);
    const int rows = d - k - CB;
    if (rows > 0) {
      TK_COUNT(h);
      k_trsm_panel<<<ceil_div(rows, 128), 128, 0, h->stream>>>(M, d, k, h->d_status);
      const int Tt = ceil_div(rows, CT);
      TK_COUNT(h);
      k_syrk_trailing<<<Tt * (Tt + 1) / 2, 256, 0, h->stream>>>(M, d, k, h->d_status);
    }
  }
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// ------------------------------------------------------------ triangular solves
// Blocked: per block of CB unknowns, one CTA solves the diagonal block and then
// a multi-CTA GEMV removes it from the remaining right-hand side.

__global__ void k_trsv_block(const double* L, int d, int k, double* b, int upper,
                             const int* status) {
  // solve the CB diagonal block in place (single warp, sequential over CB)
  __shared__ double x[CB];
  if (*status) return;
  const int nb = min(CB, d - k);
  if (threadIdx.x < nb) x[threadIdx.x] = b[k + threadIdx.x];
  __syncwarp();
  if (threadIdx.x == 0) {
    if (!upper) {
      for (int i = 0; i < nb; ++i) {
        double v = x[i];
        for (int j = 0; j < i; ++j) v -= L[(size_t)(k + i) * d + k + j] * x[j];
        x[i] = v / L[(size_t)(k + i) * d + k + i];
      }
    } else {                                  // L^T: row i of L^T is column i of L
      for (int i = nb - 1; i >= 0; --i) {
        double v = x[i];
        for (int j = i + 1; j < nb; ++j) v -= L[(size_t)(k + j) * d + k + i] * x[j];
        x[i] = v / L[(size_t)(k + i) * d + k + i];
      }
    }
  }
  __syncwarp();
  if (threadIdx.x < nb) b[k + threadIdx.x] = x[threadIdx.x];
}

// Lower: b[i] -= sum_{j in block} L[i][j] x[j] for i >= k + CB.
// Upper (L^T): b[i] -= sum_{j in block} L[j][i] x[j] for i < k.
__global__ void k_trsv_update(const double* L, int d, int k, double* b, int upper,
                              const int* status) {
  if (*status) return;
  const int nb = min(CB, d - k);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (!upper) {
    const int row = k + nb + i;
    if (row >= d) return;
    double v = 0.0;
    for (int j = 0; j < nb; ++j) v += L[(size_t)row * d + k + j] * b[k + j];
    b[row] -= v;
  } else {
    if (i >= k) return;
    double v = 0.0;
    for (int j = 0; j < nb; ++j) v += L[(size_t)(k + j) * d + i] * b[k + j];
    b[i] -= v;
  }
}

// g = (L L^T)^-1 rhs  (g may alias rhs)
tucker_status chol_solve(tucker_handle* h, const double* L, int d, const double* rhs, double* g) {
  if (g != rhs)
    TK_CUDA(h, cudaMemcpyAsync(g, rhs, sizeof(double) * d, cudaMemcpyDeviceToDevice, h->stream));
  for (int k = 0; k < d; k += CB) {
    TK_COUNT(h);
    k_trsv_block<<<1, 32, 0, h->stream>>>(L, d, k, g, 0, h->d_status);
    const int rows = d - k - CB;
    if (rows > 0) { TK_COUNT(h); k_trsv_update<<<ceil_div(rows, 128), 128, 0, h->stream>>>(L, d, k, g, 0, h->d_status); }
  }
  const int last = ((d - 1) / CB) * CB;
  for (int k = last; k >= 0; k -= CB) {
    TK_COUNT(h);
    k_trsv_block<<<1, 32, 0, h->stream>>>(L, d, k, g, 1, h->d_status);
    if (k > 0) { TK_COUNT(h); k_trsv_update<<<ceil_div(k, 128), 128, 0, h->stream>>>(L, d, k, g, 1, h->d_status); }
  }
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// g += r; out[0] = ||r||^2, out[1] = ||g||^2  (single CTA, fixed order)
__global__ void __launch_bounds__(1024) k_refine_update(double* g, const double* r, int d,
                                                        double* out) {
  __shared__ double red[2][32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    const double gi = g[i] + r[i];
    g[i] = gi;
    a = fma(r[i], r[i], a);
    b = fma(gi, gi, b);
  }
  a = warp_sum(a);
  b = warp_sum(b);
  if ((threadIdx.x & 31) == 0) { red[0][threadIdx.x >> 5] = a; red[1][threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s0 += red[0][w]; s1 += red[1][w]; }
    out[0] = s0;
    out[1] = s1;
  }
}

tucker_status launch_refine_update(tucker_handle* h, double* g, const double* r, int d,
                                   double* out2) {
  TK_COUNT(h);
  k_refine_update<<<1, 1024, 0, h->stream>>>(g, r, d, out2);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

tucker_status launch_regdiag(tucker_handle* h, double* out, int d, double lambda, const double* D) {
  TK_COUNT(h);
  k_regdiag<<<ceil_div(d, 256), 256, 0, h->stream>>>(out, d, lambda, D);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

tucker_status launch_add_diag(tucker_handle* h, double* M, int d, const double* diag) {
  TK_COUNT(h);
  k_add_diag<<<ceil_div(d, 256), 256, 0, h->stream>>>(M, d, diag);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
