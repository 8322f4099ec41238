// CUDA-core (SIMT) kernels over the implicit Kronecker rows of the sample.
//
// A row of the design matrix is never stored: k_u[r] = prod_n A^(n)[i_n(u), r_n]
// with r = (r_1..r_N) row-major (the data structure that queries entries of
// K from the factors, Alg. 3 line 2).  Kernels:
//   k_syrk_simt<T>   G = sum_u w_u k_u k_u^T, 64x64 output tiles of the upper
//                    triangle, samples split across CTAs, FP64 or FP32 FMA;
//   k_tile_reduce    sums the per-split tiles in a fixed order into a
//                    symmetric FP64 G (deterministic);
//   k_kron_axpy      out = sum_u c_u k_u with c_u = s * a_u * b_u (FP64):
//                    h = sum w x k (normal-equation right-hand side), or the
//                    implicit FP64 product (sum w k k^T) g of the refinement;
//   k_kron_dot       z_u = k_u . g (and k_u . v) for every row (FP64).
// These are the FP64/FP32 paths and the FP64 residual of the tensor-core path.
#include "common.cuh"

namespace tk {

RowSet make_rowset(const FactorSet& F, uint32_t* const* idx, const double* w, const int* n_rows) {
  RowSet s;
  memset(&s, 0, sizeof(s));
  s.N = F.N;
  s.is64 = F.is64;
  s.d = F.d;
  int st = 1;
  for (int n = F.N - 1; n >= 0; --n) { s.stride[n] = st; st *= F.R[n]; }
  for (int n = 0; n < F.N; ++n) { s.R[n] = F.R[n]; s.A[n] = F.A[n]; s.idx[n] = idx[n]; }
  s.w = w;
  s.n_rows = n_rows;
  return s;
}

__device__ __forceinline__ double kron_entry(const RowSet& s, int u, int c) {
  double v = 1.0;
  for (int n = 0; n < s.N; ++n) {
    const int cn = (c / s.stride[n]) % s.R[n];
    v *= load_as_double(s.A[n], (int64_t)s.idx[n][u] * s.R[n] + cn, s.is64);
  }
  return v;
}

constexpr int ST = 64;       // tile edge
constexpr int SKC = 16;      // samples per smem chunk

__device__ __forceinline__ void decode_upper_tile(int p, int Tt, int* ti, int* tj) {
  int i = 0, rem = p;
  while (rem >= Tt - i) { rem -= Tt - i; ++i; }
  *ti = i;
  *tj = i + rem;
}

template <class T>
__global__ void __launch_bounds__(256) k_syrk_simt(RowSet s, T* partial, int nsplit) {
  __shared__ T Ka[SKC][ST + 1];
  __shared__ T Kb[SKC][ST + 1];
  const int Tt = (s.d + ST - 1) / ST;
  int ti, tj;
  decode_upper_tile(blockIdx.x, Tt, &ti, &tj);
  const int nrows = *s.n_rows;
  const int chunk = (nrows + nsplit - 1) / nsplit;
  const int s0 = blockIdx.y * chunk;
  const int s1 = min(nrows, s0 + chunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int base = s0; base < s1; base += SKC) {
    for (int e = threadIdx.x; e < 2 * SKC * ST; e += blockDim.x) {
      const int which = e / (SKC * ST);
      const int rem = e % (SKC * ST);
      const int sl = rem / ST, r = rem % ST;
      const int u = base + sl;
      const int c = (which ? tj : ti) * ST + r;
      T v = T(0);
      if (u < s1 && c < s.d) v = T((s.w ? sqrt(s.w[u]) : 1.0) * kron_entry(s, u, c));
      if (which) Kb[sl][r] = v; else Ka[sl][r] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < SKC; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) { a[i] = Ka[k][ty * 4 + i]; b[i] = Kb[k][tx * 4 + i]; }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* out = partial + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * ST * ST;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) out[(ty * 4 + i) * ST + tx * 4 + j] = acc[i][j];
}

// G[r][c] = G[c][r] = sum_split partial[split][tile][r - ti*64][c - tj*64]
template <class T>
__global__ void k_tile_reduce(const T* partial, int nsplit, int ntiles, int d, double* G) {
  const int Tt = (d + ST - 1) / ST;
  int ti, tj;
  decode_upper_tile(blockIdx.x, Tt, &ti, &tj);
  for (int e = threadIdx.x; e < ST * ST; e += blockDim.x) {
    const int r = ti * ST + e / ST, c = tj * ST + e % ST;
    if (r >= d || c >= d) continue;
    double v = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) v += (double)partial[((size_t)sp * ntiles + blockIdx.x) * ST * ST + e];
    G[(size_t)r * d + c] = v;
    G[(size_t)c * d + r] = v;
  }
}

constexpr int AXPY_SAMPLES = 32;

// partial[split][r] = sum_{u in split} coef * a[u] * b[u] * k_u[r]
__global__ void __launch_bounds__(256) k_kron_axpy(RowSet s, const double* a, const double* b,
                                                   double coef, double* partial, int nsplit) {
  extern __shared__ double rows[];        // AXPY_SAMPLES x sumR, then AXPY_SAMPLES coefs
  int off[TUCKER_MAX_ORDER], sumR = 0;
  for (int n = 0; n < s.N; ++n) { off[n] = sumR; sumR += s.R[n]; }
  double* cu = rows + AXPY_SAMPLES * sumR;
  const int nrows = *s.n_rows;
  const int chunk = (nrows + nsplit - 1) / nsplit;
  const int s0 = blockIdx.y * chunk, s1 = min(nrows, s0 + chunk);
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  int rn[TUCKER_MAX_ORDER];
  for (int n = 0; n < s.N; ++n) rn[n] = off[n] + (r / s.stride[n]) % s.R[n];
  double acc = 0.0;
  for (int base = s0; base < s1; base += AXPY_SAMPLES) {
    const int ns = min(AXPY_SAMPLES, s1 - base);
    for (int e = threadIdx.x; e < ns * sumR; e += blockDim.x) {
      const int sl = e / sumR, q = e % sumR;
      int n = 0;
      while (n + 1 < s.N && q >= off[n + 1]) ++n;
      const int u = base + sl;
      rows[sl * sumR + q] = load_as_double(s.A[n], (int64_t)s.idx[n][u] * s.R[n] + (q - off[n]), s.is64);
    }
    for (int e = threadIdx.x; e < ns; e += blockDim.x) {
      const int u = base + e;
      cu[e] = coef * a[u] * (b ? b[u] : 1.0);
    }
    __syncthreads();
    if (r < s.d) {
      for (int sl = 0; sl < ns; ++sl) {
        double k = rows[sl * sumR + rn[0]];
        for (int n = 1; n < s.N; ++n) k *= rows[sl * sumR + rn[n]];
        acc = fma(cu[sl], k, acc);
      }
    }
    __syncthreads();
  }
  if (r < s.d) partial[(size_t)blockIdx.y * s.d + r] = acc;
}

// out[r] = (base ? base[r] : 0) - (diag ? diag[r] * y[r] : 0) + sum_split partial[split][r]
__global__ void k_vec_reduce(const double* partial, int nsplit, int d, const double* base,
                             const double* diag, const double* y, double* out) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < d; r += gridDim.x * blockDim.x) {
    double v = base ? base[r] : 0.0;
    if (diag) v -= diag[r] * y[r];
    for (int sp = 0; sp < nsplit; ++sp) v += partial[(size_t)sp * d + r];
    out[r] = v;
  }
}

// z1[u] = k_u . g1, z2[u] = k_u . g2 (g2 nullable), one warp per row.
__global__ void __launch_bounds__(256) k_kron_dot(RowSet s, const double* g1, const double* g2,
                                                  double* z1, double* z2) {
  extern __shared__ double gs[];
  for (int r = threadIdx.x; r < s.d; r += blockDim.x) {
    gs[r] = g1[r];
    if (g2) gs[s.d + r] = g2[r];
  }
  __syncthreads();
  const int nrows = *s.n_rows;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = warp; u < nrows; u += nwarps) {
    double a1 = 0.0, a2 = 0.0;
    for (int r = lane; r < s.d; r += 32) {
      const double k = kron_entry(s, u, r);
      a1 = fma(k, gs[r], a1);
      if (g2) a2 = fma(k, gs[s.d + r], a2);
    }
    a1 = warp_sum(a1);
    if (g2) a2 = warp_sum(a2);
    if (lane == 0) { z1[u] = a1; if (z2) z2[u] = a2; }
  }
}

// --------------------------------------------------------------- host side

int gram_simt_splits(tucker_handle* h, int d, int64_t cap) {
  const int Tt = (d + ST - 1) / ST;
  const int tiles = Tt * (Tt + 1) / 2;
  int want = (4 * h->num_sms + tiles - 1) / tiles;
  int maxs = (int)((cap + 255) / 256);
  if (want > maxs) want = maxs;
  if (want < 1) want = 1;
  return want;
}

size_t gram_simt_partial_bytes(int d, int nsplit, int is64) {
  const int Tt = (d + ST - 1) / ST;
  return (size_t)nsplit * Tt * (Tt + 1) / 2 * ST * ST * (is64 ? 8 : 4);
}

tucker_status launch_gram_simt(tucker_handle* h, const RowSet& s, int use64, int nsplit,
                               void* partial, double* G) {
  const int Tt = (s.d + ST - 1) / ST;
  const int tiles = Tt * (Tt + 1) / 2;
  dim3 grid(tiles, nsplit);
  if (h->timing) cudaEventRecord(h->ev[10], h->stream);
  if (use64) {
    TK_COUNT(h);
    k_syrk_simt<double><<<grid, 256, 0, h->stream>>>(s, (double*)partial, nsplit);
    TK_LAUNCH(h);
    if (h->timing) cudaEventRecord(h->ev[11], h->stream);
    TK_COUNT(h);
    k_tile_reduce<double><<<tiles, 256, 0, h->stream>>>((double*)partial, nsplit, tiles, s.d, G);
  } else {
    TK_COUNT(h);
    k_syrk_simt<float><<<grid, 256, 0, h->stream>>>(s, (float*)partial, nsplit);
    TK_LAUNCH(h);
    if (h->timing) cudaEventRecord(h->ev[11], h->stream);
    TK_COUNT(h);
    k_tile_reduce<float><<<tiles, 256, 0, h->stream>>>((float*)partial, nsplit, tiles, s.d, G);
  }
  TK_LAUNCH(h);
  return TUCKER_OK;
}

int axpy_splits(tucker_handle* h, int d, int64_t cap) {
  const int rb = (d + 255) / 256;
  int want = (4 * h->num_sms + rb - 1) / rb;
  int maxs = (int)((cap + AXPY_SAMPLES - 1) / AXPY_SAMPLES);
  if (want > maxs) want = maxs;
  if (want < 1) want = 1;
  return want;
}

// out = base - diag.*y + coef * sum_u a_u b_u k_u   (partial: nsplit x d doubles)
tucker_status launch_kron_axpy(tucker_handle* h, const RowSet& s, const double* a,
                               const double* b, double coef, int nsplit, double* partial,
                               const double* base, const double* diag, const double* y,
                               double* out) {
  int sumR = 0;
  for (int n = 0; n < s.N; ++n) sumR += s.R[n];
  size_t smem = (size_t)AXPY_SAMPLES * (sumR + 1) * sizeof(double);
  dim3 grid((s.d + 255) / 256, nsplit);
  TK_COUNT(h);
  k_kron_axpy<<<grid, 256, smem, h->stream>>>(s, a, b, coef, partial, nsplit);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_vec_reduce<<<(s.d + 255) / 256, 256, 0, h->stream>>>(partial, nsplit, s.d, base, diag, y, out);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

tucker_status launch_kron_dot(tucker_handle* h, const RowSet& s, const double* g1,
                              const double* g2, double* z1, double* z2) {
  size_t smem = (size_t)s.d * (g2 ? 2 : 1) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_kron_dot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_COUNT(h);
  k_kron_dot<<<h->num_sms * 4, 256, smem, h->stream>>>(s, g1, g2, z1, z2);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
