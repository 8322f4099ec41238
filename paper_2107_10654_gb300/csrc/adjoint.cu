// Adjoint of the sketched solve with the sample held fixed.
//
// Forward: M = sum_u w_u k_u k_u^T + diag(regdiag), h = sum_u w_u x_u k_u, g = M^-1 h.
// For a cotangent gbar and v = M^-1 gbar (a transposed solve with the same
// Cholesky factor, M being symmetric):
//     dx_u          = w_u (k_u . v)
//     dk_u          = w_u ((x_u - k_u . g) v - (k_u . v) g)
//     dA^(n)[i_n,:] += contraction of dk_u with the other factor rows:
//                      dA^(n)[i_n, r_n] += sum_{r : r_n} dk_u[r] prod_{m != n} A^(m)[i_m, r_m]
// One warp per sampled row. dk_u = alpha_u v - beta_u g is never formed: the
// first contraction of each chain reads v and g (L1-resident) with two
// accumulators. Mode 1 contracts modes 2..N in turn; the other modes share
// T1 = dk_u x_1 a_1 and contract the remaining modes outermost first, so every
// step is a warp-wide TTV on a small per-warp shared-memory tensor. FP64
// atomics add the R_n row contributions into dA^(n).
#include "common.cuh"

namespace tk {

struct AdjArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  int d;
  int S;                  // ping-pong buffer length, d / min(R_1, R_2)
  int per_warp;           // doubles of shared memory per warp
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

// out[o * inner + j] = sum_t in[(o * Dm + t) * inner + j] a[t]: a mode-m
// product with a vector on a row-major tensor viewed as (outer, Dm, inner).
__device__ __forceinline__ void warp_ttv(const double* in, double* out, int outer, int Dm,
                                         int inner, const double* a, int lane) {
  const int n = outer * inner;
  for (int q = lane; q < n; q += 32) {
    const int o = q / inner, j = q - o * inner;
    const double* p = in + (int64_t)o * Dm * inner + j;
    double s = 0.0;
    for (int t = 0; t < Dm; ++t) s = fma(p[(int64_t)t * inner], a[t], s);
    out[q] = s;
  }
  __syncwarp();
}

// The same product applied to dk = al v - be g, read from global memory.
__device__ __forceinline__ void warp_ttv_vg(const double* __restrict__ v,
                                            const double* __restrict__ g, double al, double be,
                                            double* out, int outer, int Dm, int inner,
                                            const double* a, int lane) {
  const int n = outer * inner;
  for (int q = lane; q < n; q += 32) {
    const int o = q / inner, j = q - o * inner;
    const int64_t b = (int64_t)o * Dm * inner + j;
    double sv = 0.0, sg = 0.0;
    for (int t = 0; t < Dm; ++t) {
      const double at = a[t];
      sv = fma(__ldg(v + b + (int64_t)t * inner), at, sv);
      sg = fma(__ldg(g + b + (int64_t)t * inner), at, sg);
    }
    out[q] = fma(al, sv, -be * sg);
  }
  __syncwarp();
}

__global__ void __launch_bounds__(256) k_adjoint_rows(AdjArgs a) {
  extern __shared__ double sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  int off[TUCKER_MAX_ORDER], sumR = 0;
  for (int n = 0; n < a.N; ++n) { off[n] = sumR; sumR += a.R[n]; }
  double* rows = sm + (int64_t)wib * a.per_warp;   // sumR factor values of this sample
  double* T1 = rows + sumR;                         // d / R_1
  double* P = T1 + a.d / a.R[0];                    // S
  double* Q = P + a.S;                              // S
  const int nrows = *a.n_rows;
  const int wpb = blockDim.x >> 5;
  for (int u = blockIdx.x * wpb + wib; u < nrows; u += gridDim.x * wpb) {
    uint32_t iu[TUCKER_MAX_ORDER];
    for (int n = 0; n < a.N; ++n) iu[n] = a.idx[n][u];
    for (int q = lane; q < sumR; q += 32) {
      int n = 0;
      while (n + 1 < a.N && q >= off[n + 1]) ++n;
      rows[q] = load_as_double(a.A[n], (int64_t)iu[n] * a.R[n] + (q - off[n]), a.is64);
    }
    const double w = a.w[u], al = w * (a.x[u] - a.zg[u]), be = w * a.zv[u];
    if (lane == 0) a.dx[u] = be;
    __syncwarp();
    if (a.N == 1) {
      for (int r = lane; r < a.R[0]; r += 32)
        atomicAdd(&a.dA[0][(int64_t)iu[0] * a.R[0] + r], fma(al, a.v[r], -be * a.g[r]));
      continue;
    }
    // mode 1: contract modes 2..N of dk, r_1 kept outermost
    int inner = a.d / (a.R[0] * a.R[1]);
    warp_ttv_vg(a.v, a.g, al, be, P, a.R[0], a.R[1], inner, rows + off[1], lane);
    double* cur = P;
    double* nxt = Q;
    for (int m = 2; m < a.N; ++m) {
      inner /= a.R[m];
      warp_ttv(cur, nxt, a.R[0], a.R[m], inner, rows + off[m], lane);
      double* t = cur; cur = nxt; nxt = t;
    }
    for (int r = lane; r < a.R[0]; r += 32)
      atomicAdd(&a.dA[0][(int64_t)iu[0] * a.R[0] + r], cur[r]);
    __syncwarp();
    // T1 = dk x_1 a_1, shared by modes 2..N
    warp_ttv_vg(a.v, a.g, al, be, T1, 1, a.R[0], a.d / a.R[0], rows, lane);
    for (int n = 1; n < a.N; ++n) {
      cur = T1;
      int nb = 0;
      int in1 = a.d / a.R[0];
      for (int m = 1; m < n; ++m) {            // modes before n: each is outermost
        in1 /= a.R[m];
        nxt = nb ? Q : P;
        warp_ttv(cur, nxt, 1, a.R[m], in1, rows + off[m], lane);
        cur = nxt; nb ^= 1;
      }
      int in2 = in1 / a.R[n];                  // prod_{k > n} R_k
      for (int m = n + 1; m < a.N; ++m) {      // modes after n, r_n kept outermost
        in2 /= a.R[m];
        nxt = nb ? Q : P;
        warp_ttv(cur, nxt, a.R[n], a.R[m], in2, rows + off[m], lane);
        cur = nxt; nb ^= 1;
      }
      for (int r = lane; r < a.R[n]; r += 32)
        atomicAdd(&a.dA[n][(int64_t)iu[n] * a.R[n] + r], cur[r]);
      __syncwarp();
    }
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
  int sumR = 0;
  for (int n = 0; n < F.N; ++n) {
    a.R[n] = F.R[n]; a.A[n] = F.A[n]; a.idx[n] = idx[n]; a.dA[n] = dA[n];
    sumR += F.R[n];
    TK_COUNT(h);
    k_zero<<<64, 256, 0, h->stream>>>(dA[n], F.I[n] * F.R[n]);
  }
  a.w = w; a.x = x; a.zg = zg; a.zv = zv; a.g = g; a.v = v; a.n_rows = n_rows; a.dx = dx;
  const int rmin = F.N > 1 ? (F.R[0] < F.R[1] ? F.R[0] : F.R[1]) : F.R[0];
  a.S = (int)(F.d / rmin);
  a.per_warp = sumR + (int)(F.d / F.R[0]) + 2 * a.S;
  a.per_warp = (a.per_warp + 1) & ~1;                        // 16-byte aligned warp slices
  const size_t warp_bytes = sizeof(double) * (size_t)a.per_warp;
  const size_t smem_max = 220 * 1024;
  int wpb = (int)(smem_max / warp_bytes);
  if (wpb > 8) wpb = 8;
  if (wpb < 1) return fail(h, TUCKER_EINVAL, "adjoint: %zu B of shared memory per warp",
                           warp_bytes);
  const size_t smem = warp_bytes * wpb;
  if (smem > 48 * 1024)
    TK_CUDA(h, cudaFuncSetAttribute(k_adjoint_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int64_t blocks = (cap + wpb - 1) / wpb;
  const int64_t bmax = (int64_t)h->num_sms * (wpb == 8 ? 8 : 2048 / (32 * wpb));
  if (blocks > bmax) blocks = bmax;
  if (blocks < 1) blocks = 1;
  TK_COUNT(h);
  k_adjoint_rows<<<(int)blocks, 32 * wpb, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
