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
#include <algorithm>

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

// Cholesky factor of the SPD R x R matrix Lm (shared memory, in place; lane i
// of warp 0 owns row i when R <= 32, else thread 0) and its inverse
// L^-T L^-1 into Lout (row-major).  Called by every thread of the CTA.
__device__ void spd_inverse(double* Lm, int Rn, double* Lout, int* status) {
  if (Rn <= 32) {
    if (threadIdx.x < 32) {                          // lane i owns row i
      const int lane = threadIdx.x;
      for (int j = 0; j < Rn; ++j) {
        double piv = Lm[j * Rn + j];
        if (!(piv > 0.0)) { if (lane == 0) set_status(status, DEV_NOTSPD); piv = 1.0; }
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
      if (!(v > 0.0)) { set_status(status, DEV_NOTSPD); v = 1.0; }
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
  spd_inverse(Lm, Rn, Lout, a.status);
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

// ------------------------------------------------ sketched factor update
// Mode n: rows u of the factor design B_n = W G_(n)^T (W = (x)_{k != n} A^(k),
// rows indexed row-major by the multi-index over the modes k != n) drawn from
// the product of those modes' leverage scores, deduplicated; with
// w_u = c_u / (m p_u), p_u = prod (q / Q) in mode order (the core sampler's
// arithmetic),
//     M = sum_u w_u b_u b_u^T + lambda I,   Y = sum_u w_u x_u b_u^T,   A^(n) = Y M^-1,
// b_u = G_(n) (x)_{k != n} A^(k)[j_k] and x_u the mode-n fiber of X at row u.
// The product of leverage scores is an (R_n / prod_{k != n} R_k)-overestimate
// of the leverage scores of B_n (its rows lie in the column space of W).
// The fibers and the sums Y are in X's element type T (FP32 values of X are
// exact in FP32); b_u, w_u b_u, M and its inverse are FP64.
struct FiberArgs {
  int N, n;                                // order; the updated mode
  int R[TUCKER_MAX_ORDER];
  int64_t I[TUCKER_MAX_ORDER];
  int64_t stride[TUCKER_MAX_ORDER];        // element strides of X (row-major)
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  const void* X;
  const double* core;
  int d;
  const uint64_t* keys;                    // distinct keys over the modes k != n
  const uint32_t* counts;
  const int* nu;
  const uint64_t* cdf[TUCKER_MAX_ORDER];   // indexed by mode k (k != n)
  int64_t m;                               // draws
  double lambda;
  int splits;                              // CTAs along the sample in the normal kernel
  int postn;                               // prod_{k > n} R_k
  FastDiv div_r[TUCKER_MAX_ORDER];         // by R_k
  FastDiv div_post;                        // by postn
  void* xs;                                // [cap][I_n] fibers
  double* wb;                              // [cap][R_n]  w_u b_u (FP64)
  double* bb;                              // [cap][R_n]  b_u (FP64)
  double* partY;                           // [splits][I_n][R_n]
  double* partM;                           // [splits][R_n][R_n]
  void* A_out;                             // I_n x R_n, X's dtype
  int* status;
  int cp;                                  // 1: CP design rows (Hadamard of the factor rows)
};

constexpr int FB_WARPS = 8;

// Warp per distinct row: decode, weight, design row b_u and the fiber.  For b_u
// the lanes walk the core index o over the modes k != n (o = (pre, post) around
// mode n, row-major), form w_o = prod_{k != n} a_k[r_k(o)] once (multiply-high
// divisions by R_k) and add G[pre, r, post] w_o into R_n accumulators (RB >= R_n,
// registers); R_n warp sums in a fixed order.  The fiber: lanes over i_n, eight
// loads in flight.
template <typename T, int RB>
__global__ void __launch_bounds__(FB_WARPS * 32) k_fiber_rows(FiberArgs a) {
  __shared__ double arow[FB_WARPS][TUCKER_MAX_ORDER * TUCKER_MAX_RANK];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nu = *a.nu, N = a.N, n = a.n, Rn = a.R[n];
  const int dn = a.d / Rn;                  // core entries per r_n
  const int postn = a.postn;
  double* ar = arow[wid];
  for (int64_t u = (int64_t)blockIdx.x * FB_WARPS + wid; u < nu;
       u += (int64_t)gridDim.x * FB_WARPS) {
    // multi-index over the modes k != n (last fastest), probability, fiber base
    uint64_t key = a.keys[u];
    int64_t j[TUCKER_MAX_ORDER];
    for (int k = N - 1; k >= 0; --k) {
      if (k == n) { j[k] = 0; continue; }
      j[k] = (int64_t)(key % (uint64_t)a.I[k]);
      key /= (uint64_t)a.I[k];
    }
    // p and w by lane 0 alone (FP64 divisions are expensive on this GPU), then shared
    int64_t base = 0;
    for (int k = 0; k < N; ++k)
      if (k != n) base += j[k] * a.stride[k];
    double w = 0.0;
    if (lane == 0) {
      double p = 1.0;
      bool first = true;
      for (int k = 0; k < N; ++k) {
        if (k == n) continue;
        const uint64_t* C = a.cdf[k];
        const uint64_t Q = C[a.I[k] - 1];
        const uint64_t q = C[j[k]] - (j[k] > 0 ? C[j[k] - 1] : 0);
        const double f = (double)q / (double)Q;
        p = first ? f : p * f;
        first = false;
      }
      w = (double)a.counts[u] / ((double)a.m * p);
    }
    w = __shfl_sync(0xffffffffu, w, 0);
    // factor rows a_k(j_k), k != n, into shared memory (offset k * TUCKER_MAX_RANK)
    for (int k = 0; k < N; ++k) {
      if (k == n) continue;
      for (int r = lane; r < a.R[k]; r += 32)
        ar[k * TUCKER_MAX_RANK + r] = load_as_double(a.A[k], j[k] * a.R[k] + r, a.is64);
    }
    __syncwarp();
    if (a.cp) {
      // CP: z_u[r] = prod_{k != n} a_k(j_k)[r], the Khatri-Rao row (modes in order)
      for (int r = lane; r < Rn; r += 32) {
        double b = 1.0;
        bool first = true;
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          const double v = ar[k * TUCKER_MAX_RANK + r];
          b = first ? v : b * v;
          first = false;
        }
        a.bb[u * Rn + r] = b;
        a.wb[u * Rn + r] = w * b;
      }
    } else {
    double acc[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) acc[r] = 0.0;
    for (int o = lane; o < dn; o += 32) {
      uint32_t rem = (uint32_t)o;
      double wv = 1.0;
      for (int k = N - 1; k >= 0; --k) {
        if (k == n) continue;
        const uint32_t qk = fdiv(rem, a.div_r[k]);
        wv *= ar[k * TUCKER_MAX_RANK + (rem - qk * (uint32_t)a.R[k])];
        rem = qk;
      }
      const uint32_t pre = fdiv((uint32_t)o, a.div_post);
      const double* gp = a.core + (size_t)pre * Rn * postn + (o - pre * postn);
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r < Rn) acc[r] = fma(gp[(size_t)r * postn], wv, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r < Rn) {
        const double b = warp_sum(acc[r]);
        if (lane == 0) {
          a.bb[u * Rn + r] = b;
          a.wb[u * Rn + r] = w * b;
        }
      }
    }
    }
    // the fiber x_u[i] = X[base + i stride_n], eight loads per lane in flight
    T* xs = static_cast<T*>(a.xs) + u * a.I[n];
    const int64_t In = a.I[n], sn = a.stride[n];
    for (int64_t i0 = lane; i0 < In; i0 += 32 * 8) {
      T v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t i = i0 + 32 * q;
        v[q] = i < In ? (a.is64 ? (T)static_cast<const double*>(a.X)[base + i * sn]
                                : (T)static_cast<const float*>(a.X)[base + i * sn])
                      : (T)0;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + 32 * q < In) xs[i0 + 32 * q] = v[q];
    }
    __syncwarp();
  }
}

// Split normal equations: CTA (row block, split s) sums its share of the sample,
// Y_s[i][r] = sum_u xs[u][i] wb[u][r] for 128 rows i, and (row block 0)
// M_s[r][r'] = sum_u wb[u][r] b[u][r'].  Fixed order within a split; RB >= R_n
// keeps the accumulators in registers.
template <typename T, int RB>
__global__ void __launch_bounds__(128) k_fiber_normal(FiberArgs a) {
  extern __shared__ double fsm[];
  double* wbd = fsm;                                // [64][Rn] staged rows of wb (FP64)
  double* bbd = wbd + 64 * a.R[a.n];                // [64][Rn] staged rows of b (row block 0)
  T* wbs = reinterpret_cast<T*>(bbd + 64 * a.R[a.n]);   // [64][Rn] wb in T
  const int nu = *a.nu, Rn = a.R[a.n];
  const int64_t In = a.I[a.n];
  const int s = blockIdx.y;
  const int64_t chunk = (nu + a.splits - 1) / a.splits;
  const int64_t u0 = s * chunk, u1 = min((int64_t)nu, u0 + chunk);
  const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
  T acc[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) acc[r] = (T)0;
  const T* xs = static_cast<const T*>(a.xs);
  const double* wb = a.wb;
  const bool mblock = blockIdx.x == 0;              // this CTA also forms M_s
  const int e0 = threadIdx.x, r0 = e0 / max(Rn, 1), c0 = e0 - r0 * Rn;
  const bool mthread = mblock && e0 < Rn * Rn;
  double m4[4] = {0.0, 0.0, 0.0, 0.0};             // four chains: FP64 FMA latency
  for (int64_t ub = u0; ub < u1; ub += 64) {
    const int nb = (int)min((int64_t)64, u1 - ub);
    __syncthreads();
    for (int e = threadIdx.x; e < nb * Rn; e += 128) {
      const double v = wb[ub * Rn + e];
      wbs[e] = (T)v;
      if (mblock) {
        wbd[e] = v;
        bbd[e] = a.bb[ub * Rn + e];
      }
    }
    __syncthreads();
    if (mthread)
      for (int q = 0; q < nb; ++q) m4[q & 3] = fma(wbd[q * Rn + r0], bbd[q * Rn + c0], m4[q & 3]);
    if (i < In) {
      for (int q0 = 0; q0 < nb; q0 += 16) {        // sixteen fiber loads in flight
        T xv[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          xv[j] = q0 + j < nb ? xs[(ub + q0 + j) * In + i] : (T)0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int q = q0 + j < nb ? q0 + j : q0;  // a zero x adds nothing
#pragma unroll
          for (int r = 0; r < RB; ++r)
            if (r < Rn) acc[r] = fma(xv[j], wbs[q * Rn + r], acc[r]);
        }
      }
    }
  }
  if (i < In) {
#pragma unroll
    for (int r = 0; r < RB; ++r)
      if (r < Rn) a.partY[((int64_t)s * In + i) * Rn + r] = (double)acc[r];
  }
  if (mblock)                                        // R_n^2 <= 128 here (else below)
    for (int e = threadIdx.x; e < Rn * Rn; e += 128) {
      if (e == e0 && mthread) {
        a.partM[(int64_t)s * Rn * Rn + e] = (m4[0] + m4[1]) + (m4[2] + m4[3]);
        continue;
      }
      const int r = e / Rn, c = e % Rn;             // R_n > 11: the rest, from global memory
      double v = 0.0;
      for (int64_t u = u0; u < u1; ++u) v = fma(wb[u * Rn + r], a.bb[u * Rn + c], v);
      a.partM[(int64_t)s * Rn * Rn + e] = v;
    }
}

// A^(n) = Y M^-1: every CTA sums the M partials (fixed order), adds lambda I,
// factors and inverts it (spd_inverse), then forms its FIN_ROWS rows of Y from
// the partials and applies the inverse.
constexpr int FIN_ROWS = 16;
__global__ void __launch_bounds__(256) k_fiber_finish(FiberArgs a) {
  extern __shared__ double fin[];
  const int Rn = a.R[a.n];
  double* Lm = fin;                                  // Rn x Rn
  double* Mi = Lm + Rn * Rn;                         // Rn x Rn
  double* Ys = Mi + Rn * Rn;                         // FIN_ROWS x Rn
  const int64_t In = a.I[a.n];
  for (int e = threadIdx.x; e < Rn * Rn; e += blockDim.x) {
    const int r = e / Rn, c = e % Rn;
    // the symmetric part, so that both triangles carry the same value; sixteen
    // loads of each in flight, added in order
    double v = 0.0, vt = 0.0;
    for (int s0 = 0; s0 < a.splits; s0 += 16) {
      double t[16], tt[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const bool ok = s0 + q < a.splits;
        t[q] = ok ? a.partM[(int64_t)(s0 + q) * Rn * Rn + e] : 0.0;
        tt[q] = ok ? a.partM[(int64_t)(s0 + q) * Rn * Rn + c * Rn + r] : 0.0;
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        v += t[q];
        vt += tt[q];
      }
    }
    Lm[e] = 0.5 * (v + vt) + (r == c ? a.lambda : 0.0);
  }
  __syncthreads();
  spd_inverse(Lm, Rn, Mi, a.status);
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * FIN_ROWS;
  const int rows = (int)min((int64_t)FIN_ROWS, In - i0);
  for (int e = threadIdx.x; e < rows * Rn; e += blockDim.x) {
    const int64_t i = i0 + e / Rn;
    const int r = e % Rn;
    double v = 0.0;
    for (int s0 = 0; s0 < a.splits; s0 += 16) {     // sixteen loads in flight, added in order
      double t[16];
#pragma unroll
      for (int q = 0; q < 16; ++q)
        t[q] = s0 + q < a.splits ? a.partY[((int64_t)(s0 + q) * In + i) * Rn + r] : 0.0;
#pragma unroll
      for (int q = 0; q < 16; ++q) v += t[q];
    }
    Ys[e] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < rows * Rn; e += blockDim.x) {
    const int li = e / Rn, x = e % Rn;
    double v = 0.0;
    for (int k = 0; k < Rn; ++k) v = fma(Mi[x * Rn + k], Ys[li * Rn + k], v);
    const int64_t i = i0 + li;
    if (a.is64) static_cast<double*>(a.A_out)[i * Rn + x] = v;
    else static_cast<float*>(a.A_out)[i * Rn + x] = (float)v;
  }
}

size_t fiber_workspace_bytes(const FactorSet& F, int n, int64_t cap, int splits) {
  const size_t es = F.is64 ? 8 : 4;
  const int Rn = F.R[n];
  return (size_t)cap * F.I[n] * es + 256 + 2 * ((size_t)cap * Rn * 8 + 256) +
         (size_t)splits * F.I[n] * Rn * 8 + 256 + (size_t)splits * Rn * Rn * 8 + 256;
}

int fiber_splits(int64_t cap) { return (int)std::max<int64_t>(1, std::min<int64_t>(64, cap / 256)); }

tucker_status launch_fiber_update(tucker_handle* h, const FactorSet& F, int n, const void* X,
                                  const double* core, const uint64_t* keys,
                                  const uint32_t* counts, const int* d_nu, int64_t cap,
                                  const uint64_t* const* cdf_others, int64_t m, double lambda,
                                  char* ws, size_t ws_bytes, void* A_out, int cp) {
  const int splits = fiber_splits(cap);
  if (fiber_workspace_bytes(F, n, cap, splits) > ws_bytes)
    return fail(h, TUCKER_EINTERNAL, "fiber workspace too small");
  const size_t es = F.is64 ? 8 : 4;
  const int Rn = F.R[n];
  FiberArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  a.n = n;
  int64_t st = 1;
  for (int k = F.N - 1; k >= 0; --k) {
    a.R[k] = F.R[k];
    a.I[k] = F.I[k];
    a.A[k] = F.A[k];
    a.stride[k] = st;
    st *= F.I[k];
  }
  int pos = 0;
  for (int k = 0; k < F.N; ++k) if (k != n) a.cdf[k] = cdf_others[pos++];
  a.is64 = F.is64;
  a.X = X;
  a.core = core;
  a.d = F.d;
  a.keys = keys;
  a.counts = counts;
  a.nu = d_nu;
  a.m = m;
  a.lambda = lambda;
  a.splits = splits;
  a.postn = 1;                              // the Tucker core's trailing size (unused for CP)
  if (!cp)
    for (int k = n + 1; k < F.N; ++k) a.postn *= F.R[k];
  for (int k = 0; k < F.N; ++k) a.div_r[k] = make_fastdiv((uint32_t)F.R[k]);
  a.div_post = make_fastdiv((uint32_t)a.postn);
  char* q = ws;
  auto take = [&](size_t bytes) { char* r = q; q += (bytes + 255) & ~size_t(255); return r; };
  a.xs = take((size_t)cap * F.I[n] * es);
  a.wb = reinterpret_cast<double*>(take((size_t)cap * Rn * 8));
  a.bb = reinterpret_cast<double*>(take((size_t)cap * Rn * 8));
  a.partY = reinterpret_cast<double*>(take((size_t)splits * F.I[n] * Rn * 8));
  a.partM = reinterpret_cast<double*>(take((size_t)splits * Rn * Rn * 8));
  a.A_out = A_out;
  a.status = h->d_status;
  a.cp = cp;
  const int g1 = (int)std::min<int64_t>(ceil_div(cap, FB_WARPS), (int64_t)h->num_sms * 16);
  TK_COUNT(h);
#define TK_FIBER_ROWS(RB)                                                                  \
  do {                                                                                     \
    if (F.is64) k_fiber_rows<double, RB><<<std::max(g1, 1), FB_WARPS * 32, 0, h->stream>>>(a); \
    else k_fiber_rows<float, RB><<<std::max(g1, 1), FB_WARPS * 32, 0, h->stream>>>(a);          \
  } while (0)
  if (Rn <= 4) TK_FIBER_ROWS(4);
  else if (Rn <= 8) TK_FIBER_ROWS(8);
  else if (Rn <= 16) TK_FIBER_ROWS(16);
  else if (Rn <= 32) TK_FIBER_ROWS(32);
  else TK_FIBER_ROWS(64);
#undef TK_FIBER_ROWS
  TK_LAUNCH(h);
  const dim3 g2((unsigned)ceil_div(F.I[n], 128), (unsigned)splits);
  const size_t sm2 = (size_t)64 * Rn * (16 + es);
  TK_COUNT(h);
  // (over 48 KB of dynamic shared memory for R_n > 32: the limit is raised per instance)
#define TK_FIBER_NORMAL(RB)                                                        \
  do {                                                                             \
    if (F.is64) {                                                                  \
      TK_CUDA(h, cudaFuncSetAttribute(k_fiber_normal<double, RB>,                  \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)sm2));                                  \
      k_fiber_normal<double, RB><<<g2, 128, sm2, h->stream>>>(a);                  \
    } else {                                                                       \
      TK_CUDA(h, cudaFuncSetAttribute(k_fiber_normal<float, RB>,                   \
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                      (int)sm2));                                  \
      k_fiber_normal<float, RB><<<g2, 128, sm2, h->stream>>>(a);                   \
    }                                                                              \
  } while (0)
  if (Rn <= 4) TK_FIBER_NORMAL(4);
  else if (Rn <= 8) TK_FIBER_NORMAL(8);
  else if (Rn <= 16) TK_FIBER_NORMAL(16);
  else if (Rn <= 32) TK_FIBER_NORMAL(32);
  else TK_FIBER_NORMAL(64);
#undef TK_FIBER_NORMAL
  TK_LAUNCH(h);
  const size_t sm3 = (size_t)(2 * Rn * Rn + FIN_ROWS * Rn) * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_fiber_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm3));
  TK_COUNT(h);
  k_fiber_finish<<<(unsigned)ceil_div(F.I[n], FIN_ROWS), 256, sm3, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
