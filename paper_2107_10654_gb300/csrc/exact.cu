// Exact core update for dense X (the plain method), n-mode product chains and
// the FP64 residual used for losses.
//
// Exact core (Alg. 2 core line, solved through the eigendecomposition of the
// proof of Lemma 4.1): with A^(n)T A^(n) = V_n diag(s_n) V_n^T,
//     y = K^T vec X = vec(X x_1 A^(1)T ... x_N A^(N)T)       (n-mode products, Sec. 2)
//     z = y x_n V_n^T;  z /= (s_1 (x) ... (x) s_N + lambda);  g = z x_n V_n.
// The first product streams X once (HBM-bound: one warp per row of the last
// mode, lanes over the row, R_N accumulators, A^(N) in shared memory); the
// rest act on tensors with at most prod(I)/I_N * R_N entries.
#include <algorithm>

#include "common.cuh"

namespace tk {

// Sum v[0..RP) over the 32 lanes so that lane l ends with the total of entry
// r(l) = bits (4, 3, ..) of l: halving exchanges (RP/2 + RP/4 + ... + 1
// shuffles) then plain butterflies over the remaining lane bits.  Lanes with
// (l & (32/RP - 1)) == 0 hold distinct r = l / (32/RP).
template <class T, int RP>
__device__ __forceinline__ T transpose_reduce(T (&v)[RP], int lane) {
  int width = RP;
#pragma unroll
  for (int o = 16; o >= 32 / RP; o >>= 1) {
    const bool upper = lane & o;
    const int h = width >> 1;
#pragma unroll
    for (int j = 0; j < RP / 2; ++j) {
      if (j < h) {
        const T send = upper ? v[j] : v[j + h];
        const T recv = __shfl_xor_sync(0xffffffffu, send, o);
        v[j] = (upper ? v[j + h] : v[j]) + recv;
      }
    }
    width = h;
  }
  T x = v[0];
#pragma unroll
  for (int o = (32 / RP) >> 1; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Rows blocked per warp: RB rows are contracted at once so that every
// 16-byte load of A^T from shared memory feeds RB rows (the shared-memory
// traffic per byte of X falls by RB) and RB independent row loads are in
// flight per lane.  Row r's accumulators see the same operations in the same
// order as a warp working on that row alone.
template <int RP> struct RowBlock { static constexpr int RB = RP <= 8 ? 4 : RP <= 16 ? 2 : 1; };

// Sum of squares of the elements read, with the arithmetic of k_tensor_sumsq:
// FP64 FMAs for FP64 data; for FP32 data error-free products p + e = x^2
// (e = fma(x, x, -p)) added with Neumaier's compensation.
template <class T> struct SqAcc {
  double s = 0.0;
  __device__ __forceinline__ void add(T v) { s = fma((double)v, (double)v, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <> struct SqAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float p = v * v;
    const float e = fmaf(v, v, -p);
    const float t = s + p;
    c += (fabsf(s) >= fabsf(p)) ? ((s - t) + p) : ((p - t) + s);
    c += e;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// acc[r][j] = lane's partial of sum_i rows[r][i] At[j][i], r < nr; with SQ also
// the squares of the row elements into sq.
template <class T, int RP, int RB, bool SQ = false>
__device__ __forceinline__ void rows_contract(const T* const* rows, int nr, int I, const T* At,
                                              bool vec, int lane, T (&acc)[RB][RP],
                                              SqAcc<T>* sq = nullptr) {
  constexpr int VEC = 16 / sizeof(T);
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int j = 0; j < RP; ++j) acc[r][j] = T(0);
  if (vec) {
    // the loads of the next 16-byte column group are issued before the
    // multiply-adds of the current one (2 RB loads in flight per lane)
    T xv[RB][VEC], xn[RB][VEC];
    if (lane * VEC < I) {
#pragma unroll
      for (int r = 0; r < RB; ++r)
        if (r < nr)
          *reinterpret_cast<uint4*>(xv[r]) = __ldg(reinterpret_cast<const uint4*>(rows[r] + lane * VEC));
    }
    for (int i0 = lane * VEC; i0 < I; i0 += 32 * VEC) {
      if (i0 + 32 * VEC < I) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if (r < nr)
            *reinterpret_cast<uint4*>(xn[r]) =
                __ldg(reinterpret_cast<const uint4*>(rows[r] + i0 + 32 * VEC));
      }
      if (SQ) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if (r < nr)
#pragma unroll
            for (int q = 0; q < VEC; ++q) sq->add(xv[r][q]);
      }
#pragma unroll
      for (int j = 0; j < RP; ++j) {
        T av[VEC];
        *reinterpret_cast<uint4*>(av) = *reinterpret_cast<const uint4*>(At + j * I + i0);
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
          for (int q = 0; q < VEC; ++q) acc[r][j] = fma(xv[r][q], av[q], acc[r][j]);
      }
#pragma unroll
      for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int q = 0; q < VEC; ++q) xv[r][q] = xn[r][q];
    }
  } else {
    for (int i = lane; i < I; i += 32) {
      T x[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) x[r] = r < nr ? rows[r][i] : T(0);
      if (SQ) {
#pragma unroll
        for (int r = 0; r < RB; ++r)
          if (r < nr) sq->add(x[r]);
      }
#pragma unroll
      for (int j = 0; j < RP; ++j) {
        const T a = At[j * I + i];
#pragma unroll
        for (int r = 0; r < RB; ++r) acc[r][j] = fma(x[r], a, acc[r][j]);
      }
    }
  }
}

// out[p][r] = sum_i X[p][i] A[i][r]   (X: P x I row-major; out FP64 P x R)
// One warp per RB consecutive rows; A^T in shared memory ([r][i],
// conflict-free); 16-byte loads of X when the row length allows; R <= RP
// accumulators per row and lane.
// With SQ every CTA also writes the sum of squares of the rows it read to
// sq_partial[blockIdx.x] (rows are assigned to warps in a fixed pattern, so the
// partials and their fixed-order sum are reproducible).
template <class T, int RP, bool SQ>
__global__ void __launch_bounds__(256) k_ttm_last(const T* X, int64_t P, int I, const T* A, int R,
                                                  double* out, double* sq_partial) {
  pdl_wait();
  constexpr int RB = RowBlock<RP>::RB;
  extern __shared__ unsigned char smraw[];
  T* At = reinterpret_cast<T*>(smraw);               // RP x I (zero rows beyond R)
  for (int e = threadIdx.x; e < RP * I; e += blockDim.x) {
    const int r = e / I, i = e % I;
    At[e] = r < R ? A[(int64_t)i * R + r] : T(0);
  }
  __syncthreads();
  constexpr int VEC = 16 / sizeof(T);
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool vec = (I % VEC) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  SqAcc<T> sq;
  for (int64_t p0 = warp * RB; p0 < P; p0 += nwarps * RB) {
    const int nr = (int)(P - p0 < RB ? P - p0 : RB);
    const T* rows[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) rows[r] = X + (p0 + (r < nr ? r : 0)) * I;
    T acc[RB][RP];
    rows_contract<T, RP, RB, SQ>(rows, nr, I, At, vec, lane, acc, &sq);
    constexpr int G = 32 / RP;
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (r >= nr) break;
      const T tot = transpose_reduce<T, RP>(acc[r], lane);
      if ((lane % G) == 0) {
        const int c = lane / G;
        if (c < R) out[(p0 + r) * R + c] = (double)tot;
      }
    }
  }
  if (SQ) {
    __shared__ double red[8];
    const double v = warp_sum(sq.value());
    if (lane == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      sq_partial[blockIdx.x] = t;
    }
  }
}

// Fused contraction of the last two modes:
// part[p][c][a][b] = sum_{i in chunk c, j} X[p][i][j] A1[i][a] A2[j][b]
// (A1 = A^(N-1), I1 x R1; A2 = A^(N), I2 x R2; the I1 rows of a slab cut into
// nchunk chunks).
// It runs in warp-sized work items: each warp of the grid takes
// items (slab p, row chunk c) in turn, reduces the chunk's rows against A2 RB at
// a time in increasing i and adds A1[i][a] * t[b] into its accumulators, then
// writes the item's R1 R2 partial sums (k_sum_chunks adds a slab's chunks in
// order).  No CTA barrier separates the items, so a warp never waits for the
// others between chunks.
template <class T, int RP>
__global__ void __launch_bounds__(256) k_ttm_last2w(const T* X, int64_t pre, int I1, int I2,
                                                    const T* A1, int R1, const T* A2, int R2,
                                                    int nchunk, double* out) {
  pdl_wait();
  constexpr int RB = RowBlock<RP>::RB;
  extern __shared__ unsigned char smraw[];
  T* At = reinterpret_cast<T*>(smraw);                         // RP x I2
  T* A1s = reinterpret_cast<T*>(smraw + (((size_t)RP * I2 * sizeof(T) + 15) & ~size_t(15)));
  for (int e = threadIdx.x; e < RP * I2; e += blockDim.x) {
    const int r = e / I2, j = e % I2;
    At[e] = r < R2 ? A2[(int64_t)j * R2 + r] : T(0);
  }
  for (int e = threadIdx.x; e < I1 * R1; e += blockDim.x) A1s[e] = A1[e];
  constexpr int VEC = 16 / sizeof(T);
  constexpr int G = 32 / RP;
  const int lane = threadIdx.x & 31;
  const int RR = R1 * R2;
  const bool vec = (I2 % VEC) == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  int ea[8], esrc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = lane + 32 * q;
    ea[q] = e < RR ? e / R2 : -1;
    esrc[q] = ((e % R2) % RP) * G;
  }
  __syncthreads();
  const int crows = (I1 + nchunk - 1) / nchunk;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t item = gw; item < pre * nchunk; item += nw) {
    const int64_t p = item / nchunk;
    const int c = (int)(item - p * nchunk);
    const int i0 = c * crows, iend = min(I1, i0 + crows);
    T y[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) y[q] = T(0);
    const T* slab = X + p * (int64_t)I1 * I2;
    for (int i = i0; i < iend; i += RB) {
      const int nr = min(RB, iend - i);
      const T* rows[RB];
#pragma unroll
      for (int r = 0; r < RB; ++r) rows[r] = slab + (int64_t)(i + (r < nr ? r : 0)) * I2;
      T acc[RB][RP];
      rows_contract<T, RP, RB>(rows, nr, I2, At, vec, lane, acc);
#pragma unroll
      for (int r = 0; r < RB; ++r) {
        if (r >= nr) break;
        const T t = transpose_reduce<T, RP>(acc[r], lane);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (32 * q >= RR) break;
          const T tb = __shfl_sync(0xffffffffu, t, esrc[q]);
          if (ea[q] >= 0) y[q] = fma(A1s[(i + r) * R1 + ea[q]], tb, y[q]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = lane + 32 * q;
      if (e < RR) out[item * RR + e] = (double)y[q];
    }
  }
}

// out[p][e] = sum_c part[p][c][e] in increasing c.
__global__ void k_sum_chunks(const double* part, int64_t pre, int nchunk, int RR, double* out) {
  pdl_wait();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < pre * RR;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / RR;
    const int e = (int)(t - p * RR);
    double v = 0.0;
    for (int c = 0; c < nchunk; ++c) v += part[(p * nchunk + c) * RR + e];
    out[t] = v;
  }
}

// out[p][r][q] = sum_i X[p][i][q] A[i][r]   (big X, middle mode; coalesced over q)
// out[p][r][q] = sum_i X[p][i][q] A[i][r]   (big X, middle mode; coalesced over q)
// A thread owns QB consecutive columns q (16-byte loads of X when post and the
// base allow) and RC outputs r at a time; eight rows i are loaded before
// their multiply-adds, which run in increasing i.
template <class T, int RC>
__global__ void __launch_bounds__(256) k_ttm_mid(const T* X, int64_t pre, int I, int64_t post,
                                                 const T* A, int R, double* out) {
  pdl_wait();
  extern __shared__ unsigned char smraw[];
  T* As = reinterpret_cast<T*>(smraw);
  for (int e = threadIdx.x; e < I * R; e += blockDim.x) As[e] = A[e];
  __syncthreads();
  constexpr int QB = 16 / sizeof(T);
  const bool vec = post % QB == 0 && (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  const int qb = vec ? QB : 1;
  const int64_t pq = post / qb;                           // column groups per slab
  const int64_t total = pre * pq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = t / pq, q0 = (t - p * pq) * qb;
    const T* xp = X + p * I * post + q0;
    for (int r0 = 0; r0 < R; r0 += RC) {
      T acc[RC][QB];
#pragma unroll
      for (int j = 0; j < RC; ++j)
#pragma unroll
        for (int c = 0; c < QB; ++c) acc[j][c] = T(0);
      for (int i0 = 0; i0 < I; i0 += 8) {
        T xs[8][QB];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (vec) {
            if (i0 + u < I)
              *reinterpret_cast<uint4*>(xs[u]) =
                  __ldg(reinterpret_cast<const uint4*>(xp + (int64_t)(i0 + u) * post));
            else
#pragma unroll
              for (int c = 0; c < QB; ++c) xs[u][c] = T(0);
          } else {
            xs[u][0] = i0 + u < I ? __ldg(xp + (int64_t)(i0 + u) * post) : T(0);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (i0 + u >= I) break;
#pragma unroll
          for (int j = 0; j < RC; ++j) {
            if (r0 + j >= R) break;
            const T a = As[(i0 + u) * R + r0 + j];
#pragma unroll
            for (int c = 0; c < QB; ++c)
              if (c < qb) acc[j][c] = fma(xs[u][c], a, acc[j][c]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < RC; ++j)
        if (r0 + j < R)
#pragma unroll
          for (int c = 0; c < QB; ++c)
            if (c < qb) out[(p * R + r0 + j) * post + q0 + c] = (double)acc[j][c];
    }
  }
}

// contract: out[p][r][q] = sum_{i<I} in[p][i][q] A[i][r]   (out middle dim R)
// expand:   out[p][i][q] = sum_{r<R} in[p][r][q] A[i][r]   (out middle dim I)
__global__ void k_ttm_small(const double* in, int64_t pre, int64_t post, const void* A, int is64,
                            int I, int R, int contract, double* out) {
  pdl_wait();
  const int K = contract ? I : R, M = contract ? R : I;
  const int64_t total = pre * M * post;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = t % post;
    const int mo = (int)((t / post) % M);
    const int64_t p = t / (post * M);
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
      const double a = contract ? load_as_double(A, (int64_t)k * R + mo, is64)
                                : load_as_double(A, (int64_t)mo * R + k, is64);
      acc = fma(in[(p * K + k) * post + q], a, acc);
    }
    out[t] = acc;
  }
}

// Same as k_ttm_small, one warp per output (lanes over the contracted index)
// for long contractions; fixed butterfly order.
__global__ void k_ttm_small_warp(const double* in, int64_t pre, int64_t post, const void* A,
                                 int is64, int I, int R, int contract, double* out) {
  pdl_wait();
  const int K = contract ? I : R, M = contract ? R : I;
  const int64_t total = pre * M * post;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = warp; t < total; t += nwarps) {
    const int64_t q = t % post;
    const int mo = (int)((t / post) % M);
    const int64_t p = t / (post * M);
    double acc = 0.0;
    for (int k = lane; k < K; k += 32) {
      const double a = contract ? load_as_double(A, (int64_t)k * R + mo, is64)
                                : load_as_double(A, (int64_t)mo * R + k, is64);
      acc = fma(in[(p * K + k) * post + q], a, acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[t] = acc;
  }
}

// Contract mode with a short trailing extent (post divides 32, R <= 16): one
// warp per leading index p, lane = (k phase, q) with q = lane % post, all R
// outputs of the lane's q in registers; in[p][k][q] is read once, coalesced,
// and the k phases are added by a fixed butterfly over the phase bits.
template <int RM>
__global__ void k_ttm_small_rows(const double* in, int64_t pre, int64_t post, const void* A,
                                 int is64, int I, int R, double* out) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int q = lane % (int)post, kph = lane / (int)post, nph = 32 / (int)post;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < pre; p += nwarps) {
    double acc[RM];
#pragma unroll
    for (int r = 0; r < RM; ++r) acc[r] = 0.0;
    const double* base = in + (p * I) * post + q;
    for (int k = kph; k < I; k += nph) {
      const double x = base[(int64_t)k * post];
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) acc[r] = fma(x, load_as_double(A, (int64_t)k * R + r, is64), acc[r]);
    }
#pragma unroll
    for (int r = 0; r < RM; ++r)
      for (int o = (int)post; o < 32; o <<= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
    if (kph == 0)
#pragma unroll
      for (int r = 0; r < RM; ++r)
        if (r < R) out[(p * R + r) * post + q] = acc[r];
  }
}

// g = (x V_n) [ ((x V_n)^T y) / (x s_n + lambda) ]   -- one CTA, d <= 8192
struct EigArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  const double* V[TUCKER_MAX_ORDER];   // R x R, V[a][k]
  const double* s[TUCKER_MAX_ORDER];   // R eigenvalues
  const double* y;
  double lambda;
  double* g;
  int d;
};

__global__ void __launch_bounds__(1024) k_kron_eig_core(EigArgs a) {
  extern __shared__ double buf[];
  double* z0 = buf;
  double* z1 = buf + a.d;
  for (int i = threadIdx.x; i < a.d; i += blockDim.x) z0[i] = a.y[i];
  __syncthreads();
  // forward: z <- z x_n V_n^T  (z[p][k][q] = sum_a z[p][a][q] V[a][k])
  for (int pass = 0; pass < 2; ++pass) {
    int pre = 1;
    for (int n = 0; n < a.N; ++n) {
      const int R = a.R[n];
      const int post = a.d / (pre * R);
      for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
        const int q = t % post, k = (t / post) % R, p = t / (post * R);
        double acc = 0.0;
        for (int j = 0; j < R; ++j) {
          const double v = pass == 0 ? a.V[n][j * R + k] : a.V[n][k * R + j];
          acc = fma(z0[(p * R + j) * post + q], v, acc);
        }
        z1[t] = acc;
      }
      __syncthreads();
      double* tmp = z0; z0 = z1; z1 = tmp;
      pre *= R;
    }
    if (pass == 0) {
      for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
        double ev = 1.0;
        int rem = t;
        for (int n = a.N - 1; n >= 0; --n) { ev *= a.s[n][rem % a.R[n]]; rem /= a.R[n]; }
        z0[t] /= (ev + a.lambda);
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < a.d; i += blockDim.x) a.g[i] = z0[i];
}

// Residual sum of squares  sum_p sum_i (X[p][i] - T[p] . A^(N)[i])^2  in FP64,
// T = G x_1 A^(1) ... x_{N-1} A^(N-1) (P x R rows).  Block partials.
__global__ void __launch_bounds__(256) k_residual_dense(const void* X, int is64, int64_t P, int I,
                                                        const double* T, const void* A, int R,
                                                        double* partial) {
  pdl_wait();
  extern __shared__ double As[];             // I x R
  __shared__ double red[8];
  for (int e = threadIdx.x; e < I * R; e += blockDim.x) As[e] = load_as_double(A, e, is64);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double acc = 0.0;
  for (int64_t p = warp; p < P; p += nwarps) {
    const double* t = T + p * R;
    for (int i = lane; i < I; i += 32) {
      double xh = 0.0;
      for (int r = 0; r < R; ++r) xh = fma(t[r], As[i * R + r], xh);
      const double e = load_as_double(X, p * I + i, is64) - xh;
      acc = fma(e, e, acc);
    }
  }
  acc = warp_sum(acc);
  if (lane == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(256) k_residual_coo(const uint64_t* keys, const void* vals,
                                                      int is64, int64_t nnz, int I,
                                                      const double* T, const void* A, int R,
                                                      double* partial) {
  pdl_wait();
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[e];
    const int64_t p = (int64_t)(k / (uint64_t)I);
    const int i = (int)(k % (uint64_t)I);
    double xh = 0.0;
    for (int r = 0; r < R; ++r) xh = fma(T[p * R + r], load_as_double(A, (int64_t)i * R + r, is64), xh);
    const double d = load_as_double(vals, e, is64) - xh;
    acc = fma(d, d, acc);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials(const double* partial, int n, double* out) {
  pdl_wait();
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = t;
  }
}

// sum of squares of a device FP64/FP32 array (block partials + final sum)
__global__ void k_sumsq(const void* v, int is64, int64_t n, double* partial) {
  pdl_wait();
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double x = load_as_double(v, i, is64);
    s = fma(x, x, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// ||X||^2 of a dense tensor for the Gram-identity loss.  FP32 data: every
// square is split without error, x^2 = p + e with p = fl(x x) and e = fma(x,
// x, -p), and each thread sums its p in FP32 with Neumaier's compensation
// (e and the compensation in a second FP32 sum); the per-thread pairs are
// added in FP64.  The loss L = ||X||^2 - 2 g.y + g.Hg cancels most of ||X||^2
// (by about 5e-6 relative on the 512^3 workload), so ||X||^2 must be accurate
// well below the FP32 rounding of a single sum.  FP64 data: FP64 products.
__global__ void __launch_bounds__(256) k_tensor_sumsq(const void* X, int is64, int vec,
                                                      int64_t n, double* partial) {
  pdl_wait();
  __shared__ double red[8];
  double acc;
  if (is64) {
    const double* x = static_cast<const double*>(X);
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      s = fma(x[i], x[i], s);
    acc = s;
  } else {
    const float* x = static_cast<const float*>(X);
    float s = 0.f, c = 0.f;
    auto add = [&](float v) {
      const float p = v * v;
      const float e = fmaf(v, v, -p);
      const float t = s + p;
      c += (fabsf(s) >= fabsf(p)) ? ((s - t) + p) : ((p - t) + s);
      c += e;
      s = t;
    };
    const int64_t n4 = vec ? n >> 2 : 0;                // 16-byte loads when X is aligned
    const float4* x4 = reinterpret_cast<const float4*>(x);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
      const float4 v = __ldg(x4 + i);
      add(v.x); add(v.y); add(v.z); add(v.w);
    }
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      add(x[i]);
    acc = (double)s + (double)c;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    partial[blockIdx.x] = t;
  }
}

// y = K^T vec(X) from the last factor update's product chain B = (X x_{k<N}
// A^(k)T) laid out (pre, I_N) with pre = prod_{k<N} R_k: y[p R_N + r] =
// sum_i A^(N)[i][r] B[p][i] (one warp per entry, FP64).
__global__ void k_kt_x_from_last(const double* B, int64_t pre, int64_t IN, const void* A,
                                 int is64, int RN, double* y) {
  pdl_wait();
  const int lane = threadIdx.x & 31;
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= pre * RN) return;
  const int64_t p = e / RN;
  const int r = (int)(e - p * RN);
  double acc = 0.0;
  for (int64_t i = lane; i < IN; i += 32) acc = fma(B[p * IN + i], load_as_double(A, i * RN + r, is64), acc);
  acc = warp_sum(acc);
  if (lane == 0) y[e] = acc;
}

// out = g.(x_n G_n) g (one CTA; the Kronecker product applied mode by mode in
// shared memory), and out[1] = g.y, out[2] = g.g: the terms of the loss
// L = ||X||^2 - 2 g.y + g.Hg + lambda (||g||^2 + sum ||A^(n)||^2).
struct KronQuadArgs {
  int N, d;
  int R[TUCKER_MAX_ORDER];
  const double* gram[TUCKER_MAX_ORDER];
  const double* g;
  const double* y;
  double* out;
};

__global__ void __launch_bounds__(1024) k_kron_quad(KronQuadArgs a) {
  extern __shared__ double kq[];
  double* z0 = kq;
  double* z1 = kq + a.d;
  __shared__ double red[3][32];
  for (int t = threadIdx.x; t < a.d; t += blockDim.x) z0[t] = a.g[t];
  __syncthreads();
  int pre = 1;
  for (int k = 0; k < a.N; ++k) {
    const int Rk = a.R[k];
    const int post = a.d / (pre * Rk);
    for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
      const int q = t % post, r = (t / post) % Rk, pp = t / (post * Rk);
      double acc = 0.0;
      for (int j = 0; j < Rk; ++j) acc = fma(a.gram[k][r * Rk + j], z0[(pp * Rk + j) * post + q], acc);
      z1[t] = acc;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < a.d; t += blockDim.x) z0[t] = z1[t];
    __syncthreads();
    pre *= Rk;
  }
  double q = 0.0, gy = 0.0, gg = 0.0;
  for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
    const double gt = a.g[t];
    q = fma(gt, z0[t], q);
    gy = fma(gt, a.y[t], gy);
    gg = fma(gt, gt, gg);
  }
  q = warp_sum(q);
  gy = warp_sum(gy);
  gg = warp_sum(gg);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red[0][w] = q; red[1][w] = gy; red[2][w] = gg; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { s0 += red[0][k]; s1 += red[1][k]; s2 += red[2][k]; }
    a.out[0] = s0;
    a.out[1] = s1;
    a.out[2] = s2;
  }
}

// ------------------------------------------------------------------- host side

static int grid_for(tucker_handle* h, int64_t work, int per = 256) {
  int64_t g = (work + per - 1) / per;
  int64_t cap = (int64_t)h->num_sms * 32;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

// Contract the last mode of the dense X: out = X_(as P x I_N) A^(N)  (FP64 out)
template <class T>
static tucker_status ttm_last_t(tucker_handle* h, const T* X, int64_t P, int I, const T* A, int R,
                                double* out, double* sq_partial, int sq_cap, double* sq_out) {
  const int RP = R <= 4 ? 4 : R <= 8 ? 8 : R <= 16 ? 16 : 32;
  const size_t smem = (size_t)RP * I * sizeof(T);
  if (smem > 200 * 1024) return fail(h, TUCKER_ENOTSUP, "I_N * R_N too large for the TTM kernel");
  const bool sq = sq_partial != nullptr;
  auto k = sq ? (RP == 4 ? k_ttm_last<T, 4, true> : RP == 8 ? k_ttm_last<T, 8, true>
                 : RP == 16 ? k_ttm_last<T, 16, true> : k_ttm_last<T, 32, true>)
              : (RP == 4 ? k_ttm_last<T, 4, false> : RP == 8 ? k_ttm_last<T, 8, false>
                 : RP == 16 ? k_ttm_last<T, 16, false> : k_ttm_last<T, 32, false>);
  TK_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TK_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
  int64_t grid = (int64_t)h->num_sms * (per_sm > 0 ? per_sm : 1);
  const int64_t need = (P + 31) / 32;                 // 8 warps x 4 rows per CTA
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if (sq && grid > sq_cap) return fail(h, TUCKER_EINTERNAL, "square-sum partials too few");
  TK_CUDA(h, launch_dep(h, k, (int)grid, 256, smem, X, P, I, A, R, out, sq_partial));
  if (sq) TK_CUDA(h, launch_dep(h, k_sum_partials, 1, 1024, 0, sq_partial, (int)grid, sq_out));
  return TUCKER_OK;
}

// sq_partial (nullable, sq_cap doubles): also ||X||^2 into *sq_out, from the
// same pass over X.
tucker_status ttm_last(tucker_handle* h, const void* X, int is64, int64_t P, int I, const void* A,
                       int R, double* out, double* sq_partial = nullptr, int sq_cap = 0,
                       double* sq_out = nullptr) {
  if (R > 32) return fail(h, TUCKER_ENOTSUP, "R_N > 32 in the TTM kernel");
  if (is64)
    return ttm_last_t<double>(h, (const double*)X, P, I, (const double*)A, R, out, sq_partial,
                              sq_cap, sq_out);
  return ttm_last_t<float>(h, (const float*)X, P, I, (const float*)A, R, out, sq_partial, sq_cap,
                           sq_out);
}

tucker_status ttm_mid(tucker_handle* h, const void* X, int is64, int64_t pre, int I, int64_t post,
                      const void* A, int R, double* out) {
  const size_t smem = (size_t)I * R * (is64 ? 8 : 4);
  const int grid = grid_for(h, pre * post);
  if (is64) {
    auto k = R <= 8 ? k_ttm_mid<double, 8> : k_ttm_mid<double, 16>;
    TK_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TK_CUDA(h, launch_dep(h, k, grid, 256, smem, (const double*)X, pre, I, post, (const double*)A,
                          R, out));
  } else {
    auto k = R <= 8 ? k_ttm_mid<float, 8> : k_ttm_mid<float, 16>;
    TK_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TK_CUDA(h, launch_dep(h, k, grid, 256, smem, (const float*)X, pre, I, post, (const float*)A, R,
                          out));
  }
  return TUCKER_OK;
}

tucker_status ttm_small(tucker_handle* h, const double* in, int64_t pre, int64_t post,
                        const void* A, int is64, int I, int R, int contract, double* out) {
  const int64_t total = pre * (contract ? R : I) * post;
  const int K = contract ? I : R;
  if (contract && K >= 64 && post <= 32 && 32 % post == 0 && R <= 16) {
    const int64_t blocks = (pre * 32 + 255) / 256;
    const int grid = (int)std::min<int64_t>(blocks, (int64_t)h->num_sms * 16);
    TK_CUDA(h, launch_dep(h, R <= 8 ? k_ttm_small_rows<8> : k_ttm_small_rows<16>, grid, 256, 0, in,
                          pre, post, A, is64, I, R, out));
  } else if (K >= 64 && total < (int64_t)h->num_sms * 2048) {
    TK_CUDA(h, launch_dep(h, k_ttm_small_warp, grid_for(h, total * 32), 256, 0, in, pre, post, A,
                          is64, I, R, contract, out));
  } else {
    TK_CUDA(h, launch_dep(h, k_ttm_small, grid_for(h, total), 256, 0, in, pre, post, A, is64, I, R,
                          contract, out));
  }
  return TUCKER_OK;
}

template <class T>
static tucker_status ttm_last2_t(tucker_handle* h, const T* X, int64_t pre, int I1, int I2,
                                 const T* A1, int R1, const T* A2, int R2, double* part,
                                 double* out) {
  const int RP = R2 <= 4 ? 4 : R2 <= 8 ? 8 : R2 <= 16 ? 16 : 32;
  const size_t smem = (((size_t)RP * I2 * sizeof(T) + 15) & ~size_t(15)) +
                      (((size_t)I1 * R1 * sizeof(T) + 15) & ~size_t(15));
  auto k = RP == 4 ? k_ttm_last2w<T, 4> : RP == 8 ? k_ttm_last2w<T, 8>
         : RP == 16 ? k_ttm_last2w<T, 16> : k_ttm_last2w<T, 32>;
  TK_CUDA(h, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  TK_CUDA(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem));
  int64_t grid = (int64_t)h->num_sms * (per_sm > 0 ? per_sm : 1);
  // row chunks per slab: about four items per warp of the grid, each chunk at
  // least 4 RB rows, the partials within the prod(I)/I_N * R_N buffer
  const int RB = RP <= 8 ? 4 : RP <= 16 ? 2 : 1;
  int nchunk = 1;
  while (pre * nchunk < 4 * grid * 8 && I1 / (2 * nchunk) >= 4 * RB && 2 * nchunk * R1 <= I1)
    nchunk *= 2;
  const int64_t items = pre * nchunk;
  if (grid * 8 > items) grid = (items + 7) / 8;
  const int RR = R1 * R2;
  TK_CUDA(h, launch_dep(h, k, (int)grid, 256, smem, X, pre, I1, I2, A1, R1, A2, R2, nchunk,
                        nchunk > 1 ? part : out));
  if (nchunk > 1)
    TK_CUDA(h, launch_dep(h, k_sum_chunks, ceil_div(pre * RR, 256), 256, 0, part, pre, nchunk, RR,
                          out));
  return TUCKER_OK;
}

// Can the last two modes be contracted in one streaming pass?
static bool fused_last2_ok(tucker_handle* h, const FactorSet& F) {
  const int N = F.N;
  if (N < 3) return false;
  const int64_t I1 = F.I[N - 2], I2 = F.I[N - 1];
  const int R1 = F.R[N - 2], R2 = F.R[N - 1];
  const int64_t pre = (int64_t)(F.total / (uint64_t)(I1 * I2));
  const int RP = R2 <= 4 ? 4 : R2 <= 8 ? 8 : R2 <= 16 ? 16 : 32;
  const size_t smem = (size_t)RP * I2 * (F.is64 ? 8 : 4) + (size_t)I1 * R1 * 8 + 8 * R1 * R2 * 8 + 16;
  return R2 <= 32 && R1 * R2 <= 256 && R1 <= I1 && pre >= h->num_sms && smem <= 160 * 1024;
}

// y = X x_1 A^(1)T ... x_N A^(N)T  (all modes), FP64 d-vector.  buf: two
// scratch arrays of prod(I)/I_N * R_N doubles.
tucker_status ttm_chain_all(tucker_handle* h, const FactorSet& F, const void* X, double* buf0,
                            double* buf1, double* y) {
  const int N = F.N;
  if (fused_last2_ok(h, F)) {
    const int I1 = (int)F.I[N - 2], I2 = (int)F.I[N - 1];
    const int64_t pre = (int64_t)(F.total / (uint64_t)((int64_t)I1 * I2));
    double* cur = (N == 2) ? y : buf0;
    // chunk partials in the other buffer (pre * 16 * R1 R2 doubles at most, within
    // the prod(I) / I_N * R_N of a buffer because I_{N-1} >= 32 * chunks)
    double* part = cur == buf0 ? buf1 : buf0;
    if (F.is64)
      TK_TRY(ttm_last2_t<double>(h, (const double*)X, pre, I1, I2, (const double*)F.A[N - 2],
                                 F.R[N - 2], (const double*)F.A[N - 1], F.R[N - 1], part, cur));
    else
      TK_TRY(ttm_last2_t<float>(h, (const float*)X, pre, I1, I2, (const float*)F.A[N - 2],
                                F.R[N - 2], (const float*)F.A[N - 1], F.R[N - 1], part, cur));
    int64_t P = pre;
    int64_t post = (int64_t)F.R[N - 2] * F.R[N - 1];
    for (int n = N - 3; n >= 0; --n) {
      const int64_t pr = P / F.I[n];
      double* nxt = (n == 0) ? y : (cur == buf0 ? buf1 : buf0);
      TK_TRY(ttm_small(h, cur, pr, post, F.A[n], F.is64, (int)F.I[n], F.R[n], 1, nxt));
      cur = nxt;
      P = pr;
      post *= F.R[n];
    }
    return TUCKER_OK;
  }
  int64_t P = (int64_t)(F.total / (uint64_t)F.I[N - 1]);
  double* cur = (N == 1) ? y : buf0;
  TK_TRY(ttm_last(h, X, F.is64, P, (int)F.I[N - 1], F.A[N - 1], F.R[N - 1], cur));
  int64_t post = F.R[N - 1];
  for (int n = N - 2; n >= 0; --n) {
    int64_t pre = P / F.I[n];
    double* nxt = (n == 0) ? y : (cur == buf0 ? buf1 : buf0);
    TK_TRY(ttm_small(h, cur, pre, post, F.A[n], F.is64, (int)F.I[n], F.R[n], 1, nxt));
    cur = nxt;
    P = pre;
    post *= F.R[n];
  }
  return TUCKER_OK;
}

// B = X x_{k != n} A^(k)T, laid out (prod_{k<n} R_k, I_n, prod_{k>n} R_k) in `out`.
// ylast: NULL, or X x_N A^(N)T already formed (used when n != N - 1: the chains
// of all modes but the last start with that product, which does not change
// until the last mode's update, so an ALS sweep forms it once).
tucker_status ttm_chain_except(tucker_handle* h, const FactorSet& F, const void* X, int n,
                               double* buf0, double* buf1, double* out, const double* ylast) {
  const int N = F.N;
  // shape tracked as dims[] with the current extent of each mode
  int64_t ext[TUCKER_MAX_ORDER];
  for (int k = 0; k < N; ++k) ext[k] = F.I[k];
  auto prod = [&](int a, int b) { int64_t p = 1; for (int k = a; k < b; ++k) p *= ext[k]; return p; };
  const double* cur = nullptr;
  double* bufs[2] = {buf0, buf1};
  int which = 0;
  int remaining = 0;
  for (int k = 0; k < N; ++k) if (k != n) ++remaining;
  if (remaining == 0) return fail(h, TUCKER_EINVAL, "order-1 ALS is not supported");
  // first contraction straight from X
  int first = (n != N - 1) ? N - 1 : N - 2;
  double* dst = (--remaining == 0) ? out : bufs[which];
  if (ylast && first == N - 1 && remaining > 0) {
    dst = const_cast<double*>(ylast);             // read only below: the next step writes elsewhere
  } else if (first == N - 1) {
    TK_TRY(ttm_last(h, X, F.is64, prod(0, N - 1), (int)F.I[N - 1], F.A[N - 1], F.R[N - 1], dst));
  } else {
    TK_TRY(ttm_mid(h, X, F.is64, prod(0, first), (int)F.I[first], prod(first + 1, N), F.A[first],
                   F.R[first], dst));
  }
  ext[first] = F.R[first];
  cur = dst;
  which ^= 1;
  for (int k = first - 1; k >= 0; --k) {
    if (k == n) continue;
    dst = (--remaining == 0) ? out : bufs[which];
    TK_TRY(ttm_small(h, cur, prod(0, k), prod(k + 1, N), F.A[k], F.is64, (int)F.I[k], F.R[k], 1, dst));
    ext[k] = F.R[k];
    cur = dst;
    which ^= 1;
  }
  return TUCKER_OK;
}

tucker_status kron_eig_core(tucker_handle* h, const FactorSet& F, double* const* V,
                            double* const* s, const double* y, double lambda, double* g) {
  EigArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  for (int n = 0; n < F.N; ++n) { a.R[n] = F.R[n]; a.V[n] = V[n]; a.s[n] = s[n]; }
  a.y = y; a.lambda = lambda; a.g = g; a.d = F.d;
  const size_t smem = (size_t)2 * F.d * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_kron_eig_core, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_COUNT(h);
  k_kron_eig_core<<<1, 1024, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// T = G x_1 A^(1) ... x_{N-1} A^(N-1)  (P x R_N rows, P = prod_{n<N} I_n)
tucker_status model_rows(tucker_handle* h, const FactorSet& F, const double* g, double* buf0,
                         double* buf1, double** T_out) {
  const int N = F.N;
  const double* cur = g;
  int64_t pre = 1;
  int64_t post = 1;
  for (int k = 1; k < N; ++k) post *= F.R[k];
  double* bufs[2] = {buf0, buf1};
  int which = 0;
  for (int n = 0; n < N - 1; ++n) {
    double* dst = bufs[which];
    TK_TRY(ttm_small(h, cur, pre, post, F.A[n], F.is64, (int)F.I[n], F.R[n], 0, dst));
    cur = dst;
    which ^= 1;
    pre *= F.I[n];
    post /= F.R[n + 1];
  }
  *T_out = const_cast<double*>(cur);
  return TUCKER_OK;
}

// ||X - X-hat(g)||^2 (dense or COO) in FP64 into *out (device).
tucker_status residual_sq(tucker_handle* h, const FactorSet& F, const tucker_tensor* X,
                          const double* g, double* buf0, double* buf1, double* partial,
                          int npartial, double* out) {
  double* T = nullptr;
  TK_TRY(model_rows(h, F, g, buf0, buf1, &T));
  const int N = F.N;
  const int I = (int)F.I[N - 1], R = F.R[N - 1];
  const int64_t P = (int64_t)(F.total / (uint64_t)I);
  int grid = npartial;
  if (X->dense) {
    const size_t smem = (size_t)I * R * 8;
    TK_CUDA(h, cudaFuncSetAttribute(k_residual_dense, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    TK_CUDA(h, launch_dep(h, k_residual_dense, grid, 256, smem, X->dense, F.is64, P, I,
                          (const double*)T, F.A[N - 1], R, partial));
  } else {
    TK_CUDA(h, launch_dep(h, k_residual_coo, grid, 256, 0, X->keys, X->vals, F.is64, X->nnz, I,
                          (const double*)T, F.A[N - 1], R, partial));
  }
  TK_CUDA(h, launch_dep(h, k_sum_partials, 1, 1024, 0, (const double*)partial, grid, out));
  return TUCKER_OK;
}

tucker_status sumsq(tucker_handle* h, const void* v, int is64, int64_t n, double* partial,
                    int npartial, double* out) {
  TK_CUDA(h, launch_dep(h, k_sumsq, npartial, 256, 0, v, is64, n, partial));
  TK_CUDA(h, launch_dep(h, k_sum_partials, 1, 1024, 0, (const double*)partial, npartial, out));
  return TUCKER_OK;
}

tucker_status tensor_sumsq(tucker_handle* h, const void* X, int is64, int64_t n, double* partial,
                           int npartial, double* out) {
  const int vec = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  TK_CUDA(h, launch_dep(h, k_tensor_sumsq, npartial, 256, 0, X, is64, vec, n, partial));
  TK_CUDA(h, launch_dep(h, k_sum_partials, 1, 1024, 0, (const double*)partial, npartial, out));
  return TUCKER_OK;
}

tucker_status kt_x_from_last(tucker_handle* h, const FactorSet& F, const double* B, double* y) {
  const int N = F.N, RN = F.R[N - 1];
  const int64_t pre = F.d / RN, IN = F.I[N - 1];
  const int64_t warps = pre * RN;
  TK_CUDA(h, launch_dep(h, k_kt_x_from_last, ceil_div(warps * 32, 256), 256, 0, B, pre, IN,
                        F.A[N - 1], F.is64, RN, y));
  return TUCKER_OK;
}

tucker_status kron_quad(tucker_handle* h, const FactorSet& F, double* const* gram, const double* g,
                        const double* y, double* out) {
  KronQuadArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  a.d = F.d;
  for (int n = 0; n < F.N; ++n) { a.R[n] = F.R[n]; a.gram[n] = gram[n]; }
  a.g = g;
  a.y = y;
  a.out = out;
  const size_t smem = 2 * (size_t)F.d * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_kron_quad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TK_COUNT(h);
  k_kron_quad<<<1, 1024, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// ------------------------------------------ whitening for the missing-data beta
// Row r of a symmetric d x d matrix M: y = (V_1 (x) ... (x) V_N)^T M[r, :]^T,
// stored as column r of `out` (so `out` = (M Vk)^T = Vk^T M).  Two passes give
// Vk^T M Vk.  With `scale` the second pass also adds lambda on the diagonal and
// divides by sqrt(D_c D_r), D = (x)_n ev_n + lambda: the matrix
//     D^-1/2 Vk^T (M + lambda I) Vk D^-1/2,
// whose eigenvalues are those of the pencil (M + lambda I, K^T K + lambda I)
// when K^T K = Vk diag((x)_n ev_n) Vk^T (the factor eigendecompositions).
struct RotArgs {
  int N, d;
  int R[TUCKER_MAX_ORDER];
  const double* V[TUCKER_MAX_ORDER];   // R x R, V[a][k]
  const double* ev[TUCKER_MAX_ORDER];  // R eigenvalues
  const double* in;
  double* out;
  double lambda;
  int scale;
};

__device__ __forceinline__ double kron_ev(const RotArgs& a, int t) {
  double ev = 1.0;
  for (int n = a.N - 1; n >= 0; --n) {
    ev *= a.ev[n][t % a.R[n]];
    t /= a.R[n];
  }
  return ev + a.lambda;
}

__global__ void __launch_bounds__(512) k_kron_rot_rows(RotArgs a) {
  extern __shared__ double zb[];
  double* z0 = zb;
  double* z1 = zb + a.d;
  const int r = blockIdx.x;
  for (int i = threadIdx.x; i < a.d; i += blockDim.x) z0[i] = a.in[(size_t)r * a.d + i];
  __syncthreads();
  int pre = 1;
  for (int n = 0; n < a.N; ++n) {               // z <- z x_n V_n^T
    const int R = a.R[n];
    const int post = a.d / (pre * R);
    for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
      const int q = t % post, k = (t / post) % R, p = t / (post * R);
      double acc = 0.0;
      for (int j = 0; j < R; ++j) acc = fma(z0[(p * R + j) * post + q], a.V[n][j * R + k], acc);
      z1[t] = acc;
    }
    __syncthreads();
    double* tmp = z0; z0 = z1; z1 = tmp;
    pre *= R;
  }
  const double dr = a.scale ? kron_ev(a, r) : 1.0;
  for (int c = threadIdx.x; c < a.d; c += blockDim.x) {
    double v = z0[c];
    if (a.scale) v = (v + (c == r ? a.lambda : 0.0)) / sqrt(kron_ev(a, c) * dr);
    a.out[(size_t)c * a.d + r] = v;
  }
}

tucker_status kron_whiten(tucker_handle* h, const FactorSet& F, double* const* V,
                          double* const* ev, double lambda, const double* M, double* tmp,
                          double* out) {
  if (F.d > 8192) return fail(h, TUCKER_ENOTSUP, "whitening of d = %d", F.d);
  RotArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  a.d = F.d;
  for (int n = 0; n < F.N; ++n) { a.R[n] = F.R[n]; a.V[n] = V[n]; a.ev[n] = ev[n]; }
  a.lambda = lambda;
  const size_t smem = (size_t)2 * F.d * sizeof(double);
  TK_CUDA(h, cudaFuncSetAttribute(k_kron_rot_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  a.in = M; a.out = tmp; a.scale = 0;
  TK_COUNT(h);
  k_kron_rot_rows<<<F.d, 512, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  a.in = tmp; a.out = out; a.scale = 1;
  TK_COUNT(h);
  k_kron_rot_rows<<<F.d, 512, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// x = y / ||y||, norm_out = ||y|| (one CTA; FP64; fixed summation order).
__global__ void __launch_bounds__(1024) k_vec_normalize(const double* y, int d, double* x,
                                                        double* norm_out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < d; i += blockDim.x) acc = fma(y[i], y[i], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const double nrm = sqrt(red[0]);
  for (int i = threadIdx.x; i < d; i += blockDim.x) x[i] = nrm > 0.0 ? y[i] / nrm : 0.0;
  if (threadIdx.x == 0) *norm_out = nrm;
}

tucker_status vec_normalize(tucker_handle* h, const double* y, int d, double* x, double* norm_out) {
  TK_COUNT(h);
  k_vec_normalize<<<1, 1024, 0, h->stream>>>(y, d, x, norm_out);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
