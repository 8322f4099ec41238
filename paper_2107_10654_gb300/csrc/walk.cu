// FP64 products with the implicit sampled rows of K, evaluated level by level
// along the sorted sample (used for the right-hand side h, the refinement
// residual and the adjoint).
//
// The sampled keys are sorted, so rows that share the leading indices
// (i_1, ..., i_n) are contiguous.  With k_u = a_1 (x) a_2 (x) ... (x) a_N
// (a_n = A^(n)[i_n(u)]) and g viewed as an R_1 x ... x R_N tensor:
//   dot:  V_1 = g x_1 a_1 (a table over i_1), V_n = V_{n-1} x_n a_n, z_u = V_N;
//         moving to the next row only the levels whose index changed are
//         recomputed (V_n has prod_{k>n} R_k entries);
//   axpy: W_N = c_u for one row; when the index at level n changes the level
//         accumulators are folded upwards, W_{n-1} += a_n (x) W_n, so every
//         run of rows with one i_1 yields W_1 = sum_u c_u a_2 (x) ... (x) a_N;
//         finally out = sum_{i_1} A^(1)[i_1] (x) W_1[i_1].
// Work is split into pieces: at most CH consecutive rows of one i_1 segment,
// one warp per piece, so every SM is busy whatever the number of leading
// indices.  A warp loads the indices (and coefficients) of 32 rows at once,
// one per lane, and broadcasts them row by row with shuffles.  Piece partial
// sums are combined in a fixed order, so the results are deterministic.
// The arithmetic is exact reassociation of sum_r k_u[r] g[r] and
// sum_u c_u k_u[r] in FP64.
#include <algorithm>

#include "common.cuh"

namespace tk {

constexpr int WK_WARPS = 8;                 // warps (pieces) per CTA
constexpr int WK_MIN_ROWS = 32;             // rows per piece, at least (one per lane)
constexpr int64_t WK_PIECE_TARGET = 16384;  // pieces are widened beyond this count
constexpr int WK_WARP_SMEM = 12 * 1024;     // axpy: bytes of shared memory per warp, at most
constexpr int WK_DOT_SMEM = 24 * 1024;      // dot: bytes of shared memory per warp, at most

// dot: V_1 of the piece (nvec vectors) and 32 lanes' factor rows
static __host__ __device__ size_t dot_warp_bytes(int L1, int fstore, int nvec) {
  return ((size_t)nvec * L1 + (size_t)32 * fstore) * 8;
}

struct WalkArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  int lsz[TUCKER_MAX_ORDER + 1];     // lsz[n] = prod_{k >= n} R_k (level-n vector size), lsz[N] = 1
  int lofs[TUCKER_MAX_ORDER + 1];    // axpy: offset of level n >= 1 in a warp's accumulators
  int lstore;                         // axpy: doubles of accumulators per warp
  int fofs[TUCKER_MAX_ORDER];        // dot: first column of mode n >= 2 in a lane's factor rows
  int fstore;                         // dot: factor entries per lane (sum of R_n, n >= 2)
  const double* A[TUCKER_MAX_ORDER];  // FP64 factors
  const float* A32[TUCKER_MAX_ORDER]; // FP32 factors (the FP32 walks)
  int d;
  int I1;
  int CH;
  const uint32_t* idx[TUCKER_MAX_ORDER];
  const int* seg_begin;               // [I1]
  const int* seg_end;                 // [I1]
  const int64_t* pcnt;                // [I1] pieces of each segment
  const int64_t* pstart;              // [I1] first piece of each segment
  const int64_t* npieces;             // [1]
  const int* p_i1;                    // [maxP]
  const int* p_u0;
  const int* p_u1;
  // dot
  const double* g1;
  const double* g2;                   // nullable
  double* z1;
  double* z2;
  double* V1;                         // [nvec][I1][lsz1]
  // axpy: c_u = coef * ca[u] * (cb ? cb[u] : 1)
  const double* ca;
  const double* cb;
  double coef;
  double* Wp;                          // [maxP][lsz1] piece partials
  double* W1;                          // [I1][lsz1]
};

__device__ __forceinline__ double fac(const WalkArgs& a, int n, uint32_t i, int r) {
  return __ldg(a.A[n] + (size_t)i * a.R[n] + r);
}

// Factor entry in the walk's arithmetic type T (FP64 copies, or the FP32 originals).
template <class T> __device__ __forceinline__ T fac_t(const WalkArgs& a, int n, uint32_t i, int r);
template <> __device__ __forceinline__ double fac_t<double>(const WalkArgs& a, int n, uint32_t i, int r) {
  return __ldg(a.A[n] + (size_t)i * a.R[n] + r);
}
template <> __device__ __forceinline__ float fac_t<float>(const WalkArgs& a, int n, uint32_t i, int r) {
  return __ldg(a.A32[n] + (size_t)i * a.R[n] + r);
}
template <class T> __device__ __forceinline__ const T* fac_base(const WalkArgs& a, int n);
template <> __device__ __forceinline__ const double* fac_base<double>(const WalkArgs& a, int n) { return a.A[n]; }
template <> __device__ __forceinline__ const float* fac_base<float>(const WalkArgs& a, int n) { return a.A32[n]; }

// Segment table: seg_begin[i1] / seg_end[i1] of the real rows (sorted keys).
__global__ void k_segments(const uint32_t* idx0, const int* n_rows, int* seg_begin, int* seg_end) {
  const int n = *n_rows;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const uint32_t v = idx0[u];
    if (u == 0 || idx0[u - 1] != v) seg_begin[v] = u;
    if (u == n - 1 || idx0[u + 1] != v) seg_end[v] = u + 1;
  }
}

__global__ void k_piece_count(const int* seg_begin, const int* seg_end, int I1, int CH,
                              int64_t* pcnt) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I1; i += gridDim.x * blockDim.x) {
    const int len = seg_end[i] - seg_begin[i];
    pcnt[i] = len > 0 ? (len + CH - 1) / CH : 0;
  }
}

__global__ void k_piece_fill(const int* seg_begin, const int* seg_end, int I1, int CH,
                             const int64_t* pcnt, const int64_t* pstart, int* p_i1, int* p_u0,
                             int* p_u1) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < I1; i += gridDim.x * blockDim.x) {
    const int b = seg_begin[i], e = seg_end[i];
    for (int64_t q = 0; q < pcnt[i]; ++q) {
      const int64_t p = pstart[i] + q;
      const int u0 = b + (int)q * CH;
      p_i1[p] = i;
      p_u0[p] = u0;
      p_u1[p] = min(e, u0 + CH);
    }
  }
}

// V_1[v][i1][j] = sum_{r_1} A^(1)[i1][r_1] g_v[r_1 * lsz1 + j] for the segments with rows,
// stored in the walk's arithmetic type T.
template <class T>
__global__ void k_walk_v1(WalkArgs a) {
  pdl_wait();
  const int L1 = a.lsz[1];
  const int nvec = a.g2 ? 2 : 1;
  T* V1 = reinterpret_cast<T*>(a.V1);
  const int64_t total = (int64_t)a.I1 * L1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = (int)(t / L1), j = (int)(t % L1);
    if (a.pcnt[i1] == 0) continue;
    for (int v = 0; v < nvec; ++v) {
      const double* g = v ? a.g2 : a.g1;
      T acc = T(0);
      for (int r = 0; r < a.R[0]; ++r)
        acc = fma(fac_t<T>(a, 0, (uint32_t)i1, r), (T)g[(size_t)r * L1 + j], acc);
      V1[((size_t)v * a.I1 + i1) * L1 + j] = acc;
    }
  }
}

// z = sum over the trailing modes L..N-1 of (x)_{l >= L} a_l[r_l] * V[r_L, ..., r_{N-1}]
// for this lane's row; F holds the lane's factor rows, entry (mode l, column r)
// at F[(fofs[l] + r) * 32 + lane].  Nested loops with runtime ranks; the
// innermost level is one FMA per element of V.
template <class T, int N, int L>
struct FlatDot {
  static __device__ __forceinline__ void run(const WalkArgs& a, const T* V1, const T* V2,
                                             bool two, const T* F, int lane, T* z1, T* z2) {
    T s1 = T(0), s2 = T(0);
    const int step = a.lsz[L + 1];
    for (int r = 0; r < a.R[L]; ++r) {
      T t1, t2;
      FlatDot<T, N, L + 1>::run(a, V1 + r * step, V2 + r * step, two, F, lane, &t1, &t2);
      const T f = F[(a.fofs[L] + r) * 32 + lane];
      s1 = fma(f, t1, s1);
      if (two) s2 = fma(f, t2, s2);
    }
    *z1 = s1;
    *z2 = s2;
  }
};
template <class T, int N>
struct FlatDot<T, N, N> {
  static __device__ __forceinline__ void run(const WalkArgs&, const T* V1, const T* V2, bool,
                                             const T*, int, T* z1, T* z2) {
    *z1 = V1[0];
    *z2 = V2[0];
  }
};

// z_u = k_u . g for the rows of one piece per warp, one row per lane: V_1 of
// the piece's i_1 (shared by its rows) is copied to shared memory, each lane
// stages its own factor rows of modes 2..N, and contracts them against V_1.
template <class T, int N>
__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_dot(WalkArgs a) {
  pdl_wait();
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * WK_WARPS + warp;
  if (p >= *a.npieces) return;                              // warp-uniform; no CTA barriers below
  const bool two = a.g2 != nullptr;
  const int nvec = two ? 2 : 1;
  const int L1 = a.lsz[1];
  T* V = reinterpret_cast<T*>(sm + (size_t)warp * (nvec * L1 + 32 * a.fstore));
  T* F = V + nvec * L1;
  const int i1 = a.p_i1[p], u0 = a.p_u0[p], u1 = a.p_u1[p];
  const T* V1 = reinterpret_cast<const T*>(a.V1);
  for (int v = 0; v < nvec; ++v) {
    const T* src = V1 + ((size_t)v * a.I1 + i1) * L1;
    for (int j = lane; j < L1; j += 32) V[v * L1 + j] = src[j];
  }
  const T* V2 = V + (two ? L1 : 0);
  for (int base = u0; base < u1; base += 32) {
    const int u = base + lane;
    const bool act = u < u1;
    __syncwarp();
    for (int n = 1; n < N; ++n) {
      const uint32_t i = act ? __ldg(a.idx[n] + u) : 0u;
      for (int r = 0; r < a.R[n]; ++r) F[(a.fofs[n] + r) * 32 + lane] = act ? fac_t<T>(a, n, i, r) : T(0);
    }
    __syncwarp();
    T z1, z2;
    FlatDot<T, N, 1>::run(a, V, V2, two, F, lane, &z1, &z2);
    if (act) {
      a.z1[u] = (double)z1;
      if (a.z2) a.z2[u] = (double)z2;
    }
  }
}

// k_walk_dot with two levels for wide V_1 (orders >= 3, lsz[2] a multiple of 32):
// the 32 rows of a batch share few values of i_2 (the key order), so for each
// distinct i_2 of the batch the warp forms V_2 = V_1 x_2 a_2(i_2) (lsz[2]
// entries) once in shared memory, and each lane contracts its row against its
// V_2 only: lsz[2] + ... instead of lsz[1] + lsz[2] + ... multiply-adds per row.
// A batch with more than WD_RUNS values of i_2 takes the one-level path.
constexpr int WD_RUNS = 4;

static __host__ __device__ size_t dot2_warp_bytes(int L1, int L2, int fstore, int nvec) {
  return dot_warp_bytes(L1, fstore, nvec) + (size_t)WD_RUNS * nvec * L2 * 8;
}

template <class T, int N>
__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_dot2(WalkArgs a) {
  pdl_wait();
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * WK_WARPS + warp;
  if (p >= *a.npieces) return;                              // warp-uniform; no CTA barriers below
  const bool two = a.g2 != nullptr;
  const int nvec = two ? 2 : 1;
  const int L1 = a.lsz[1], L2 = a.lsz[2], R1 = a.R[1];
  T* V = reinterpret_cast<T*>(sm + (size_t)warp * (dot2_warp_bytes(L1, L2, a.fstore, nvec) / 8));
  T* F = V + nvec * L1;
  T* W = F + 32 * a.fstore;                                 // [WD_RUNS][nvec][L2]
  const int i1 = a.p_i1[p], u0 = a.p_u0[p], u1 = a.p_u1[p];
  const T* V1 = reinterpret_cast<const T*>(a.V1);
  for (int v = 0; v < nvec; ++v) {
    const T* src = V1 + ((size_t)v * a.I1 + i1) * L1;
    for (int j = lane; j < L1; j += 32) V[v * L1 + j] = src[j];
  }
  const unsigned le = (2u << lane) - 1u;                    // lanes <= this lane
  for (int base = u0; base < u1; base += 32) {
    const int u = base + lane;
    const bool act = u < u1;
    __syncwarp();
    uint32_t ix[N];
#pragma unroll
    for (int n = 1; n < N; ++n) ix[n] = act ? __ldg(a.idx[n] + u) : 0u;
    for (int n = 1; n < N; ++n)
      for (int r = 0; r < a.R[n]; ++r)
        F[(a.fofs[n] + r) * 32 + lane] = act ? fac_t<T>(a, n, ix[n], r) : T(0);
    // runs of equal i_2 among the batch's active rows (sorted, so equal values are adjacent)
    const uint32_t up = __shfl_up_sync(0xffffffffu, ix[1], 1);
    const unsigned heads = __ballot_sync(0xffffffffu, act && (lane == 0 || up != ix[1]));
    const int nruns = __popc(heads);
    __syncwarp();
    T z1, z2;
    if (nruns <= WD_RUNS) {
      unsigned hm = heads;
      for (int h = 0; h < nruns; ++h, hm &= hm - 1u) {      // V_2 of run h
        const int hl = __ffs(hm) - 1;                       // lane of the run's first row
        const uint32_t i2 = __shfl_sync(0xffffffffu, ix[1], hl);
        const T* a2 = fac_base<T>(a, 1) + (size_t)i2 * R1;
        for (int v = 0; v < nvec; ++v)
          for (int q = lane; q < L2; q += 32) {
            T acc = T(0);
            for (int r = 0; r < R1; ++r) acc = fma(__ldg(a2 + r), V[v * L1 + r * L2 + q], acc);
            W[((size_t)h * nvec + v) * L2 + q] = acc;
          }
      }
      __syncwarp();
      const int run = __popc(heads & le) - 1;               // this lane's run (act lanes)
      const T* w1 = W + (size_t)(run < 0 ? 0 : run) * nvec * L2;
      FlatDot<T, N, 2>::run(a, w1, w1 + (two ? L2 : 0), two, F, lane, &z1, &z2);
    } else {
      FlatDot<T, N, 1>::run(a, V, V + (two ? L1 : 0), two, F, lane, &z1, &z2);
    }
    if (act) {
      a.z1[u] = (double)z1;
      if (a.z2) a.z2[u] = (double)z2;
    }
  }
}

template <int N>
__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_axpy(WalkArgs a) {
  pdl_wait();
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * WK_WARPS + warp;
  if (p >= *a.npieces) return;                              // warp-uniform
  double* wst = sm + (size_t)warp * a.lstore;               // W_1 .. W_{N-1} at lofs[n]
  const int u0 = a.p_u0[p], u1 = a.p_u1[p];
  for (int e = lane; e < a.lstore; e += 32) wst[e] = 0.0;
  __syncwarp();
  uint32_t prev[TUCKER_MAX_ORDER];
  double cprev = 0.0;
  bool have = false;
  // batches of 32 rows; after the last row one more step (j == cnt of the
  // final batch, or an empty batch at base == u1) flushes every level
  for (int base = u0; base <= u1; base += 32) {
    const int cnt = min(32, u1 - base);
    uint32_t mine[TUCKER_MAX_ORDER];
    double cm = 0.0;
    for (int n = 1; n < N; ++n) mine[n] = lane < cnt ? __ldg(a.idx[n] + base + lane) : 0u;
    if (lane < cnt) cm = a.coef * a.ca[base + lane] * (a.cb ? a.cb[base + lane] : 1.0);
    for (int j = 0; j <= cnt; ++j) {
      const bool last = (j == cnt);
      if (last && cnt == 32) break;                          // rows continue in the next batch
      uint32_t cur[TUCKER_MAX_ORDER];
      int lvl = 1;                                           // levels >= lvl are flushed
      double c = 0.0;
      if (!last) {
        for (int n = 1; n < N; ++n) cur[n] = __shfl_sync(0xffffffffu, mine[n], j);
        c = __shfl_sync(0xffffffffu, cm, j);
        lvl = N;
        for (int n = N - 1; n >= 1; --n)
          if (!have || cur[n] != prev[n]) lvl = n;
      }
      if (have) {
        // fold the previous row: W_{N-1} += c * a_N ; then W_{n-1} += a_n (x) W_n for n > lvl
        if (N >= 2) {
          double* WN1 = wst + a.lofs[N - 1];
          const int RN = a.R[N - 1];
          for (int r = lane; r < RN; r += 32) WN1[r] = fma(cprev, fac(a, N - 1, prev[N - 1], r), WN1[r]);
          __syncwarp();
          for (int n = N - 1; n > lvl; --n) {
            const int sz = a.lsz[n];
            double* lo = wst + a.lofs[n];
            double* up = wst + a.lofs[n - 1];
            const int Rm = a.R[n - 1];
            for (int e = lane; e < Rm * sz; e += 32) {
              const int r = e / sz, jj = e - r * sz;
              up[e] = fma(fac(a, n - 1, prev[n - 1], r), lo[jj], up[e]);
            }
            __syncwarp();
            for (int jj = lane; jj < sz; jj += 32) lo[jj] = 0.0;
            __syncwarp();
          }
        } else {
          if (lane == 0) wst[a.lofs[1]] += cprev;            // N == 1: W_1 is a scalar
          __syncwarp();
        }
      }
      if (last) break;
      cprev = c;
      for (int n = 1; n < N; ++n) prev[n] = cur[n];
      have = true;
    }
    if (cnt < 32) break;
  }
  const int L1 = a.lsz[1];
  double* out = a.Wp + (size_t)p * L1;
  for (int e = lane; e < L1; e += 32) out[e] = wst[a.lofs[1] + e];
}

// The same piece partials with the W_1 entries spread over the lanes (orders
// 2 .. 4 with lsz[1] <= 32 KE): lane l owns the entries e = l + 32 k and adds
// c_u * prod_{n >= 2} A^(n)[i_n(u)][r_n(e)] for every row of the piece, so the
// rows carry no dependence on one another and the factor loads of successive
// rows overlap (the level fold above waits on each row's loads in turn).
template <class T, int N, int KE>
__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_axpy_lanes(WalkArgs a) {
  pdl_wait();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * WK_WARPS + warp;
  if (p >= *a.npieces) return;                              // warp-uniform
  const int L1 = a.lsz[1];
  const int u0 = a.p_u0[p], u1 = a.p_u1[p];
  int col[KE][N - 1];                                       // r_n(e), n = 2 .. N
  T acc[KE];
  const bool shared_last = N >= 3 && 32 % a.R[N - 1] == 0;
#pragma unroll
  for (int k = 0; k < KE; ++k) {
    acc[k] = T(0);
    const int e = lane + 32 * k;
#pragma unroll
    for (int n = 1; n < N; ++n) col[k][n - 1] = e < L1 ? (e / a.lsz[n + 1]) % a.R[n] : 0;
  }
  for (int base = u0; base < u1; base += 32) {
    const int cnt = min(32, u1 - base);
    uint32_t mine[N];
    T cm = T(0);
#pragma unroll
    for (int n = 1; n < N; ++n) mine[n] = lane < cnt ? __ldg(a.idx[n] + base + lane) : 0u;
    if (lane < cnt) cm = (T)(a.coef * a.ca[base + lane] * (a.cb ? a.cb[base + lane] : 1.0));
    constexpr int UNROLL = KE >= 8 ? 1 : 4;                 // rows in flight, within the registers
    if (shared_last) {
      // R_N divides 32: every entry of a lane has r_N = lane mod R_N, so c_u a_N
      // is formed once per row
#pragma unroll UNROLL
      for (int j = 0; j < cnt; ++j) {
        const T c = __shfl_sync(0xffffffffu, cm, j);
        const T* row[N];
#pragma unroll
        for (int n = 1; n < N; ++n)
          row[n] = fac_base<T>(a, n) + (size_t)__shfl_sync(0xffffffffu, mine[n], j) * a.R[n];
        const T cl = N >= 3 ? c * __ldg(row[N - 1] + col[0][N - 2]) : c;
#pragma unroll
        for (int k = 0; k < KE; ++k) {
          T t = cl;
#pragma unroll
          for (int n = N - 2; n >= 2; --n) t *= __ldg(row[n] + col[k][n - 1]);
          acc[k] = fma(t, __ldg(row[1] + col[k][0]), acc[k]);
        }
      }
    } else {
#pragma unroll UNROLL
      for (int j = 0; j < cnt; ++j) {
        const T c = __shfl_sync(0xffffffffu, cm, j);
        const T* row[N];
#pragma unroll
        for (int n = 1; n < N; ++n)
          row[n] = fac_base<T>(a, n) + (size_t)__shfl_sync(0xffffffffu, mine[n], j) * a.R[n];
#pragma unroll
        for (int k = 0; k < KE; ++k) {
          T t = c;
#pragma unroll
          for (int n = N - 1; n >= 2; --n) t *= __ldg(row[n] + col[k][n - 1]);
          acc[k] = fma(t, __ldg(row[1] + col[k][0]), acc[k]);
        }
      }
    }
  }
  double* out = a.Wp + (size_t)p * L1;
#pragma unroll
  for (int k = 0; k < KE; ++k) {
    const int e = lane + 32 * k;
    if (e < L1) out[e] = (double)acc[k];
  }
}

// Two levels for wide W_1 (lsz[2] a multiple of 32, orders >= 3): along the sorted
// sample the rows of one segment come in runs of equal i_2, and
//   W_1 = sum_runs a_2(i_2) (x) W_2,  W_2 = sum_{u in run} c_u a_3 (x) ... (x) a_N,
// so a row adds into W_2 (lsz[2] entries) and a run folds W_2 into W_1 once:
// about lsz[2] instead of lsz[1] multiply-adds per row, where FP64 issues under
// two per clock per SM.  Lane l owns the W_2 entries q = l + 32 k2 and the W_1
// entries e = l + 32 k, whose q(e) = e mod lsz[2] = l + 32 (k mod KE2) and
// r_2(e) = k / KE2 are its own, so the fold reads no other lane's data.
template <class T, int N, int KE, int KE2>
__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_axpy_lanes2(WalkArgs a) {
  pdl_wait();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t p = (int64_t)blockIdx.x * WK_WARPS + warp;
  if (p >= *a.npieces) return;                              // warp-uniform
  const int L1 = a.lsz[1];
  const int u0 = a.p_u0[p], u1 = a.p_u1[p];
  int col[KE2][N - 2];                                      // r_n(q), n = 2 .. N - 1
#pragma unroll
  for (int k2 = 0; k2 < KE2; ++k2) {
    const int q = lane + 32 * k2;
#pragma unroll
    for (int n = 2; n < N; ++n) col[k2][n - 2] = (q / a.lsz[n + 1]) % a.R[n];
  }
  T acc[KE], w2[KE2];
#pragma unroll
  for (int k = 0; k < KE; ++k) acc[k] = T(0);
#pragma unroll
  for (int k2 = 0; k2 < KE2; ++k2) w2[k2] = T(0);
  const bool shared_last = N >= 4 && 32 % a.R[N - 1] == 0;
  uint32_t prev = 0;
  bool have = false;
  auto fold = [&](uint32_t i2) {
    const T* a2 = fac_base<T>(a, 1) + (size_t)i2 * a.R[1];
#pragma unroll
    for (int k = 0; k < KE; ++k) acc[k] = fma(__ldg(a2 + k / KE2), w2[k % KE2], acc[k]);
#pragma unroll
    for (int k2 = 0; k2 < KE2; ++k2) w2[k2] = T(0);
  };
  for (int base = u0; base < u1; base += 32) {
    const int cnt = min(32, u1 - base);
    uint32_t mine[N];
    T cm = T(0);
#pragma unroll
    for (int n = 1; n < N; ++n) mine[n] = lane < cnt ? __ldg(a.idx[n] + base + lane) : 0u;
    if (lane < cnt) cm = (T)(a.coef * a.ca[base + lane] * (a.cb ? a.cb[base + lane] : 1.0));
    for (int j = 0; j < cnt; ++j) {
      const uint32_t i2 = __shfl_sync(0xffffffffu, mine[1], j);
      if (have && i2 != prev) fold(prev);                   // warp-uniform
      prev = i2;
      have = true;
      const T c = __shfl_sync(0xffffffffu, cm, j);
      const T* row[N];
#pragma unroll
      for (int n = 2; n < N; ++n)
        row[n] = fac_base<T>(a, n) + (size_t)__shfl_sync(0xffffffffu, mine[n], j) * a.R[n];
      // the last mode's column of entry l + 32 k2 is the same for every k2 when
      // R_N divides 32: c_u a_N[r_N] is then formed once per row
      T cl = c;
      if (N >= 4 && shared_last) cl = c * __ldg(row[N - 1] + col[0][N - 3]);
#pragma unroll
      for (int k2 = 0; k2 < KE2; ++k2) {
        T t = cl;
#pragma unroll
        for (int n = N - 1; n >= 3; --n)
          if (!(n == N - 1 && shared_last)) t *= __ldg(row[n] + col[k2][n - 2]);
        w2[k2] = fma(t, __ldg(row[2] + col[k2][0]), w2[k2]);
      }
    }
  }
  if (have) fold(prev);
  double* out = a.Wp + (size_t)p * L1;
#pragma unroll
  for (int k = 0; k < KE; ++k) out[lane + 32 * k] = (double)acc[k];
}

// W1[i1][j] = sum of the piece partials of segment i1 (fixed order); 0 if empty.
__global__ void k_walk_reduce(WalkArgs a) {
  pdl_wait();
  const int L1 = a.lsz[1];
  const int64_t total = (int64_t)a.I1 * L1;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i1 = (int)(t / L1), j = (int)(t % L1);
    const int64_t p0 = a.pstart[i1], np = a.pcnt[i1];
    double s = 0.0;
    for (int64_t q = 0; q < np; ++q) s += a.Wp[(size_t)(p0 + q) * L1 + j];
    a.W1[t] = s;
  }
}

// out[r1 * lsz1 + j] = base - diag .* y + sum_{i1} A1[i1][r1] * W1[i1][j]
// (W1 is zero for i1 without rows).  One warp per output, lanes over i1, the
// lane partial sums combined by a fixed butterfly: deterministic.
__global__ void k_walk_expand(WalkArgs a, const double* base, const double* diag, const double* y,
                              double* out) {
  pdl_wait();
  const int lsz1 = a.lsz[1];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < a.d; t += nwarps) {
    const int r1 = t / lsz1, j = t % lsz1;
    double v = 0.0;
    for (int i1 = lane; i1 < a.I1; i1 += 32) {
      const double f = a.A32[0] ? (double)__ldg(a.A32[0] + (size_t)i1 * a.R[0] + r1)
                                : fac(a, 0, (uint32_t)i1, r1);
      v = fma(f, a.W1[(size_t)i1 * lsz1 + j], v);
    }
    v = warp_sum(v);
    if (lane == 0) {
      double o = base ? base[t] : 0.0;
      if (diag) o -= diag[t] * y[t];
      out[t] = o + v;
    }
  }
}

// The reduction and expansion in two wide launches.  k_walk_fold: CTA b owns
// the segments i1 in [b C, (b + 1) C), sums each segment's piece partials in a
// fixed order into shared memory (W_1 rows) and forms its share of the
// expansion, part[b][r1 lsz1 + j] = sum_{its i1} A1[i1][r1] W_1[i1][j].
// k_walk_sum: out[t] = base - diag .* y + sum_b part[b][t] in the order of b.
__global__ void __launch_bounds__(256) k_walk_fold(WalkArgs a, int chunk, double* part) {
  pdl_wait();
  extern __shared__ double wrow[];                  // chunk x lsz1, then chunk x R1 of A1
  const int L1 = a.lsz[1], R1 = a.R[0];
  const int i1a = blockIdx.x * chunk;
  const int nloc = min(chunk, a.I1 - i1a);
  double* a1 = wrow + (size_t)chunk * L1;
  for (int e = threadIdx.x; e < nloc * R1; e += blockDim.x) {
    const int q = e / R1, r = e - q * R1;
    a1[e] = a.A32[0] ? (double)__ldg(a.A32[0] + (size_t)(i1a + q) * R1 + r)
                     : fac(a, 0, (uint32_t)(i1a + q), r);
  }
  for (int e = threadIdx.x; e < nloc * L1; e += blockDim.x) {
    const int q = e / L1, j = e - q * L1;
    const int i1 = i1a + q;
    const int64_t p0 = a.pstart[i1], np = a.pcnt[i1];
    const double* src = a.Wp + (size_t)p0 * L1 + j;
    double s = 0.0;
    int64_t k = 0;
    for (; k + 4 <= np; k += 4) {                   // four loads in flight, summed in order
      const double v0 = src[(size_t)k * L1], v1 = src[(size_t)(k + 1) * L1];
      const double v2 = src[(size_t)(k + 2) * L1], v3 = src[(size_t)(k + 3) * L1];
      s += v0; s += v1; s += v2; s += v3;
    }
    for (; k < np; ++k) s += src[(size_t)k * L1];
    wrow[e] = s;
  }
  __syncthreads();
  double* out = part + (size_t)blockIdx.x * a.d;
  for (int t = threadIdx.x; t < a.d; t += blockDim.x) {
    const int r1 = t / L1, j = t - r1 * L1;
    double v = 0.0;
    for (int q = 0; q < nloc; ++q) v = fma(a1[q * R1 + r1], wrow[q * L1 + j], v);
    out[t] = v;
  }
}

// Eight threads per output: thread q of an output sums the partials b = q, q + 8,
// ... in order, and the eight sums are added by a fixed shuffle tree, so the
// result is deterministic; every partial load of a thread is in flight at once
// when nb <= 64.
__global__ void k_walk_sum(const double* part, int nb, int d, const double* base,
                           const double* diag, const double* y, double* out) {
  pdl_wait();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int t = (int)(gt >> 3), q = (int)(gt & 7);
  double v = 0.0;
  if (t < d) {
    int b = q;
    for (; b + 56 < nb; b += 64) {
      double x[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) x[k] = part[(size_t)(b + 8 * k) * d + t];
#pragma unroll
      for (int k = 0; k < 8; ++k) v += x[k];
    }
    for (; b < nb; b += 8) v += part[(size_t)b * d + t];
  }
  v += __shfl_xor_sync(0xffffffffu, v, 1);
  v += __shfl_xor_sync(0xffffffffu, v, 2);
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  if (t < d && q == 0) {
    double o = base ? base[t] : 0.0;
    if (diag) o -= diag[t] * y[t];
    out[t] = o + v;
  }
}

// ------------------------------------------------------------------ host side

struct WalkGeom {
  int64_t I1;
  int L1;
  int CH;
  int64_t maxP;
};

static WalkGeom walk_geom(int64_t I1, int d, int R1, int64_t cap, int sms) {
  WalkGeom g;
  g.I1 = I1;
  g.L1 = d / R1;
  const int64_t c = cap > 0 ? cap : 1;
  // about 32 pieces (warps) per SM, and no more than WK_PIECE_TARGET pieces
  int64_t want = (int64_t)sms * 32;
  if (want > WK_PIECE_TARGET) want = WK_PIECE_TARGET;
  if (want < 1) want = 1;
  const int64_t ch = (c + want - 1) / want;
  g.CH = (int)(ch < WK_MIN_ROWS ? WK_MIN_ROWS : ch);
  g.maxP = (c + g.CH - 1) / g.CH + (I1 < c ? I1 : c);
  return g;
}

// Scratch layout (doubles): seg_begin/seg_end (I1 ints each) | pcnt, pstart (I1 int64
// each) + npieces | p_i1, p_u0, p_u1 (maxP ints each) | W1 (I1 x L1) | V1 (2 x I1 x L1)
// or Wp (maxP x L1), whichever is larger (dot and axpy do not overlap).
struct WalkPtrs {
  int* seg_begin;
  int* seg_end;
  int64_t* pcnt;
  int64_t* pstart;
  int64_t* npieces;
  int* p_i1;
  int* p_u0;
  int* p_u1;
  double* W1;
  double* V1;
  double* Wp;
};

static size_t walk_carve(const WalkGeom& g, double* base, WalkPtrs* w) {
  size_t off = 0;
  auto take = [&](size_t doubles) {
    double* p = base ? base + off : nullptr;
    off += (doubles + 1) & ~size_t(1);                 // 16-byte aligned pieces
    return p;
  };
  double* sb = take((size_t)g.I1);                     // 2 * I1 ints
  double* pc = take((size_t)2 * g.I1 + 1);
  double* pi = take(((size_t)3 * g.maxP + 1) / 2);
  w->W1 = take((size_t)g.I1 * g.L1);
  const size_t v1 = (size_t)2 * g.I1 * g.L1, wp = (size_t)g.maxP * g.L1;
  double* big = take(v1 > wp ? v1 : wp);
  w->seg_begin = reinterpret_cast<int*>(sb);
  w->seg_end = w->seg_begin ? w->seg_begin + g.I1 : nullptr;
  w->pcnt = reinterpret_cast<int64_t*>(pc);
  w->pstart = w->pcnt ? w->pcnt + g.I1 : nullptr;
  w->npieces = w->pstart ? w->pstart + g.I1 : nullptr;
  w->p_i1 = reinterpret_cast<int*>(pi);
  w->p_u0 = w->p_i1 ? w->p_i1 + g.maxP : nullptr;
  w->p_u1 = w->p_u0 ? w->p_u0 + g.maxP : nullptr;
  w->V1 = big;
  w->Wp = big;
  return off + 64;
}

static void level_sizes(int N, const int* R, int* lsz, int* lofs, int* lstore, int* fofs,
                        int* fstore) {
  lsz[N] = 1;
  for (int n = N - 1; n >= 0; --n) lsz[n] = lsz[n + 1] * R[n];
  int off = 0;
  for (int n = 1; n <= N; ++n) { lofs[n] = off; off += lsz[n]; }
  *lstore = (off + 1) & ~1;
  off = 0;
  for (int n = 1; n < N; ++n) { fofs[n] = off; off += R[n]; }
  *fstore = off;
}

// Whether the level vectors of the walk fit in shared memory for these ranks.
bool walk_fits(int N, const int* R, int64_t I1) {
  int lsz[TUCKER_MAX_ORDER + 1], lofs[TUCKER_MAX_ORDER + 1], fofs[TUCKER_MAX_ORDER];
  int lstore, fstore;
  level_sizes(N, R, lsz, lofs, &lstore, fofs, &fstore);
  return (size_t)lstore * 8 <= (size_t)WK_WARP_SMEM &&
         dot_warp_bytes(lsz[1], fstore, 2) <= (size_t)WK_DOT_SMEM &&
         (double)I1 * lsz[1] <= double(1 << 26);
}

size_t walk_scratch_doubles(int64_t I1, int d, int R1, int64_t cap, int sms) {
  if ((double)I1 * (d / R1) > double(1 << 26)) return 64;    // level walk not used
  WalkPtrs w;
  return walk_carve(walk_geom(I1, d, R1, cap, sms), nullptr, &w);
}

static WalkArgs walk_args(const RowSet& s, const WalkGeom& g, const WalkPtrs& w) {
  WalkArgs a;
  memset(&a, 0, sizeof(a));
  a.N = s.N;
  a.d = s.d;
  a.I1 = (int)g.I1;
  a.CH = g.CH;
  for (int n = 0; n < s.N; ++n) {
    a.R[n] = s.R[n];
    a.A[n] = static_cast<const double*>(s.A[n]);
    a.idx[n] = s.idx[n];
  }
  level_sizes(s.N, s.R, a.lsz, a.lofs, &a.lstore, a.fofs, &a.fstore);
  a.seg_begin = w.seg_begin;
  a.seg_end = w.seg_end;
  a.pcnt = w.pcnt;
  a.pstart = w.pstart;
  a.npieces = w.npieces;
  a.p_i1 = w.p_i1;
  a.p_u0 = w.p_u0;
  a.p_u1 = w.p_u1;
  a.V1 = w.V1;
  a.Wp = w.Wp;
  a.W1 = w.W1;
  return a;
}

static int grid_for(tucker_handle* h, int64_t work, int threads) {
  int64_t g = (work + threads - 1) / threads;
  if (g > (int64_t)h->num_sms * 16) g = (int64_t)h->num_sms * 16;
  return (int)(g < 1 ? 1 : g);
}

using WalkKernel = void (*)(WalkArgs);

template <class T>
static WalkKernel walk_dot2_kernel_t(int N) {
  switch (N) {
    case 3: return k_walk_dot2<T, 3>;
    case 4: return k_walk_dot2<T, 4>;
    case 5: return k_walk_dot2<T, 5>;
    default: return nullptr;
  }
}

template <class T>
static WalkKernel walk_dot_kernel_t(int N) {
  switch (N) {
    case 1: return k_walk_dot<T, 1>;
    case 2: return k_walk_dot<T, 2>;
    case 3: return k_walk_dot<T, 3>;
    case 4: return k_walk_dot<T, 4>;
    case 5: return k_walk_dot<T, 5>;
    case 6: return k_walk_dot<T, 6>;
    case 7: return k_walk_dot<T, 7>;
    default: return k_walk_dot<T, 8>;
  }
}

static WalkKernel walk_axpy_kernel(int N) {
  switch (N) {
    case 1: return k_walk_axpy<1>;
    case 2: return k_walk_axpy<2>;
    case 3: return k_walk_axpy<3>;
    case 4: return k_walk_axpy<4>;
    case 5: return k_walk_axpy<5>;
    case 6: return k_walk_axpy<6>;
    case 7: return k_walk_axpy<7>;
    default: return k_walk_axpy<8>;
  }
}

// The lane-parallel axpy for orders 2 .. 4 and lsz[1] <= 512 (else nullptr).
template <class T, int N>
static WalkKernel axpy_lanes_by_width(int L1) {
  if (L1 <= 32) return k_walk_axpy_lanes<T, N, 1>;
  if (L1 <= 64) return k_walk_axpy_lanes<T, N, 2>;
  if (L1 <= 128) return k_walk_axpy_lanes<T, N, 4>;
  if (L1 <= 256) return k_walk_axpy_lanes<T, N, 8>;
  if (L1 <= 512) return k_walk_axpy_lanes<T, N, 16>;
  return nullptr;
}

template <class T>
static WalkKernel walk_axpy_lanes_kernel(int N, int L1) {
  switch (N) {
    case 2: return axpy_lanes_by_width<T, 2>(L1);
    case 3: return axpy_lanes_by_width<T, 3>(L1);
    case 4: return axpy_lanes_by_width<T, 4>(L1);
    default: return nullptr;
  }
}

// The two-level axpy for orders 3 and 4 with lsz[2] in {32, 64, 128} and
// lsz[1] <= 512 (else nullptr).
template <class T, int N, int KE2>
static WalkKernel axpy_lanes2_by_width(int L1) {
  if (L1 == 32 * KE2) return k_walk_axpy_lanes2<T, N, KE2, KE2>;
  if (L1 == 64 * KE2) return k_walk_axpy_lanes2<T, N, 2 * KE2, KE2>;
  if (L1 == 128 * KE2 && 4 * KE2 <= 16) return k_walk_axpy_lanes2<T, N, 4 * KE2, KE2>;
  if (L1 == 256 * KE2 && 8 * KE2 <= 16) return k_walk_axpy_lanes2<T, N, 8 * KE2, KE2>;
  if (L1 == 512 * KE2 && 16 * KE2 <= 16) return k_walk_axpy_lanes2<T, N, 16 * KE2, KE2>;
  return nullptr;
}

template <class T>
static WalkKernel walk_axpy_lanes2_kernel(int N, int L1, int L2) {
  if (L2 % 32 != 0 || L1 % L2 != 0) return nullptr;
  const int ke2 = L2 / 32;
  if (N == 3) {
    if (ke2 == 1) return axpy_lanes2_by_width<T, 3, 1>(L1);
    if (ke2 == 2) return axpy_lanes2_by_width<T, 3, 2>(L1);
    if (ke2 == 4) return axpy_lanes2_by_width<T, 3, 4>(L1);
  } else if (N == 4) {
    if (ke2 == 1) return axpy_lanes2_by_width<T, 4, 1>(L1);
    if (ke2 == 2) return axpy_lanes2_by_width<T, 4, 2>(L1);
    if (ke2 == 4) return axpy_lanes2_by_width<T, 4, 4>(L1);
  }
  return nullptr;
}

// One warp per piece: ceil(maxP / WK_WARPS) CTAs; warps past the piece count exit.
static tucker_status launch_by_order(tucker_handle* h, WalkKernel k, int64_t maxP, size_t smem,
                                     const WalkArgs& a) {
  TK_CUDA(h, cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  TK_CUDA(h, launch_dep(h, k, (int)((maxP + WK_WARPS - 1) / WK_WARPS), WK_WARPS * 32, smem, a));
  return TUCKER_OK;
}

// Build the segment and piece tables for a sample (once per sample set).
tucker_status walk_segments(tucker_handle* h, const RowSet& s, int64_t I1, const WalkBuf& wb) {
  if (!walk_fits(s.N, s.R, I1)) return TUCKER_OK;          // the per-element kernels are used
  const WalkGeom g = walk_geom(I1, s.d, s.R[0], wb.cap, h->num_sms);
  WalkPtrs w;
  walk_carve(g, wb.p, &w);
  TK_CUDA(h, cudaMemsetAsync(w.seg_begin, 0, sizeof(int) * 2 * I1, h->stream));
  TK_COUNT(h);
  k_segments<<<grid_for(h, wb.cap, 256), 256, 0, h->stream>>>(s.idx[0], s.n_rows, w.seg_begin,
                                                              w.seg_end);
  TK_LAUNCH(h);
  TK_CUDA(h, launch_dep(h, k_piece_count, grid_for(h, I1, 256), 256, 0, w.seg_begin, w.seg_end,
                        (int)I1, g.CH, w.pcnt));
  launch_scan_i64(h, w.pcnt, w.pstart, I1, w.npieces);
  TK_LAUNCH(h);
  TK_CUDA(h, launch_dep(h, k_piece_fill, grid_for(h, I1, 128), 128, 0, w.seg_begin, w.seg_end,
                        (int)I1, g.CH, w.pcnt, w.pstart, w.p_i1, w.p_u0, w.p_u1));
  return TUCKER_OK;
}

// Whether the FP32 walks apply to this sample: FP32 factors, orders 2-4, d / R_1 <= 512.
bool walk_f32_ok(const RowSet& s) {
  return !s.is64 && s.N >= 2 && s.N <= 4 && s.d / s.R[0] <= 512;
}

// z1[u] = k_u . g1, z2[u] = k_u . g2 (g2 nullable) for the real rows; with f32 the
// products and sums are FP32 (the FP32 factors of s), else FP64 (s holds FP64 factors).
tucker_status walk_dot(tucker_handle* h, const RowSet& s, int64_t I1, const WalkBuf& wb,
                       const double* g1, const double* g2, double* z1, double* z2, bool f32) {
  if (f32 ? !walk_f32_ok(s) : !s.is64)
    return fail(h, TUCKER_EINTERNAL, "walk needs FP64 factors (FP32 ones for the FP32 walk)");
  const WalkGeom g = walk_geom(I1, s.d, s.R[0], wb.cap, h->num_sms);
  WalkPtrs w;
  walk_carve(g, wb.p, &w);
  WalkArgs a = walk_args(s, g, w);
  a.g1 = g1; a.g2 = g2; a.z1 = z1; a.z2 = z2;
  const int nvec = g2 ? 2 : 1;
  size_t smem = (size_t)WK_WARPS * dot_warp_bytes(a.lsz[1], a.fstore, nvec);
  // two levels when the runs of equal (i_1, i_2) are long and V_2 is a whole number of warps
  const size_t smem2 = (size_t)WK_WARPS * dot2_warp_bytes(a.lsz[1], a.lsz[2], a.fstore, nvec);
  const bool lvl2 = s.N >= 3 && s.N <= 5 && a.lsz[2] % 32 == 0 && wb.I2 > 0 &&
                    (double)wb.cap >= 4.0 * (double)I1 * (double)wb.I2 && smem2 <= 200 * 1024;
  if (lvl2) smem = smem2;
  if (f32) {
    for (int n = 0; n < s.N; ++n) a.A32[n] = static_cast<const float*>(s.A[n]);
    TK_CUDA(h, launch_dep(h, k_walk_v1<float>, grid_for(h, I1 * a.lsz[1], 256), 256, 0, a));
    TK_TRY(launch_by_order(h, lvl2 ? walk_dot2_kernel_t<float>(s.N) : walk_dot_kernel_t<float>(s.N),
                           g.maxP, smem, a));
  } else {
    TK_CUDA(h, launch_dep(h, k_walk_v1<double>, grid_for(h, I1 * a.lsz[1], 256), 256, 0, a));
    TK_TRY(launch_by_order(h, lvl2 ? walk_dot2_kernel_t<double>(s.N) : walk_dot_kernel_t<double>(s.N),
                           g.maxP, smem, a));
  }
  return TUCKER_OK;
}

// out = base - diag .* y + coef * sum_u ca_u cb_u k_u  (real rows); f32 as for walk_dot
// (the piece partials, their sums and the expansion stay FP64).
tucker_status walk_axpy(tucker_handle* h, const RowSet& s, int64_t I1, const WalkBuf& wb,
                        const double* ca, const double* cb, double coef, const double* base,
                        const double* diag, const double* y, double* out, bool f32) {
  if (f32 ? !walk_f32_ok(s) : !s.is64)
    return fail(h, TUCKER_EINTERNAL, "walk needs FP64 factors (FP32 ones for the FP32 walk)");
  const WalkGeom g = walk_geom(I1, s.d, s.R[0], wb.cap, h->num_sms);
  WalkPtrs w;
  walk_carve(g, wb.p, &w);
  WalkArgs a = walk_args(s, g, w);
  a.ca = ca; a.cb = cb; a.coef = coef;
  if (f32) for (int n = 0; n < s.N; ++n) a.A32[n] = static_cast<const float*>(s.A[n]);
  WalkKernel lanes = f32 ? walk_axpy_lanes_kernel<float>(s.N, a.lsz[1])
                         : walk_axpy_lanes_kernel<double>(s.N, a.lsz[1]);
  // two levels when the runs of equal (i_1, i_2) are long enough to pay for their folds
  if (s.N >= 3 && wb.I2 > 0 && (double)wb.cap >= 4.0 * (double)I1 * (double)wb.I2) {
    WalkKernel two = f32 ? walk_axpy_lanes2_kernel<float>(s.N, a.lsz[1], a.lsz[2])
                         : walk_axpy_lanes2_kernel<double>(s.N, a.lsz[1], a.lsz[2]);
    if (two) lanes = two;
  }
  if (lanes) {
    TK_CUDA(h, launch_dep(h, lanes, (int)((g.maxP + WK_WARPS - 1) / WK_WARPS), WK_WARPS * 32, 0, a));
  } else {
    const size_t smem = (size_t)WK_WARPS * a.lstore * 8;
    TK_TRY(launch_by_order(h, walk_axpy_kernel(s.N), g.maxP, smem, a));
  }
  // segments per CTA of the fold: its partials (nb x d doubles) take the W_1 area
  // (I1 x lsz1 doubles), so nb <= I1 / R_1
  const int64_t nbmax = std::max<int64_t>(1, std::min<int64_t>(I1 / s.R[0], 2 * h->num_sms));
  const int chunk = (int)((I1 + nbmax - 1) / nbmax);
  const int nb = (int)((I1 + chunk - 1) / chunk);
  const size_t fsm = (size_t)chunk * (a.lsz[1] + s.R[0]) * sizeof(double);
  if (fsm <= 48 * 1024 && (size_t)nb * s.d <= (size_t)I1 * a.lsz[1]) {
    TK_CUDA(h, launch_dep(h, k_walk_fold, nb, 256, fsm, a, chunk, a.W1));
    TK_CUDA(h, launch_dep(h, k_walk_sum, ceil_div((int64_t)s.d * 8, 128), 128, 0, a.W1, nb, s.d, base,
                          diag, y, out));
    return TUCKER_OK;
  }
  TK_CUDA(h, launch_dep(h, k_walk_reduce, grid_for(h, I1 * a.lsz[1], 256), 256, 0, a));
  TK_CUDA(h, launch_dep(h, k_walk_expand, ceil_div(s.d, 8), 256, 0, a, base, diag, y, out));
  return TUCKER_OK;
}

}  // namespace tk
