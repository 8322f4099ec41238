// FP64 products with the implicit sampled rows of K, evaluated level by level
// along the sorted sample (used for the right-hand side h, the refinement
// residual and the adjoint).
//
// The sampled keys are sorted, so rows that share the leading indices
// (i_1, ..., i_n) are contiguous.  With k_u = a_1 (x) a_2 (x) ... (x) a_N
// (a_n = A^(n)[i_n(u)]) and g viewed as an R_1 x ... x R_N tensor:
//   dot:  V_1 = g x_1 a_1 (once per i_1 segment), V_n = V_{n-1} x_n a_n, z_u = V_N;
//         moving to the next row only the levels whose index changed are
//         recomputed (V_n has prod_{k>n} R_k entries);
//   axpy: W_N = c_u for one row; when the index at level n changes the level
//         accumulators are folded upwards, W_{n-1} += a_n (x) W_n, and each
//         i_1 segment yields W_1 = sum_u c_u a_2 (x) ... (x) a_N; finally
//         out = sum_{i_1} A^(1)[i_1] (x) W_1[i_1].
// One CTA per i_1 value; its 8 warps walk contiguous parts of the segment
// and are combined in a fixed order, so the results are deterministic.
// The arithmetic is exact reassociation of sum_r k_u[r] g[r] and
// sum_u c_u k_u[r] in FP64.
#include "common.cuh"

namespace tk {

constexpr int WK_WARPS = 8;

struct WalkArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  int lsz[TUCKER_MAX_ORDER + 1];     // lsz[n] = prod_{k >= n} R_k (level-n vector size), lsz[N] = 1
  int lofs[TUCKER_MAX_ORDER + 1];    // offset of level n (n >= 1) in a warp's level storage
  int lstore;                         // doubles of level storage per warp (one vector)
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  int d;
  const uint32_t* idx[TUCKER_MAX_ORDER];
  const int* seg_begin;               // [I_1]
  const int* seg_end;                 // [I_1]
  int I1;
  // dot
  const double* g1;
  const double* g2;                   // nullable
  double* z1;
  double* z2;
  // axpy: c_u = coef * ca[u] * (cb ? cb[u] : 1)
  const double* ca;
  const double* cb;
  double coef;
  double* W1;                          // [I_1][lsz[1]]
};

__device__ __forceinline__ double fac(const WalkArgs& a, int n, uint32_t i, int r) {
  return load_as_double(a.A[n], (int64_t)i * a.R[n] + r, a.is64);
}

// Segment table: seg_begin[i1] / seg_end[i1] of the real rows (sorted keys).
__global__ void k_segments(const uint32_t* idx0, const int* n_rows, int* seg_begin, int* seg_end) {
  const int n = *n_rows;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const uint32_t v = idx0[u];
    if (u == 0 || idx0[u - 1] != v) seg_begin[v] = u;
    if (u == n - 1 || idx0[u + 1] != v) seg_end[v] = u + 1;
  }
}

__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_dot(WalkArgs a) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nvec = a.g2 ? 2 : 1;
  double* V1 = sm;                                          // nvec x lsz[1]
  double* wst = sm + nvec * a.lsz[1] + warp * nvec * a.lstore;  // per-warp levels 2..N-1
  for (int i1 = blockIdx.x; i1 < a.I1; i1 += gridDim.x) {
    const int s0 = a.seg_begin[i1], s1 = a.seg_end[i1];
    if (s1 <= s0) continue;
    __syncthreads();
    // V_1 = g x_1 a_1
    for (int e = threadIdx.x; e < a.lsz[1]; e += blockDim.x) {
      double v1 = 0.0, v2 = 0.0;
      for (int r = 0; r < a.R[0]; ++r) {
        const double f = fac(a, 0, (uint32_t)i1, r);
        v1 = fma(f, a.g1[(size_t)r * a.lsz[1] + e], v1);
        if (a.g2) v2 = fma(f, a.g2[(size_t)r * a.lsz[1] + e], v2);
      }
      V1[e] = v1;
      if (a.g2) V1[a.lsz[1] + e] = v2;
    }
    __syncthreads();
    const int len = s1 - s0;
    const int per = (len + WK_WARPS - 1) / WK_WARPS;
    const int u0 = s0 + warp * per, u1 = min(s1, u0 + per);
    uint32_t prev[TUCKER_MAX_ORDER];
    for (int n = 0; n < a.N; ++n) prev[n] = 0xffffffffu;
    for (int u = u0; u < u1; ++u) {
      uint32_t cur[TUCKER_MAX_ORDER];
      int lvl = a.N;                                        // first changed level (1-based for n >= 1)
      for (int n = 0; n < a.N; ++n) cur[n] = a.idx[n][u];
      for (int n = a.N - 1; n >= 1; --n)
        if (cur[n] != prev[n]) lvl = n;
      if (prev[0] == 0xffffffffu) lvl = 1;
      // recompute V_{n+1} for n = lvl .. N-2 (levels stored per warp); level N handled last
      for (int n = lvl; n <= a.N - 2; ++n) {
        const int sz = a.lsz[n + 1];
        const double* src = (n == 1) ? V1 : wst + a.lofs[n];
        double* dst = wst + a.lofs[n + 1];
        for (int v = 0; v < nvec; ++v) {
          const double* s = src + (n == 1 ? v * a.lsz[1] : v * a.lstore);
          double* dd = dst + v * a.lstore;
          for (int j = lane; j < sz; j += 32) {
            double acc = 0.0;
            for (int r = 0; r < a.R[n]; ++r) acc = fma(fac(a, n, cur[n], r), s[(size_t)r * sz + j], acc);
            dd[j] = acc;
          }
        }
        __syncwarp();
      }
      // z = V_{N-1} . a_N   (V_{N-1} has R_N entries; for N == 1, V_1 is the scalar)
      double z1 = 0.0, z2 = 0.0;
      if (a.N == 1) {
        z1 = V1[0];
        if (a.g2) z2 = V1[1];
      } else {
        const double* src = (a.N == 2) ? V1 : wst + a.lofs[a.N - 1];
        const int RN = a.R[a.N - 1];
        for (int r = lane; r < RN; r += 32) {
          const double f = fac(a, a.N - 1, cur[a.N - 1], r);
          z1 = fma(f, src[r], z1);
          if (a.g2) z2 = fma(f, src[(a.N == 2 ? a.lsz[1] : a.lstore) + r], z2);
        }
        z1 = warp_sum(z1);
        if (a.g2) z2 = warp_sum(z2);
      }
      if (lane == 0) { a.z1[u] = z1; if (a.z2) a.z2[u] = z2; }
      for (int n = 0; n < a.N; ++n) prev[n] = cur[n];
      __syncwarp();
    }
  }
}

__global__ void __launch_bounds__(WK_WARPS * 32) k_walk_axpy(WalkArgs a) {
  extern __shared__ double sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per warp: accumulators W_1 .. W_{N-1} (level n has lsz[n] entries) at lofs[n]
  double* wst = sm + warp * a.lstore;
  double* Wsum = sm + WK_WARPS * a.lstore;                  // lsz[1]: combined W_1
  for (int i1 = blockIdx.x; i1 < a.I1; i1 += gridDim.x) {
    const int s0 = a.seg_begin[i1], s1 = a.seg_end[i1];
    if (s1 <= s0) continue;
    for (int e = lane; e < a.lstore; e += 32) wst[e] = 0.0;
    __syncwarp();
    const int len = s1 - s0;
    const int per = (len + WK_WARPS - 1) / WK_WARPS;
    const int u0 = s0 + warp * per, u1 = min(s1, u0 + per);
    uint32_t prev[TUCKER_MAX_ORDER];
    double cprev = 0.0;
    bool have = false;
    for (int u = u0; u <= u1; ++u) {
      uint32_t cur[TUCKER_MAX_ORDER];
      int lvl = 1;                                           // levels >= lvl are flushed
      const bool last = (u == u1);
      if (!last) {
        for (int n = 0; n < a.N; ++n) cur[n] = a.idx[n][u];
        lvl = a.N;
        for (int n = a.N - 1; n >= 1; --n)
          if (!have || cur[n] != prev[n]) lvl = n;
      }
      if (have) {
        // fold the previous row: W_{N-1} += c * a_N ; then W_{n-1} += a_n (x) W_n for n > lvl
        if (a.N >= 2) {
          double* WN1 = wst + a.lofs[a.N - 1];
          const int RN = a.R[a.N - 1];
          for (int r = lane; r < RN; r += 32) WN1[r] = fma(cprev, fac(a, a.N - 1, prev[a.N - 1], r), WN1[r]);
          __syncwarp();
          for (int n = a.N - 1; n > lvl; --n) {
            // W_{n-1}[r * lsz[n] + j] += a_{n-1}[r] * W_n[j]; W_n = 0
            const int sz = a.lsz[n];
            double* lo = wst + a.lofs[n];
            double* up = wst + a.lofs[n - 1];
            const int Rm = a.R[n - 1];
            for (int e = lane; e < Rm * sz; e += 32) {
              const int r = e / sz, j = e % sz;
              up[e] = fma(fac(a, n - 1, prev[n - 1], r), lo[j], up[e]);
            }
            __syncwarp();
            for (int j = lane; j < sz; j += 32) lo[j] = 0.0;
            __syncwarp();
          }
        } else {
          if (lane == 0) wst[a.lofs[1]] += cprev;            // N == 1: W_1 is a scalar
          __syncwarp();
        }
      }
      if (last) break;
      cprev = a.coef * a.ca[u] * (a.cb ? a.cb[u] : 1.0);
      for (int n = 0; n < a.N; ++n) prev[n] = cur[n];
      have = true;
    }
    // combine the warps' W_1 in a fixed order
    __syncthreads();
    for (int e = threadIdx.x; e < a.lsz[1]; e += blockDim.x) {
      double v = 0.0;
      for (int w = 0; w < WK_WARPS; ++w) v += sm[w * a.lstore + a.lofs[1] + e];
      a.W1[(size_t)i1 * a.lsz[1] + e] = v;
    }
    __syncthreads();
  }
}

// out[r1 * lsz1 + j] = base - diag .* y + sum_{i1} A1[i1][r1] * W1[i1][j]
// (W1 is zero for i1 without rows).  One warp per output, lanes over i1, the
// lane partial sums combined by a fixed butterfly: deterministic.
__global__ void k_walk_expand(WalkArgs a, const double* base, const double* diag, const double* y,
                              double* out) {
  const int lsz1 = a.lsz[1];
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t = warp; t < a.d; t += nwarps) {
    const int r1 = t / lsz1, j = t % lsz1;
    double v = 0.0;
    for (int i1 = lane; i1 < a.I1; i1 += 32)
      v = fma(fac(a, 0, (uint32_t)i1, r1), a.W1[(size_t)i1 * lsz1 + j], v);
    v = warp_sum(v);
    if (lane == 0) {
      double o = base ? base[t] : 0.0;
      if (diag) o -= diag[t] * y[t];
      out[t] = o + v;
    }
  }
}

// ------------------------------------------------------------------ host side

struct WalkPlan {
  WalkArgs a;
  size_t smem_dot, smem_axpy;
};

static WalkPlan walk_plan(const RowSet& s, int64_t I1, int* seg_begin, int* seg_end, double* W1) {
  WalkPlan p;
  memset(&p, 0, sizeof(p));
  WalkArgs& a = p.a;
  a.N = s.N;
  a.is64 = s.is64;
  a.d = s.d;
  a.I1 = (int)I1;
  for (int n = 0; n < s.N; ++n) { a.R[n] = s.R[n]; a.A[n] = s.A[n]; a.idx[n] = s.idx[n]; }
  a.lsz[s.N] = 1;
  for (int n = s.N - 1; n >= 0; --n) a.lsz[n] = a.lsz[n + 1] * s.R[n];
  int off = 0;
  for (int n = 1; n <= s.N; ++n) { a.lofs[n] = off; off += a.lsz[n]; }
  a.lstore = (off + 1) & ~1;
  a.seg_begin = seg_begin;
  a.seg_end = seg_end;
  a.W1 = W1;
  p.smem_dot = (size_t)(2 * a.lsz[1] + WK_WARPS * 2 * a.lstore) * sizeof(double);
  p.smem_axpy = (size_t)(WK_WARPS * a.lstore + a.lsz[1]) * sizeof(double);
  return p;
}

// Whether the level vectors of the walk fit in shared memory for these ranks.
bool walk_fits(int N, const int* R, int64_t I1) {
  int lsz[TUCKER_MAX_ORDER + 1];
  lsz[N] = 1;
  for (int n = N - 1; n >= 0; --n) lsz[n] = lsz[n + 1] * R[n];
  int store = 0;
  for (int n = 1; n <= N; ++n) store += lsz[n];
  store = (store + 1) & ~1;
  const size_t dot = (size_t)(2 * lsz[1] + WK_WARPS * 2 * store) * 8;
  const size_t axpy = (size_t)(WK_WARPS * store + lsz[1]) * 8;
  return dot <= 200 * 1024 && axpy <= 200 * 1024 && (double)I1 * lsz[1] <= double(1 << 27);
}

size_t walk_scratch_doubles(int64_t I1, int d, int R1) {
  const double n = (double)I1 * (d / R1);
  if (n > double(1 << 27)) return (size_t)2 * I1 + 64;      // level walk not used
  return (size_t)2 * I1 + (size_t)I1 * (d / R1) + 64;
}

// Build the segment table for a sample (once per sample set).
tucker_status walk_segments(tucker_handle* h, const RowSet& s, int64_t I1, int64_t cap,
                            double* scratch) {
  int* seg_begin = reinterpret_cast<int*>(scratch);
  int* seg_end = seg_begin + I1;
  TK_CUDA(h, cudaMemsetAsync(seg_begin, 0, sizeof(int) * 2 * I1, h->stream));
  int grid = ceil_div(cap, 256);
  if (grid > h->num_sms * 8) grid = h->num_sms * 8;
  if (grid < 1) grid = 1;
  TK_COUNT(h);
  k_segments<<<grid, 256, 0, h->stream>>>(s.idx[0], s.n_rows, seg_begin, seg_end);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

static WalkPlan plan_from_scratch(const RowSet& s, int64_t I1, double* scratch) {
  int* seg_begin = reinterpret_cast<int*>(scratch);
  int* seg_end = seg_begin + I1;
  double* W1 = scratch + I1 + 2;          // after 2*I1 ints (= I1 doubles), 16-byte aligned
  return walk_plan(s, I1, seg_begin, seg_end, W1);
}

static int walk_grid(tucker_handle* h, int64_t I1) {
  int64_t g = I1;
  if (g > (int64_t)h->num_sms * 8) g = (int64_t)h->num_sms * 8;
  return (int)(g < 1 ? 1 : g);
}

// z1[u] = k_u . g1, z2[u] = k_u . g2 (g2 nullable) for the real rows.
tucker_status walk_dot(tucker_handle* h, const RowSet& s, int64_t I1, double* scratch,
                       const double* g1, const double* g2, double* z1, double* z2) {
  WalkPlan p = plan_from_scratch(s, I1, scratch);
  p.a.g1 = g1; p.a.g2 = g2; p.a.z1 = z1; p.a.z2 = z2;
  TK_CUDA(h, cudaFuncSetAttribute(k_walk_dot, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)p.smem_dot));
  TK_COUNT(h);
  k_walk_dot<<<walk_grid(h, I1), WK_WARPS * 32, p.smem_dot, h->stream>>>(p.a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// out = base - diag .* y + coef * sum_u ca_u cb_u k_u  (real rows)
tucker_status walk_axpy(tucker_handle* h, const RowSet& s, int64_t I1, double* scratch,
                        const double* ca, const double* cb, double coef, const double* base,
                        const double* diag, const double* y, double* out) {
  WalkPlan p = plan_from_scratch(s, I1, scratch);
  p.a.ca = ca; p.a.cb = cb; p.a.coef = coef;
  TK_CUDA(h, cudaMemsetAsync(p.a.W1, 0, sizeof(double) * (size_t)I1 * p.a.lsz[1], h->stream));
  TK_CUDA(h, cudaFuncSetAttribute(k_walk_axpy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)p.smem_axpy));
  TK_COUNT(h);
  k_walk_axpy<<<walk_grid(h, I1), WK_WARPS * 32, p.smem_axpy, h->stream>>>(p.a);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_walk_expand<<<ceil_div(s.d, 8), 256, 0, h->stream>>>(p.a, base, diag, y, out);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
