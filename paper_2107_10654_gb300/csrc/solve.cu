// Ridge solve of the (sketched or exact) normal equations (Eq. problem_def;
// Appendix B, proof of Thm 4.2): M = G + diag(regdiag), M = L L^T by a blocked
// right-looking Cholesky, then L y = h and L^T g = y.
//
// The factorisation and the triangular solves are templated on the element
// type: FP64 (the FP64 Cholesky solver) or FP32 (the mixed solver, where the
// FP32 factor only preconditions an FP64 iterative refinement; see api.cu).
//
// Cholesky: one persistent cooperative launch (one CTA per SM, grid-wide
// barriers between phases).  Step k (panel width CB):
//   phase 1: every CTA factors the CB x CB diagonal block in shared memory
//            (the same arithmetic in every CTA, so all agree on a failed
//            pivot and leave together); CTA 0 stores L_kk; each warp solves
//            one panel row  L_ik = A_ik L_kk^-T;
//   phase 2: lower trailing tiles A_ij -= L_ik L_jk^T (CT x CT), distributed
//            over the CTAs.
// A non-positive or NaN pivot records TUCKER_ENOTSPD (no trap, no hang).
// L overwrites the lower triangle of M (row-major, d x d).
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace tk {

constexpr int CB = 32;      // panel width
constexpr int SB = 64;      // block of the triangular solves
constexpr int CHOL_THREADS = 128;   // one warp per SM sub-partition: enough for the FP64 pipe
constexpr int CHOL_CL_MAX_D = 1024; // largest order factored by one cluster (if it fits)

__global__ void k_add_diag(double* M, int d, const double* diag) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
    M[(size_t)i * d + i] += diag[i];
}

// regdiag[j] = lambda (exact) or lambda * D[j] (augmented)
__global__ void k_regdiag(double* out, int d, double lambda, const double* D) {
  pdl_wait();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x)
    out[i] = D ? lambda * D[i] : lambda;
}

__global__ void k_to_f32(const double* in, size_t n, float* out) {
  pdl_wait();
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// 1/sqrt(p) of a pivot p > 0 (CUDA's rsqrt of the element type).
__device__ __forceinline__ double rsqrt_piv(double p) { return rsqrt(p); }
__device__ __forceinline__ float rsqrt_piv(float p) { return rsqrtf(p); }

template <class T> __device__ __forceinline__ T tmax();
template <> __device__ __forceinline__ double tmax<double>() { return 1.7976931348623157e308; }
template <> __device__ __forceinline__ float tmax<float>() { return 3.402823466e38f; }

template <class T>
__device__ __forceinline__ bool pivot_ok(T p) { return p > T(0) && p <= tmax<T>(); }

// Factor the nb x nb diagonal block at (k, k) in shared memory (all threads
// of the CTA).  Right-looking, one barrier per pivot: in phase j the scaled
// column l_ij = a_ij y_j (y_j = p_j^-1/2) is written to the unused upper
// triangle a[j][i] while the trailing entries are updated from the unscaled
// column, a_ic -= (a_ij r_j) a_cj with r_j = y_j^2.  Warp 0 updates the next
// diagonal entry and computes its y while the other warps update the rest, so
// the square-root chain overlaps the update (and no warp serialises both).  Returns false (in every thread) on a pivot that is
// not positive and finite; every CTA computes the same.
template <class T>
__device__ bool factor_diag_block(const T* M, int d, int k, int nb, T (*a)[CB + 1],
                                  const uint16_t* tri, T (*P)[CB + 1] = nullptr, int np = 0,
                                  int prow0 = 0, int pstride = 1) {
  __shared__ T ys[CB + 1], rs[CB + 1];
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < CB * CB; e += blockDim.x) {
    const int i = e / CB, j = e % CB;
    a[i][j] = (i < nb && j <= i) ? M[(size_t)(k + i) * d + k + j] : T(0);
  }
  // this CTA's panel rows prow0 + q * pstride (q < np), columns k .. k + nb
  for (int e = tid; e < np * CB; e += blockDim.x) {
    const int q = e / CB, j = e % CB;
    P[q][j] = j < nb ? M[(size_t)(prow0 + q * pstride) * d + k + j] : T(0);
  }
  __syncthreads();
  if (tid == 0) {
    const T p = a[0][0];
    bad = !pivot_ok(p);
    if (!bad) { ys[0] = rsqrt_piv(p); rs[0] = ys[0] * ys[0]; }
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    if (bad) return false;                          // read after a barrier: uniform
    const T y = ys[j], r = rs[j];
    const int m = nb - 1 - j;                       // trailing size
    if (tid < 32) {
      // warp 0: the pivot chain, computed redundantly by its lanes (no divergence
      // with the update below), stored by lane 0
      const T ajj = a[j][j];
      T v = T(0), yn = T(0);
      bool ok = true;
      if (m > 0) {
        const T l = a[j + 1][j];
        v = fma(-(l * r), l, a[j + 1][j + 1]);
        ok = pivot_ok(v);
        if (ok) yn = rsqrt_piv(v);
      }
      if (tid == 0) {
        a[j][j] = ajj * y;                          // l_jj = p_j / sqrt(p_j)
        if (m > 0) {
          a[j + 1][j + 1] = v;
          if (!ok) {
            bad = 1;
          } else {
            ys[j + 1] = yn;
            rs[j + 1] = yn * yn;
          }
        }
      }
    } else {
      const int t = tid - 32, nt = blockDim.x - 32;
      // scaled column into the upper triangle: a[j][j + 1 + q] = l_{j+1+q, j}
      for (int q = t; q < m; q += nt) a[j][j + 1 + q] = a[j + 1 + q][j] * y;
      // trailing entries except (j+1, j+1): packed index e -> (ii, cc), cc <= ii < m
      const int cnt = m * (m + 1) / 2;
      for (int e = 1 + t; e < cnt; e += nt) {
        const uint32_t ic = tri[e];
        const int i = j + 1 + (int)(ic >> 8), c = j + 1 + (int)(ic & 0xffu);
        a[i][c] = fma(-(a[i][j] * r), a[c][j], a[i][c]);
      }
      // the panel rows take the same rank-1 update (their column j stays unscaled)
      if (m > 0)
        for (int e = t; e < np * m; e += nt) {
          const int q = e / m, c = j + 1 + (e - q * m);
          P[q][c] = fma(-(P[q][j] * r), a[c][j], P[q][c]);
        }
    }
    __syncthreads();
  }
  // panel rows: l_qj = p_qj y_j
  for (int e = tid; e < np * nb; e += blockDim.x) {
    const int q = e / nb, j = e % nb;
    P[q][j] *= ys[j];
  }
  // move the scaled columns from the upper to the lower triangle
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j < i) a[i][j] = a[j][i];
  }
  __syncthreads();
  return true;
}

// A_ij -= L_ik L_jk^T over the lower TS x TS tiles of the trailing matrix
// (rows and columns >= s), tiles distributed over the CTAs.  The panel rows and
// the entries of a CTA's next tile are loaded into registers while the current
// tile is multiplied.  Thread (ty, tx) owns rows ty + 16 i and columns tx + 8 j.
template <class T, int TS>
__device__ void trailing_update(T* M, int d, int k, int nb, int s, T (*Pa)[CB + 1],
                                T (*Pb)[CB + 1]) {
  constexpr int PER = TS * CB / CHOL_THREADS;   // panel elements per thread and operand
  constexpr int OR = TS / 16, OC = TS / 8;      // outputs per thread
  const int Tt = (d - s + TS - 1) / TS;
  const int ntiles = Tt * (Tt + 1) / 2;
  const int tx = threadIdx.x & 7, ty = threadIdx.x >> 3;
  auto origin = [&](int tile, int* r0, int* c0) {
    // lower tiles in row-major packed order: tile = ti (ti + 1) / 2 + tj
    int ti = (int)((sqrtf(8.0f * tile + 1.0f) - 1.0f) * 0.5f);
    while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
    while (ti * (ti + 1) / 2 > tile) --ti;
    *r0 = s + ti * TS;
    *c0 = s + (tile - ti * (ti + 1) / 2) * TS;
  };
  T ra[PER], rb[PER];
  T cn[OR][OC];                                 // the next tile's entries of this thread
  auto fetch = [&](int tile) {
    int r0, c0;
    origin(tile, &r0, &c0);
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * CHOL_THREADS, i = e / CB, c = e % CB;
      ra[q] = (r0 + i < d && c < nb) ? M[(size_t)(r0 + i) * d + k + c] : T(0);
      rb[q] = (c0 + i < d && c < nb) ? M[(size_t)(c0 + i) * d + k + c] : T(0);
    }
#pragma unroll
    for (int i = 0; i < OR; ++i) {
      const int r = r0 + ty + 16 * i;
#pragma unroll
      for (int j = 0; j < OC; ++j) {
        const int c = c0 + tx + 8 * j;
        cn[i][j] = (r < d && c < d && c <= r) ? M[(size_t)r * d + c] : T(0);
      }
    }
  };
  if ((int)blockIdx.x < ntiles) fetch(blockIdx.x);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int r0, c0;
    origin(tile, &r0, &c0);
    __syncthreads();                            // the previous tile's reads are done
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int e = threadIdx.x + q * CHOL_THREADS;
      Pa[e / CB][e % CB] = ra[q];
      Pb[e / CB][e % CB] = rb[q];
    }
    T acc[OR][OC];
#pragma unroll
    for (int i = 0; i < OR; ++i)
#pragma unroll
      for (int j = 0; j < OC; ++j) acc[i][j] = cn[i][j];
    __syncthreads();
    if (tile + (int)gridDim.x < ntiles) fetch(tile + gridDim.x);
#pragma unroll 4
    for (int c = 0; c < CB; ++c) {
      T av[OR], bv[OC];
#pragma unroll
      for (int i = 0; i < OR; ++i) av[i] = Pa[ty + 16 * i][c];
#pragma unroll
      for (int j = 0; j < OC; ++j) bv[j] = Pb[tx + 8 * j][c];
#pragma unroll
      for (int i = 0; i < OR; ++i)
#pragma unroll
        for (int j = 0; j < OC; ++j) acc[i][j] = fma(-av[i], bv[j], acc[i][j]);
    }
#pragma unroll
    for (int i = 0; i < OR; ++i) {
      const int r = r0 + ty + 16 * i;
      if (r >= d) continue;
#pragma unroll
      for (int j = 0; j < OC; ++j) {
        const int c = c0 + tx + 8 * j;
        if (c < d && c <= r) M[(size_t)r * d + c] = acc[i][j];
      }
    }
  }
}

// Blocked right-looking Cholesky.  Step k: every CTA factors the diagonal
// block redundantly and, in the same pivot loop, its share of the panel rows
// below it (rows s + cta, s + cta + G, ...); CTA 0 stores L_kk, every CTA its
// panel rows; grid barrier; the trailing tiles; grid barrier.
template <class T>
__global__ void __launch_bounds__(CHOL_THREADS) k_chol_coop(T* M, int d, int* status) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) unsigned char chol_smem[];
  T (*P)[CB + 1] = reinterpret_cast<T (*)[CB + 1]>(chol_smem);     // panel rows of this CTA
  __shared__ T Lkk[CB][CB + 1];
  constexpr int TSMAX = sizeof(T) == 4 ? 64 : 32;  // FP32 uses 64 x 64 tiles while they last
  __shared__ T Pa[TSMAX][CB + 1];
  __shared__ T Pb[TSMAX][CB + 1];
  __shared__ uint16_t tri[CB * (CB - 1) / 2 + CB];
  const int G = gridDim.x, cta = blockIdx.x;
  // packed trailing-triangle table: entry e = ii (ii + 1) / 2 + cc
  for (int ii = threadIdx.x; ii < CB; ii += blockDim.x)
    for (int cc = 0; cc <= ii; ++cc) tri[ii * (ii + 1) / 2 + cc] = (uint16_t)((ii << 8) | cc);
  __syncthreads();
  for (int k = 0; k < d; k += CB) {
    const int nb = min(CB, d - k);
    const int s = k + nb;
    const int np = s + cta < d ? (d - s - cta + G - 1) / G : 0;
    if (!factor_diag_block<T>(M, d, k, nb, Lkk, tri, P, np, s + cta, G)) {
      if (cta == 0 && threadIdx.x == 0) set_status(status, DEV_NOTSPD);
      return;                                   // every CTA takes this branch at the same k
    }
    if (cta == 0)
      for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e % nb;
        if (j <= i) M[(size_t)(k + i) * d + k + j] = Lkk[i][j];
      }
    for (int e = threadIdx.x; e < np * nb; e += blockDim.x) {
      const int q = e / nb, j = e % nb;
      M[(size_t)(s + cta + q * G) * d + k + j] = P[q][j];
    }
    grid.sync();
    if (s < d) {
      // the largest tiles that still give every CTA at least two
      const int t64 = (d - s + 63) / 64, t32 = (d - s + 31) / 32;
      if (TSMAX == 64 && t64 * (t64 + 1) / 2 >= 2 * G)
        trailing_update<T, TSMAX>(M, d, k, nb, s, Pa, Pb);
      else if (t32 * (t32 + 1) / 2 >= 2 * G)
        trailing_update<T, 32>(M, d, k, nb, s, Pa, Pb);
      else
        trailing_update<T, 16>(M, d, k, nb, s, Pa, Pb);
    }
    grid.sync();
  }
}

// dynamic shared memory of k_chol_coop: the largest panel share of a CTA
template <class T>
size_t chol_panel_smem(int d, int G) {
  const int rows = d > CB ? (d - CB + G - 1) / G : 0;
  return (size_t)(rows > 0 ? rows : 1) * (CB + 1) * sizeof(T);
}

static int coop_grid(tucker_handle* h, const void* kernel, int threads, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return h->num_sms;                         // one CTA per SM
}

template <class T>
tucker_status cholesky_t(tucker_handle* h, T* M, int d) {
  const void* kern = (const void*)k_chol_coop<T>;
  const size_t smem = chol_panel_smem<T>(d, h->num_sms);
  if (smem > 160 * 1024) return fail(h, TUCKER_ENOTSUP, "Cholesky panel of d = %d too large", d);
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = coop_grid(h, kern, CHOL_THREADS, smem);
  if (grid < 1) return fail(h, TUCKER_ECUDA, "cooperative Cholesky cannot be resident");
  void* args[] = {&M, &d, &h->d_status};
  TK_COUNT(h);
  TK_CUDA(h, cudaLaunchCooperativeKernel(kern, grid, CHOL_THREADS, args, smem, h->stream));
  return TUCKER_OK;
}

tucker_status cholesky(tucker_handle* h, double* M, int d) { return cholesky_t<double>(h, M, d); }
// ------------------------------------------------ FP32 Cholesky on one cluster
// For small d the FP32 factor of the mixed solver is computed by a single
// thread-block cluster (16 CTAs where the device allows that size, else 8)
// with the whole matrix resident in the CTAs' shared memory: CTA c owns rows
// c, c + C, c + 2C, ...  Data moves between CTAs only by stores into the
// receivers' shared memory (a remote store does not wait for a round trip),
// ordered by cluster barriers.  Step k (columns k0 .. k0 + 31):
//   1. warp 0 factors the 32 x 32 diagonal block in registers, four pivots per
//      round (lane i holds row i; every lane factors the round's 4 x 4 block,
//      then the round's columns go through shared memory with a release flag),
//      and the other warps apply each published round to this CTA's rows below
//      the block, giving the panel rows L_ik = A_ik L_kk^-T;
//   2. every CTA stores its panel rows into every CTA's panel buffer; cluster
//      barrier;
//   3. each CTA updates its own rows' trailing entries A_ic -= L_i . L_c
//      (4 rows x 4 columns per thread, 8 threads per 32-column chunk), then
//      stores its rows of the next diagonal block into every CTA; cluster
//      barrier.
// With X requested the kernel also forms X = L^-1 (the mixed solver applies
// (L L^T)^-1 as X^T X): CTA c owns columns c, c + C, ... of B = I, and at step k
// X_k = L_kk^-1 B_k (block row k, the same round-by-round substitution as the
// panel rows, run by the same warps) and then B_i -= L_ik X_k for i below the
// block, with the panel rows L_ik already in every CTA's panel buffer: the
// inverse needs no data beyond what the factorisation moves.
// Every CTA factors the same block with the same instructions, so all agree
// on a failed pivot and leave at the same step (no remote store follows).
constexpr int CLB = 32;
constexpr int CLPS = 36;                 // row stride of the panel and block buffers (floats)
constexpr int CHOL_CL_THREADS = 256;
constexpr size_t CHOL_CL_SMEM_MAX = 227 * 1024;   // the opt-in limit per CTA

struct ClGeom {
  int nr;      // own rows (and own columns of X) per CTA, at most
  int ld;      // own-row stride in floats: 4 x odd, so 8 lanes' 16-byte row loads hit distinct banks
  int xld;     // own-column stride of X in floats: odd, so 32 lanes' column reads hit distinct banks
  size_t smem;
};

__host__ __device__ inline ClGeom chol_cl_geom(int d, int C, bool inv) {
  ClGeom g;
  g.nr = (d + C - 1) / C;
  g.ld = 4 * (((d + 3) / 4) | 1);
  g.xld = d | 1;
  g.smem = sizeof(float) * ((size_t)g.nr * g.ld + (size_t)d * CLPS + (size_t)CLB * CLPS +
                            (size_t)CLB * CLB + (CLB / 4) * 12 +
                            (inv ? (size_t)g.nr * CLB + (size_t)g.nr * g.xld : 0));
  return g;
}

// 1/sqrt(p) by the SFU's approximate reciprocal square root (flushes subnormals,
// so pivots below the smallest normal float are rejected first).
__device__ __forceinline__ float rsqrt_approx(float p) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(p));
  return y;
}
__device__ __forceinline__ bool pivot_ok32(float p) {
  return p >= 1.17549435e-38f && p <= 3.402823466e38f;
}

__device__ __forceinline__ void st_release_cta(int* p, int v) {
  asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)),
               "r"(v) : "memory");
}
__device__ __forceinline__ int ld_acquire_cta(const int* p) {
  int v;
  asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v)
               : "r"((unsigned)__cvta_generic_to_shared(p)) : "memory");
  return v;
}

__global__ void __launch_bounds__(CHOL_CL_THREADS, 1) k_chol32_cluster(float* M, int d, int* status,
                                                                     float* X, float* XC) {
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), me = (int)cl.block_rank();
  const bool inv = X != nullptr;
  const ClGeom G = chol_cl_geom(d, C, inv);
  extern __shared__ __align__(16) float cls[];
  float* rows = cls;                                  // own row t = global row me + t C
  float* Pb = rows + (size_t)G.nr * G.ld;             // panel row c at (c - s) * CLPS
  float* Db = Pb + (size_t)d * CLPS;                  // diagonal block row i at i * CLPS
  float4* colb = reinterpret_cast<float4*>(Db + CLB * CLPS);  // round r: the rows' 4 L entries
  float* rbuf = reinterpret_cast<float*>(colb + (CLB / 4) * CLB);  // round r: its 4 x 4 block
  float* Xk = rbuf + (CLB / 4) * 12;                  // own column tc of X_k at tc * CLB
  float* Xc = Xk + (size_t)G.nr * CLB;                // own column tc (global me + tc C) of B, then X
  __shared__ int flag, bad_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  const int nown = d > me ? (d - me + C - 1) / C : 0;
  for (int t = warp; t < nown; t += nw) {
    const int i = me + t * C;
    for (int c = lane; c <= i; c += 32) rows[(size_t)t * G.ld + c] = M[(size_t)i * d + c];
  }
  if (tid == 0) { flag = 0; bad_s = 0; }
  if (inv)
    for (int e = tid; e < nown * G.xld; e += blockDim.x) {
      const int tc = e / G.xld, i = e - tc * G.xld;
      Xc[e] = i == me + tc * C ? 1.f : 0.f;
    }
  __syncthreads();
  // this CTA's rows of the diagonal block at k0, to every CTA's Db
  auto push_diag = [&](int k0) {
    const int nb = min(CLB, d - k0);
    const int tf = k0 > me ? (k0 - me + C - 1) / C : 0;
    const int tl = min(nown, (k0 + nb - me + C - 1) / C);
    const int nd = max(0, tl - tf);
    for (int e = tid; e < C * nd * (CLB / 4); e += blockDim.x) {
      const int u = e & 7, rest = e >> 3, tt = tf + rest % nd, x = rest / nd;
      const float4 v = *reinterpret_cast<const float4*>(rows + (size_t)tt * G.ld + k0 + 4 * u);
      *reinterpret_cast<float4*>(cl.map_shared_rank(Db, x) + (me + tt * C - k0) * CLPS + 4 * u) = v;
    }
  };
  push_diag(0);
  cl.sync();
  int step = 0;
  for (int k0 = 0; k0 < d; k0 += CLB, ++step) {
    const int nb = min(CLB, d - k0), s = k0 + nb;
    const int t0 = s > me ? (s - me + C - 1) / C : 0;   // first own row below the block
    const int np = max(0, nown - t0);
    if (warp == 0) {
      // the diagonal block (identity past nb), four pivots per round: every lane
      // factors the round's 4 x 4 block (broadcast by shuffles) and forward-
      // substitutes its row, then the rank-4 update of the later columns
      float a[CLB];
#pragma unroll
      for (int j = 0; j < CLB; ++j)
        a[j] = (lane < nb && j <= lane) ? Db[lane * CLPS + j] : (lane == j ? 1.f : 0.f);
      bool bad = false;
#pragma unroll
      for (int r = 0; r < CLB / 4; ++r) {
        const int jb = 4 * r;
        const float d00 = __shfl_sync(~0u, a[jb], jb), d10 = __shfl_sync(~0u, a[jb], jb + 1),
                    d11 = __shfl_sync(~0u, a[jb + 1], jb + 1), d20 = __shfl_sync(~0u, a[jb], jb + 2),
                    d21 = __shfl_sync(~0u, a[jb + 1], jb + 2), d22 = __shfl_sync(~0u, a[jb + 2], jb + 2),
                    d30 = __shfl_sync(~0u, a[jb], jb + 3), d31 = __shfl_sync(~0u, a[jb + 1], jb + 3),
                    d32 = __shfl_sync(~0u, a[jb + 2], jb + 3), d33 = __shfl_sync(~0u, a[jb + 3], jb + 3);
        bad |= !pivot_ok32(d00);
        const float y0 = rsqrt_approx(d00);
        const float l10 = d10 * y0, l20 = d20 * y0, l30 = d30 * y0;
        const float e11 = fmaf(-l10, l10, d11);
        bad |= !pivot_ok32(e11);
        const float y1 = rsqrt_approx(e11);
        const float l21 = fmaf(-l20, l10, d21) * y1, l31 = fmaf(-l30, l10, d31) * y1;
        const float e22 = fmaf(-l21, l21, fmaf(-l20, l20, d22));
        bad |= !pivot_ok32(e22);
        const float y2 = rsqrt_approx(e22);
        const float l32 = fmaf(-l31, l21, fmaf(-l30, l20, d32)) * y2;
        const float e33 = fmaf(-l32, l32, fmaf(-l31, l31, fmaf(-l30, l30, d33)));
        bad |= !pivot_ok32(e33);
        const float y3 = rsqrt_approx(e33);
        // row lane of L in columns jb .. jb + 3 (zero above the diagonal)
        const float x0 = lane >= jb ? a[jb] * y0 : 0.f;
        const float x1 = lane >= jb + 1 ? fmaf(-x0, l10, a[jb + 1]) * y1 : 0.f;
        const float x2 = lane >= jb + 2 ? fmaf(-x1, l21, fmaf(-x0, l20, a[jb + 2])) * y2 : 0.f;
        const float x3 =
            lane >= jb + 3 ? fmaf(-x2, l32, fmaf(-x1, l31, fmaf(-x0, l30, a[jb + 3]))) * y3 : 0.f;
        a[jb] = x0; a[jb + 1] = x1; a[jb + 2] = x2; a[jb + 3] = x3;
        float4* cb = colb + r * CLB;
        cb[lane] = make_float4(x0, x1, x2, x3);
        if (lane == 0) {
          float* rb = rbuf + r * 12;
          rb[0] = y0; rb[1] = y1; rb[2] = y2; rb[3] = y3;
          rb[4] = l10; rb[5] = l20; rb[6] = l21; rb[7] = l30; rb[8] = l31; rb[9] = l32;
        }
        __syncwarp();
        if (lane == 0) st_release_cta(&flag, step * (CLB / 4) + r + 1);
#pragma unroll
        for (int c = jb + 4; c < CLB; ++c) {
          const float4 lc = cb[c];
          a[c] = fmaf(-x3, lc.w, fmaf(-x2, lc.z, fmaf(-x1, lc.y, fmaf(-x0, lc.x, a[c]))));
        }
      }
      if (lane == 0 && bad) bad_s = 1;
      if (lane < nb && (k0 + lane) % C == me) {             // L_kk rows owned here
        float* dr = rows + (size_t)((k0 + lane) / C) * G.ld + k0;
#pragma unroll
        for (int j = 0; j < CLB; ++j)
          if (j <= lane) dr[j] = a[j];
      }
    } else {
      // own rows below the block and (with X) own columns j < s of B's block row k,
      // one per lane, each round applied as soon as it is published
      const int ncolk = inv && s > me ? (s - me + C - 1) / C : 0;
      const int nitem = np + ncolk;
      const int nchb = (nitem + 31) >> 5;
      for (int ch = warp - 1; ch < nchb; ch += nw - 1) {
        const int q = ch * 32 + lane;
        const bool has = q < np;
        const bool hasx = !has && q < nitem;
        const int tc = hasx ? q - np : 0;
        float* prow = rows + (size_t)(t0 + (has ? q : 0)) * G.ld + k0;
        float* xcol = Xc + (size_t)tc * G.xld + k0;
        float p[CLB];
#pragma unroll
        for (int u = 0; u < CLB / 4; ++u) {
          const float4 v = has ? *reinterpret_cast<const float4*>(prow + 4 * u)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
          p[4 * u] = v.x; p[4 * u + 1] = v.y; p[4 * u + 2] = v.z; p[4 * u + 3] = v.w;
        }
        if (hasx) {
#pragma unroll
          for (int r = 0; r < CLB; ++r) p[r] = r < nb ? xcol[r] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < CLB / 4; ++r) {
          const int jb = 4 * r;
          // warp 0 never waits, so this wait ends; the limit only guards against a bug
          for (int spins = 0; ld_acquire_cta(&flag) <= step * (CLB / 4) + r; )
            if (++spins > (1 << 24)) { set_status(status, DEV_INTERNAL); break; }
          const float* rb = rbuf + r * 12;
          const float4 yy = *reinterpret_cast<const float4*>(rb);       // y0 .. y3
          const float4 la = *reinterpret_cast<const float4*>(rb + 4);   // l10 l20 l21 l30
          const float2 lb = *reinterpret_cast<const float2*>(rb + 8);   // l31 l32
          const float x0 = p[jb] * yy.x;
          const float x1 = fmaf(-x0, la.x, p[jb + 1]) * yy.y;
          const float x2 = fmaf(-x1, la.z, fmaf(-x0, la.y, p[jb + 2])) * yy.z;
          const float x3 = fmaf(-x2, lb.y, fmaf(-x1, lb.x, fmaf(-x0, la.w, p[jb + 3]))) * yy.w;
          p[jb] = x0; p[jb + 1] = x1; p[jb + 2] = x2; p[jb + 3] = x3;
          const float4* cb = colb + r * CLB;
#pragma unroll
          for (int c = jb + 4; c < CLB; ++c) {
            const float4 lc = cb[c];
            p[c] = fmaf(-x3, lc.w, fmaf(-x2, lc.z, fmaf(-x1, lc.y, fmaf(-x0, lc.x, p[c]))));
          }
        }
        if (has) {
#pragma unroll
          for (int u = 0; u < CLB / 4; ++u)
            *reinterpret_cast<float4*>(prow + 4 * u) =
                make_float4(p[4 * u], p[4 * u + 1], p[4 * u + 2], p[4 * u + 3]);
        }
        if (hasx) {                                   // X_k column: into B and the staging copy
#pragma unroll
          for (int r = 0; r < CLB; ++r)
            if (r < nb) xcol[r] = p[r];
#pragma unroll
          for (int u = 0; u < CLB / 4; ++u)
            *reinterpret_cast<float4*>(Xk + tc * CLB + 4 * u) =
                make_float4(p[4 * u], p[4 * u + 1], p[4 * u + 2], p[4 * u + 3]);
        }
      }
    }
    __syncthreads();
    if (bad_s) {                                      // the same in every CTA, at the same step
      if (me == 0 && tid == 0) set_status(status, DEV_NOTSPD);
      return;
    }
    if (s >= d) break;
    // own panel rows into every CTA's panel buffer
    for (int e = tid; e < C * np * (CLB / 4); e += blockDim.x) {
      const int u = e & 7, rest = e >> 3, tt = t0 + rest % np, x = rest / np;
      const float4 v = *reinterpret_cast<const float4*>(rows + (size_t)tt * G.ld + k0 + 4 * u);
      *reinterpret_cast<float4*>(cl.map_shared_rank(Pb, x) + (size_t)(me + tt * C - s) * CLPS +
                                 4 * u) = v;
    }
    cl.sync();                                        // every panel row has arrived
    // trailing entries of the own rows i >= s, columns s <= c <= i: item = (4 own rows,
    // 32 columns), 8 threads per item, thread columns c = cb + l8 + 8 v
    const int npan = d - s;
    const int nrg = (np + 3) / 4, nck = (npan + 31) / 32;
    const int l8 = lane & 7;
    for (int it = tid >> 3; it < nrg * nck; it += blockDim.x >> 3) {
      const int rg = it / nck, ck = it - rg * nck;
      const int tA = t0 + 4 * rg, nr4 = min(4, nown - tA);
      const int ilast = me + (tA + nr4 - 1) * C;
      const int cb = s + 32 * ck;
      if (cb > ilast) continue;
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[r][v] = 0.f;
#pragma unroll 2
      for (int q4 = 0; q4 < CLB / 4; ++q4) {
        float4 ar[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          ar[r] = r < nr4 ? *reinterpret_cast<const float4*>(rows + (size_t)(tA + r) * G.ld + k0 + 4 * q4)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int v = 0; v < 4; ++v)
          b[v] = *reinterpret_cast<const float4*>(Pb + (size_t)(cb - s + l8 + 8 * v) * CLPS + 4 * q4);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int v = 0; v < 4; ++v)
            acc[r][v] = fmaf(ar[r].x, b[v].x, fmaf(ar[r].y, b[v].y,
                        fmaf(ar[r].z, b[v].z, fmaf(ar[r].w, b[v].w, acc[r][v]))));
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (r >= nr4) break;
        const int i = me + (tA + r) * C;
        float* dst = rows + (size_t)(tA + r) * G.ld;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = cb + l8 + 8 * v;
          if (c <= i) dst[c] -= acc[r][v];
        }
      }
    }
    if (inv) {
      // B_i -= L_ik X_k for the own columns j < s and the rows i >= s:
      // item = (32 rows, 4 columns), thread rows i = s + 32 rc + l8 + 8 v
      const int ncolk = s > me ? (s - me + C - 1) / C : 0;
      const int nrc = (npan + 31) / 32, ncg = (ncolk + 3) / 4;
      for (int it = tid >> 3; it < nrc * ncg; it += blockDim.x >> 3) {
        const int rc = it / ncg, cg4 = it - rc * ncg;
        float acc[4][4];
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[v][w] = 0.f;
#pragma unroll 2
        for (int q4 = 0; q4 < CLB / 4; ++q4) {
          float4 b[4], xk[4];
#pragma unroll
          for (int v = 0; v < 4; ++v)
            b[v] = *reinterpret_cast<const float4*>(Pb + (size_t)(32 * rc + l8 + 8 * v) * CLPS + 4 * q4);
#pragma unroll
          for (int w = 0; w < 4; ++w)
            xk[w] = *reinterpret_cast<const float4*>(Xk + (4 * cg4 + w) * CLB + 4 * q4);
#pragma unroll
          for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int w = 0; w < 4; ++w)
              acc[v][w] = fmaf(b[v].x, xk[w].x, fmaf(b[v].y, xk[w].y,
                          fmaf(b[v].z, xk[w].z, fmaf(b[v].w, xk[w].w, acc[v][w]))));
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int tc = 4 * cg4 + w;
          if (tc >= ncolk) break;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = s + 32 * rc + l8 + 8 * v;
            if (i < d) Xc[(size_t)tc * G.xld + i] -= acc[v][w];
          }
        }
      }
    }
    __syncthreads();
    push_diag(s);
    cl.sync();                                        // next block in place; panel reads done
  }
  for (int t = warp; t < nown; t += nw) {
    const int i = me + t * C;
    for (int c = lane; c <= i; c += 32) M[(size_t)i * d + c] = rows[(size_t)t * G.ld + c];
  }
  if (inv)                                            // X row-major and column-major (XC = X^T)
    for (int tc = warp; tc < nown; tc += nw) {
      const int j = me + tc * C;
      for (int i = lane; i < d; i += 32) {
        const float v = Xc[(size_t)tc * G.xld + i];
        XC[(size_t)j * d + i] = v;
        X[(size_t)i * d + j] = v;
      }
    }
}

// Whether a cluster of C CTAs with smem bytes of shared memory each can be
// scheduled (the device's own answer; non-portable sizes need an opt-in).
static bool cluster_fits(int C, size_t smem) {
  const void* kern = (const void*)k_chol32_cluster;
  if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                   cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(CHOL_CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n >= 1;
}

// Cluster size for the one-cluster factor of order d, with or without the
// inverse (0: neither 16 nor 8 CTAs can hold it).  Both answers are cached per d.
static int chol_cluster_size(tucker_handle* h, int d, bool inv) {
  if (d > CHOL_CL_MAX_D) return 0;
  if (h->chol_cluster_key != d) {
    for (int v = 0; v < 2; ++v) {
      int C = 0;
      for (int c : {16, 8}) {
        const size_t smem = chol_cl_geom(d, c, v == 1).smem;
        if (smem <= CHOL_CL_SMEM_MAX && cluster_fits(c, smem)) { C = c; break; }
      }
      h->chol_cluster[v] = C;
    }
    h->chol_cluster_key = d;
  }
  return h->chol_cluster[inv ? 1 : 0];
}

static tucker_status cholesky32_cluster(tucker_handle* h, float* M, int d, int C, float* X,
                                        float* XC) {
  const void* kern = (const void*)k_chol32_cluster;
  const size_t smem = chol_cl_geom(d, C, X != nullptr).smem;
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(CHOL_CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TK_COUNT(h);
  TK_CUDA(h, cudaLaunchKernelEx(&cfg, k_chol32_cluster, M, d, h->d_status, X, XC));
  return TUCKER_OK;
}

// Whether the FP32 factor of order d runs on one thread-block cluster (so the
// rest of the GPU is free for other work meanwhile).
bool chol32_on_cluster(tucker_handle* h, int d) {
  return chol_cluster_size(h, d, true) > 0 || chol_cluster_size(h, d, false) > 0;
}

// FP32 Cholesky; with X / XC given (d x d each) and d small enough, the
// explicit inverse comes out of the same launch (*inv_done = 1).
tucker_status cholesky32(tucker_handle* h, float* M, int d, float* X, float* XC, int* inv_done) {
  *inv_done = 0;
  if (X && XC) {
    const int C = chol_cluster_size(h, d, true);
    if (C > 0) {
      TK_TRY(cholesky32_cluster(h, M, d, C, X, XC));
      *inv_done = 1;
      return TUCKER_OK;
    }
  }
  const int C = chol_cluster_size(h, d, false);
  if (C > 0) return cholesky32_cluster(h, M, d, C, nullptr, nullptr);
  return cholesky_t<float>(h, M, d);
}

// ------------------------------------------------------------ triangular solves
// Inverses of the SB x SB diagonal blocks of L (one CTA per block, thread j
// forward-substitutes column j of the identity); then each solve is one
// persistent launch: per block, every CTA forms y_k = Linv_kk b_k in shared
// memory and removes it from its share of the remaining rows (warp per row),
// with one grid-wide barrier per block.  Forward L y = b, then backward
// L^T g = y reading the transposed factor row-wise.

template <class T>
__global__ void __launch_bounds__(SB) k_inv_diag_blocks(const T* L, int d, T* Linv) {
  __shared__ T a[SB][SB + 1];
  __shared__ T rp[SB];
  const int k = blockIdx.x * SB, nb = min(SB, d - k);
  for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) {
    const int i = e / SB, j = e % SB;
    a[i][j] = (i < nb && j < nb && j <= i) ? L[(size_t)(k + i) * d + k + j] : (i == j ? T(1) : T(0));
  }
  __syncthreads();
  rp[threadIdx.x] = T(1) / a[threadIdx.x][threadIdx.x];
  __syncthreads();
  const int j = threadIdx.x;                      // column j of the inverse
  T x[SB];
#pragma unroll
  for (int i = 0; i < SB; ++i) {
    T v = (i == j) ? T(1) : T(0);
#pragma unroll
    for (int c = 0; c < i; ++c) v = fma(-a[i][c], x[c], v);
    x[i] = (i < j) ? T(0) : v * rp[i];
  }
  T* out = Linv + (size_t)blockIdx.x * SB * SB;
#pragma unroll
  for (int i = 0; i < SB; ++i) out[i * SB + j] = x[i];
}

template <class T>
__global__ void __launch_bounds__(256) k_trsv_coop(const T* L, const T* LT, const T* Linv, int d,
                                                   double* b, double* y, const int* status) {
  cg::grid_group grid = cg::this_grid();
  __shared__ T yk[SB];
  __shared__ T bk[SB];
  __shared__ T Ls[SB][SB + 1];
  if (*status) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int nblk = (d + SB - 1) / SB;
  // forward: L y = b   (b is consumed as workspace)
  for (int kb = 0; kb < nblk; ++kb) {
    const int k = kb * SB, nb = min(SB, d - k);
    const T* Li = Linv + (size_t)kb * SB * SB;
    for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) Ls[e / SB][e % SB] = Li[e];
    if (threadIdx.x < SB) bk[threadIdx.x] = threadIdx.x < nb ? (T)b[k + threadIdx.x] : T(0);
    __syncthreads();
    {                                                   // yk = Linv_kk bk: 4 threads per row
      const int i = threadIdx.x >> 2, part = threadIdx.x & 3;
      T v = T(0);
      for (int j = part; j <= i; j += 4) v = fma(Ls[i][j], bk[j], v);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      if (part == 0) {
        yk[i] = v;
        if (blockIdx.x == 0 && i < nb) y[k + i] = (double)v;
      }
    }
    __syncthreads();
    for (int row = k + nb + blockIdx.x * nwarps + warp; row < d; row += gridDim.x * nwarps) {
      const T* lr = L + (size_t)row * d + k;
      T v = T(0);
      for (int j = lane; j < nb; j += 32) v = fma(lr[j], yk[j], v);
      v = warp_sum(v);
      if (lane == 0) b[row] -= (double)v;
    }
    grid.sync();
  }
  // backward: L^T g = y   (g written into b)
  for (int kb = nblk - 1; kb >= 0; --kb) {
    const int k = kb * SB, nb = min(SB, d - k);
    const T* Li = Linv + (size_t)kb * SB * SB;
    for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) Ls[e / SB][e % SB] = Li[e];
    if (threadIdx.x < SB) bk[threadIdx.x] = threadIdx.x < nb ? (T)y[k + threadIdx.x] : T(0);
    __syncthreads();
    {                                                   // (L_kk^T)^-1 = (L_kk^-1)^T
      const int i = threadIdx.x >> 2, part = threadIdx.x & 3;
      T v = T(0);
      for (int j = i + part; j < SB; j += 4) v = fma(Ls[j][i], bk[j], v);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      if (part == 0) {
        yk[i] = v;
        if (blockIdx.x == 0 && i < nb) b[k + i] = (double)v;
      }
    }
    __syncthreads();
    for (int col = blockIdx.x * nwarps + warp; col < k; col += gridDim.x * nwarps) {
      const T* lc = LT + (size_t)col * d + k;          // row col of L^T = column col of L
      T v = T(0);
      for (int j = lane; j < nb; j += 32) v = fma(lc[j], yk[j], v);
      v = warp_sum(v);
      if (lane == 0) y[col] -= (double)v;
    }
    grid.sync();
  }
}

// LT[c][r] = L[r][c] for c <= r (the transposed factor, for coalesced
// backward substitution).
template <class T>
__global__ void k_transpose_lower(const T* L, int d, T* LT) {
  __shared__ T t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  if (bx > by + 31) return;                       // tile entirely above the diagonal of L
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = by + i, c = bx + threadIdx.x;
    t[i][threadIdx.x] = (r < d && c < d && c <= r) ? L[(size_t)r * d + c] : T(0);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = bx + i, r = by + threadIdx.x;
    if (r < d && c < d && c <= r) LT[(size_t)c * d + r] = t[threadIdx.x][i];
  }
}

size_t chol_inv_doubles(int d) { return (size_t)((d + SB - 1) / SB) * SB * SB; }

// Transposed copy and inverted diagonal blocks of a computed factor.
template <class T>
tucker_status chol_prepare_t(tucker_handle* h, const T* L, int d, T* LT, T* Linv) {
  dim3 grid((d + 31) / 32, (d + 31) / 32);
  TK_COUNT(h);
  k_transpose_lower<T><<<grid, dim3(32, 8), 0, h->stream>>>(L, d, LT);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_inv_diag_blocks<T><<<(d + SB - 1) / SB, SB, 0, h->stream>>>(L, d, Linv);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

tucker_status chol_prepare(tucker_handle* h, const double* L, int d, double* LT, double* Linv) {
  return chol_prepare_t<double>(h, L, d, LT, Linv);
}
tucker_status chol_prepare32(tucker_handle* h, const float* L, int d, float* LT, float* Linv) {
  return chol_prepare_t<float>(h, L, d, LT, Linv);
}

// g = (L L^T)^-1 rhs; tmp: d doubles of scratch.  g may alias rhs.
template <class T>
tucker_status chol_solve_t(tucker_handle* h, const T* L, const T* LT, const T* Linv, int d,
                           const double* rhs, double* g, double* tmp) {
  if (g != rhs)
    TK_CUDA(h, cudaMemcpyAsync(g, rhs, sizeof(double) * d, cudaMemcpyDeviceToDevice, h->stream));
  const void* kern = (const void*)k_trsv_coop<T>;
  const int grid = coop_grid(h, kern, 256, 0);
  if (grid < 1) return fail(h, TUCKER_ECUDA, "cooperative solve cannot be resident");
  void* args[] = {(void*)&L, (void*)&LT, (void*)&Linv, &d, &g, &tmp, &h->d_status};
  TK_COUNT(h);
  TK_CUDA(h, cudaLaunchCooperativeKernel(kern, grid, 256, args, 0, h->stream));
  return TUCKER_OK;
}

tucker_status chol_solve2(tucker_handle* h, const double* L, const double* LT, const double* Linv,
                          int d, const double* rhs, double* g, double* tmp) {
  return chol_solve_t<double>(h, L, LT, Linv, d, rhs, g, tmp);
}
tucker_status chol_solve32(tucker_handle* h, const float* L, const float* LT, const float* Linv,
                           int d, const double* rhs, double* g, double* tmp) {
  return chol_solve_t<float>(h, L, LT, Linv, d, rhs, g, tmp);
}

// ------------------------------------------------ explicit inverse (small FP32 factors)
// For d <= INV_MAX_D the refinement applies M~^-1 = X^T X with X = L^-1 held
// explicitly: two GEMVs per solve instead of 2 d / 64 dependent block steps.
// X is built column by column: CTA c solves L x = e_j for its INV_COLS
// columns by forward block substitution with the inverted 64 x 64 diagonal
// blocks; the columns are independent, so no grid-wide barrier is needed.
// X is stored row-major and column-major (XC[j][i] = X[i][j]) so that both
// GEMVs read contiguous rows.
constexpr int INV_COLS = 4;
constexpr int INV_THREADS = 256;
constexpr int INV_MAX_D = 1024;

__global__ void __launch_bounds__(INV_THREADS) k_tri_inv_cols(const float* L, const float* Linv,
                                                              int d, float* X, float* XC) {
  extern __shared__ float bsm[];                  // right-hand sides, [INV_COLS][d]
  __shared__ float Ls[SB][SB + 1];
  __shared__ float yk[SB][INV_COLS];
  const int j0 = blockIdx.x * INV_COLS;
  const int ncol = min(INV_COLS, d - j0);
  const int nblk = (d + SB - 1) / SB;
  const int kb0 = j0 / SB;
  for (int e = threadIdx.x; e < INV_COLS * d; e += blockDim.x) {
    const int c = e / d, i = e % d;
    bsm[e] = (c < ncol && i == j0 + c) ? 1.f : 0.f;
  }
  // rows above the first block with a nonzero right-hand side are zero
  for (int e = threadIdx.x; e < kb0 * SB * INV_COLS; e += blockDim.x) {
    const int i = e / INV_COLS, c = e % INV_COLS;
    if (c < ncol) {
      X[(size_t)i * d + j0 + c] = 0.f;
      XC[(size_t)(j0 + c) * d + i] = 0.f;
    }
  }
  __syncthreads();
  for (int kb = kb0; kb < nblk; ++kb) {
    const int k = kb * SB, nb = min(SB, d - k);
    const float* Li = Linv + (size_t)kb * SB * SB;
    for (int e = threadIdx.x; e < SB * SB; e += blockDim.x) Ls[e / SB][e % SB] = Li[e];
    __syncthreads();
    {                                             // yk = Linv_kk b_k: thread (row i, column c)
      const int i = threadIdx.x >> 2, c = threadIdx.x & 3;
      float v = 0.f;
      if (i < nb && c < ncol) {
        const float* bc = bsm + (size_t)c * d + k;
        for (int jj = 0; jj <= i; ++jj) v = fmaf(Ls[i][jj], bc[jj], v);
        X[(size_t)(k + i) * d + j0 + c] = v;
        XC[(size_t)(j0 + c) * d + k + i] = v;
      }
      yk[i][c] = v;
    }
    __syncthreads();
    // b_i -= L_ik y_k for the rows below the block, one thread per row
    const int nb4 = (d & 3) == 0 ? nb / 4 : 0;    // 16-byte loads need 16-byte aligned rows
    for (int i = k + nb + threadIdx.x; i < d; i += blockDim.x) {
      const float4* lr = reinterpret_cast<const float4*>(L + (size_t)i * d + k);
      float acc[INV_COLS] = {0.f, 0.f, 0.f, 0.f};
      for (int q = 0; q < nb4; ++q) {
        const float4 l4 = lr[q];
#pragma unroll
        for (int c = 0; c < INV_COLS; ++c)
          acc[c] = fmaf(l4.x, yk[4 * q][c], fmaf(l4.y, yk[4 * q + 1][c],
                   fmaf(l4.z, yk[4 * q + 2][c], fmaf(l4.w, yk[4 * q + 3][c], acc[c]))));
      }
      for (int jj = nb4 * 4; jj < nb; ++jj) {
        const float l = L[(size_t)i * d + k + jj];
#pragma unroll
        for (int c = 0; c < INV_COLS; ++c) acc[c] = fmaf(l, yk[jj][c], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < INV_COLS; ++c) bsm[(size_t)c * d + i] -= acc[c];
    }
    __syncthreads();
  }
}

tucker_status chol_inverse32(tucker_handle* h, const float* L, const float* Linv, int d, float* X,
                             float* XC) {
  if (d > INV_MAX_D || !X || !XC) return fail(h, TUCKER_EINTERNAL, "explicit inverse not sized");
  const size_t smem = (size_t)INV_COLS * d * sizeof(float);
  TK_COUNT(h);
  k_tri_inv_cols<<<(d + INV_COLS - 1) / INV_COLS, INV_THREADS, smem, h->stream>>>(L, Linv, d, X, XC);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

int chol_inverse_fits(int d) { return d <= INV_MAX_D; }

// out = X^T (X rhs) in one cooperative launch: each warp forms rows of
// t = X rhs (FP32 products and sums, one warp per row, rhs staged in
// shared memory as FP32), a grid barrier, then rows of X^T t from the
// column-major copy XC.  With upd given, also upd += out and
// stats = (sum out_i^2, sum upd_i^2): partial sums per warp and per CTA,
// combined by CTA 0 in a fixed order after a second barrier.  rhs may alias out.
constexpr int IA_THREADS = 256;
constexpr int IA_MAX_CTAS = 256;                 // CTAs of one application, at most

__global__ void __launch_bounds__(IA_THREADS)
    k_inv_apply(const float* X, const float* XC, int d, const double* rhs, double* out,
                double* upd, double* stats, double* t, double* part) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) float ia_v[];             // rhs, then t, as FP32
  __shared__ double wpart[IA_THREADS / 32][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int gw = blockIdx.x * (IA_THREADS / 32) + w, nwarps = gridDim.x * (IA_THREADS / 32);
  for (int j = threadIdx.x; j < d; j += IA_THREADS) ia_v[j] = (float)rhs[j];
  __syncthreads();
  const bool vec = (d & 3) == 0;                            // 16-byte rows: float4 loads
  for (int i = gw; i < d; i += nwarps) {                    // t_i = sum_{j <= i} X_ij rhs_j
    const float* xr = X + (size_t)i * d;
    float acc = 0.f;
    if (vec) {                                              // X_ij = 0 above the diagonal
      const float4* x4 = reinterpret_cast<const float4*>(xr);
      const float4* v4 = reinterpret_cast<const float4*>(ia_v);
#pragma unroll 2
      for (int q = lane; 4 * q <= i; q += 32) {
        const float4 xv = x4[q], vv = v4[q];
        acc = fmaf(xv.x, vv.x, acc); acc = fmaf(xv.y, vv.y, acc);
        acc = fmaf(xv.z, vv.z, acc); acc = fmaf(xv.w, vv.w, acc);
      }
    } else {
#pragma unroll 4
      for (int j = lane; j <= i; j += 32) acc = fmaf(xr[j], ia_v[j], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) t[i] = (double)acc;
  }
  grid.sync();                                              // t complete; every rhs read done
  for (int j = threadIdx.x; j < d; j += IA_THREADS) ia_v[j] = (float)t[j];
  __syncthreads();
  double s_out = 0.0, s_upd = 0.0;
  for (int j = gw; j < d; j += nwarps) {                    // out_j = sum_{i >= j} X_ij t_i
    const float* xr = XC + (size_t)j * d;
    float acc = 0.f;
    if (vec) {                                              // XC_ji = X_ij = 0 for i < j
      const float4* x4 = reinterpret_cast<const float4*>(xr);
      const float4* v4 = reinterpret_cast<const float4*>(ia_v);
#pragma unroll 2
      for (int q = (j >> 2) + lane; 4 * q < d; q += 32) {
        const float4 xv = x4[q], vv = v4[q];
        acc = fmaf(xv.x, vv.x, acc); acc = fmaf(xv.y, vv.y, acc);
        acc = fmaf(xv.z, vv.z, acc); acc = fmaf(xv.w, vv.w, acc);
      }
    } else {
#pragma unroll 4
      for (int i = j + lane; i < d; i += 32) acc = fmaf(xr[i], ia_v[i], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) {
      const double o = (double)acc;
      if (out) out[j] = o;
      if (upd) {
        const double gn = upd[j] + o;
        upd[j] = gn;
        s_out = fma(o, o, s_out);
        s_upd = fma(gn, gn, s_upd);
      }
    }
  }
  if (upd && stats) {
    if (lane == 0) { wpart[w][0] = s_out; wpart[w][1] = s_upd; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < IA_THREADS / 32; ++k) { a += wpart[k][0]; b += wpart[k][1]; }
      part[2 * blockIdx.x] = a;
      part[2 * blockIdx.x + 1] = b;
    }
    grid.sync();                                            // every CTA's partial written
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < (int)gridDim.x; ++k) { a += part[2 * k]; b += part[2 * k + 1]; }
      stats[0] = a;
      stats[1] = b;
    }
  }
}

static tucker_status launch_inv_apply(tucker_handle* h, const float* X, const float* XC, int d,
                                      const double* rhs, double* out, double* upd, double* stats,
                                      double* t, double* part) {
  const void* kern = (const void*)k_inv_apply;
  const size_t smem = (size_t)d * sizeof(float);
  int grid = (d + 7) / 8;                                   // one row per warp per phase
  const int cap = coop_grid(h, kern, IA_THREADS, smem);
  if (cap < 1) return fail(h, TUCKER_ECUDA, "cooperative inverse application cannot be resident");
  if (grid > cap) grid = cap;
  if (grid > IA_MAX_CTAS) grid = IA_MAX_CTAS;
  void* args[] = {(void*)&X, (void*)&XC, &d, (void*)&rhs, &out, &upd, &stats, &t, &part};
  TK_COUNT(h);
  TK_CUDA(h, cudaLaunchCooperativeKernel(kern, grid, IA_THREADS, args, smem, h->stream));
  return TUCKER_OK;
}

// g = X^T (X rhs) (g may alias rhs); tmp: d doubles of scratch.
tucker_status chol_solve_inv32(tucker_handle* h, const float* X, const float* XC, int d,
                               const double* rhs, double* g, double* tmp) {
  return launch_inv_apply(h, X, XC, d, rhs, g, nullptr, nullptr, tmp, nullptr);
}

// r = X^T (X r), then g += r and stats = (||r||^2, ||g||^2): one refinement
// correction with the explicit inverse; tmp: d doubles, part: 2 IA_MAX_CTAS doubles.
tucker_status chol_correct_inv32(tucker_handle* h, const float* X, const float* XC, int d,
                                 double* r, double* g, double* stats, double* tmp, double* part) {
  return launch_inv_apply(h, X, XC, d, r, r, g, stats, tmp, part);
}

tucker_status launch_to_f32(tucker_handle* h, const double* in, size_t n, float* out) {
  int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)h->num_sms * 16);
  if (grid < 1) grid = 1;
  TK_CUDA(h, launch_dep(h, k_to_f32, grid, 256, 0, in, n, out));
  return TUCKER_OK;
}

// r = h - M g with the explicit symmetric FP64 matrix M (warp per row).
__global__ void k_gemv_resid(const double* M, int d, const double* g, const double* hv, double* r) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int row = warp; row < d; row += nwarps) {
    const double* mr = M + (size_t)row * d;
    double v = 0.0;
    for (int j = lane; j < d; j += 32) v = fma(mr[j], g[j], v);
    v = warp_sum(v);
    if (lane == 0) r[row] = hv[row] - v;
  }
}

tucker_status launch_gemv_resid(tucker_handle* h, const double* M, int d, const double* g,
                                const double* hv, double* r) {
  int grid = (d + 7) / 8;
  if (grid > h->num_sms * 8) grid = h->num_sms * 8;
  TK_COUNT(h);
  k_gemv_resid<<<grid, 256, 0, h->stream>>>(M, d, g, hv, r);
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
  TK_CUDA(h, launch_dep(h, k_regdiag, ceil_div(d, 256), 256, 0, out, d, lambda, D));
  return TUCKER_OK;
}

tucker_status launch_add_diag(tucker_handle* h, double* M, int d, const double* diag) {
  TK_CUDA(h, launch_dep(h, k_add_diag, ceil_div(d, 256), 256, 0, M, d, diag));
  return TUCKER_OK;
}

}  // namespace tk
