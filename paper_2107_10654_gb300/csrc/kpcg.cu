// Ridge solve by conjugate gradients with a Kronecker preconditioner
// (TUCKER_SOLVER_KRON_PCG): the inner solver of the FP64 refinement when the
// Gram of the sample is rounded (FP32, TF32, BF16).
//
// Why it works.  The sketched Gram G = sum_u w_u k_u k_u^T is an unbiased
// estimate of K^T K = (x)_n A^(n)T A^(n) (Appendix A, Thm A.3; with observed
// entries it estimates K_Omega^T K_Omega, which for a uniform mask is the
// observed fraction times K^T K).  With the eigendecompositions
// A^(n)T A^(n) = V_n diag(ev_n) V_n^T already needed for the leverage scores
// (Sec. 2 and the proof of Lemma 4.1), the matrix
//     P = (x)_n V_n  diag(s (x)_n ev_n + lbar)  (x)_n V_n^T,
//     s = (tr M - sum_j regdiag_j) / prod_n tr(A^(n)T A^(n)),  lbar = mean(regdiag),
// is spectrally close to M = G + diag(regdiag) once m is large enough for the
// sketch to be a subspace embedding (the regime Thm 3.4 works in), so CG on M
// preconditioned by P converges in a handful of iterations.  Applying P^-1
// costs 2 d sum_n R_n multiply-adds (mode products with V_n^T, a diagonal
// scale, mode products with V_n), against d^3 / 3 for a Cholesky factor.
//
// The iteration is CG in the single-reduction form of Chronopoulos and Gear
// (1989): per iteration one product s = M z with z = P^-1 r and the scalars
// gamma = r.z, delta = z.s; then beta = gamma / gamma_old,
// alpha = gamma / (delta - beta gamma / alpha_old), p = z + beta p,
// q = s + beta q, x += alpha p, r -= alpha q.
//
// GB300 mapping: one cooperative launch of C CTAs.  Every CTA keeps the full
// d-vectors r, z, p, q, x and the preconditioner's diagonal in shared memory
// and owns a contiguous block of rows of M; each iteration it multiplies its
// rows of M (FP32, 16-byte loads, one warp per row) by z, publishes that block
// of s to global memory (double-buffered by iteration parity), passes one grid
// barrier and reads all of s back.  Everything else (P^-1 r, the dot products,
// the vector updates) is computed redundantly by every CTA in the same order,
// so all CTAs hold bit-identical vectors and take the same stopping decision
// without a second barrier.  M stays in L2 across iterations at d <= 4096
// (64 MiB as FP32).
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace tk {

constexpr int KP_THREADS = 512;
constexpr int KP_WARPS = KP_THREADS / 32;
constexpr int KP_BMAX = 16;                     // d <= KP_BMAX * KP_THREADS = 8192

struct KpcgArgs {
  const float* M;                       // d x d, row-major, symmetric, regdiag included
  const double* regdiag;                // d: the lambda R diagonal contained in M
  int d;
  int N;
  int R[TUCKER_MAX_ORDER];
  FastDiv div_in[TUCKER_MAX_ORDER];     // by inner_n = prod_{m > n} R_m
  FastDiv div_r[TUCKER_MAX_ORDER];      // by R_n
  const double* V[TUCKER_MAX_ORDER];    // R_n x R_n, V[a * R_n + k] = component a of eigenvector k
  const double* ev[TUCKER_MAX_ORDER];   // R_n eigenvalues of A^(n)T A^(n)
  const double* rhs;                    // FP64 [d]
  double* out;                          // FP64 [d] solution (may alias rhs), or NULL
  double* upd;                          // NULL, or upd += solution
  double* stats;                        // with upd: (||solution||^2, ||upd||^2)
  double* part;                         // per-CTA partials: 2 * gridDim.x doubles
  float* sg;                            // 2 x d floats: s exchange, by iteration parity
  double* res;                          // nullable: [0] iterations, [1] final ||r|| / ||b||
  double tol;                           // stop at ||r|| <= tol ||b||
  int max_iter;
  int* status;                          // device status word (a bounded wait that ran out)
};

constexpr uint32_t KP_WAIT_LIMIT = 1u << 26;    // polls of the row copy's mbarrier, at most

struct KpcgShared {
  FastDiv div_in[TUCKER_MAX_ORDER];
  FastDiv div_r[TUCKER_MAX_ORDER];
  int R[TUCKER_MAX_ORDER];
  int in[TUCKER_MAX_ORDER];
  float part[3][KP_WARPS];              // per-warp partial sums
  float sum[4];                         // CTA sums, broadcast
  float coef[4];                        // alpha, beta, broadcast
  int stop;
  double bscale;                        // power of two >= max |b|: the CG runs on b / bscale
  float ev[TUCKER_MAX_ORDER * TUCKER_MAX_RANK];  // ev_n, clamped at 0, packed
  int evoff[TUCKER_MAX_ORDER];
};

// Sums of up to three per-thread values over the CTA: warp sums, then warp 0
// adds the KP_WARPS partials in a fixed order (the same in every CTA) and
// broadcasts them through sh.sum.  FP32 throughout: each CG solve only has to
// reach a relative residual of about 1e-4 (the FP64 refinement around it sets
// the accuracy of the result), and on GB300 a dependent FP64 operation costs
// tens of cycles on a path every thread of the CTA waits for.
template <int K>
__device__ __forceinline__ void block_sums(KpcgShared& sh, float a, float b, float c) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  a = warp_sum(a);
  if (K > 1) b = warp_sum(b);
  if (K > 2) c = warp_sum(c);
  if (lane == 0) {
    sh.part[0][w] = a;
    if (K > 1) sh.part[1][w] = b;
    if (K > 2) sh.part[2][w] = c;
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float v = lane < KP_WARPS ? sh.part[k][lane] : 0.f;
      v = warp_sum(v);
      if (lane == 0) sh.sum[k] = v;
    }
  }
}

// One element-wise pass of a mode-n product: dst[o][k][i] = sum_q W(q, k) src[o][q][i],
// i < inner (div_in), q, k < R_n (div_r), with W(q, k) = V_n[q][k] (forward,
// V_n^T applied) or V_n[k][q] (backward, V_n applied), times sc[e] if given.
// RN > 0: R_n known at compile time (the loop unrolls, its shared-memory loads
// issue back to back); RN == 0: any R_n.
template <int RN, bool FWD>
__device__ __forceinline__ void mode_pass(int d, int Rn, int in, const FastDiv& div_in,
                                          const FastDiv& div_r, const float* Vn, const float* cur,
                                          const float* sc, float* dst) {
  const int R = RN > 0 ? RN : Rn;
  for (int e = threadIdx.x; e < d; e += KP_THREADS) {
    const uint32_t q1 = in == 1 ? (uint32_t)e : fdiv((uint32_t)e, div_in);
    const int i = e - (int)q1 * in;
    const uint32_t o = fdiv(q1, div_r);
    const int k = (int)q1 - (int)o * R;
    const float* src = cur + (size_t)o * R * in + i;
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < (RN > 0 ? RN : 64); ++q) {
      if (RN == 0 && q >= R) break;
      acc = fmaf(FWD ? Vn[q * R + k] : Vn[k * R + q], src[q * in], acc);
    }
    dst[e] = sc ? acc * sc[e] : acc;
  }
}

template <bool FWD>
__device__ __forceinline__ void mode_pass_any(int d, int Rn, int in, const FastDiv& div_in,
                                              const FastDiv& div_r, const float* Vn,
                                              const float* cur, const float* sc, float* dst) {
  switch (Rn) {
    case 2: mode_pass<2, FWD>(d, Rn, in, div_in, div_r, Vn, cur, sc, dst); break;
    case 3: mode_pass<3, FWD>(d, Rn, in, div_in, div_r, Vn, cur, sc, dst); break;
    case 4: mode_pass<4, FWD>(d, Rn, in, div_in, div_r, Vn, cur, sc, dst); break;
    case 8: mode_pass<8, FWD>(d, Rn, in, div_in, div_r, Vn, cur, sc, dst); break;
    case 16: mode_pass<16, FWD>(d, Rn, in, div_in, div_r, Vn, cur, sc, dst); break;
    default: mode_pass<0, FWD>(d, Rn, in, div_in, div_r, Vn, cur, sc, dst); break;
  }
}

// z = P^-1 r in shared memory: mode products with V_n^T for n = 1 .. N (the
// last one fused with the diagonal scale), then with V_n for n = N .. 1: 2 N
// passes, one barrier each.  t0, t1: d floats of scratch each; Vs: the V_n in
// FP32, packed one after the other.  The divisions use the multiply-shift form.
__device__ void kron_precond(int d, int N, const KpcgShared& sh, const float* Vs,
                             const float* dg, const float* r, float* t0, float* t1, float* z) {
  const float* cur = r;
  float* bufs[2] = {t0, t1};
  int nb = 0;
  int voff = 0;
  for (int n = 0; n < N; ++n) {                        // t = (x V_n)^T r, then the scale
    float* dst = bufs[nb];
    mode_pass_any<true>(d, sh.R[n], sh.in[n], sh.div_in[n], sh.div_r[n], Vs + voff, cur,
                        n == N - 1 ? dg : nullptr, dst);
    __syncthreads();
    cur = dst;
    nb ^= 1;
    voff += sh.R[n] * sh.R[n];
  }
  for (int n = N - 1; n >= 0; --n) {                   // z = (x V_n) t
    voff -= sh.R[n] * sh.R[n];
    float* dst = n == 0 ? z : bufs[nb];
    mode_pass_any<false>(d, sh.R[n], sh.in[n], sh.div_in[n], sh.div_r[n], Vs + voff, cur,
                         nullptr, dst);
    __syncthreads();
    cur = dst;
    nb ^= 1;
  }
}

// kron_precond when every R_n equals R = 2^LR and d = R^NT: the digit of mode n
// in e is (e >> LR (NT - 1 - n)) & (R - 1), so each pass is shifts, masks and R
// multiply-adds with compile-time strides (no divisions, no per-mode dispatch);
// same arithmetic, in the same order, as kron_precond.
template <int NT, int LR>
__device__ void kron_precond_pow2(int d, const float* Vs, const float* dg, const float* r,
                                  float* t0, float* t1, float* z) {
  constexpr int R = 1 << LR, RR = R * R;
  const float* cur = r;
  float* bufs[2] = {t0, t1};
  int nb = 0;
#pragma unroll
  for (int n = 0; n < NT; ++n) {                       // t = (x V_n)^T r, then the scale
    const int sh = LR * (NT - 1 - n);
    float* dst = bufs[nb];
    const float* Vn = Vs + n * RR;
    for (int e = threadIdx.x; e < d; e += KP_THREADS) {
      const int k = (e >> sh) & (R - 1);
      const float* src = cur + (e - (k << sh));
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) acc = fmaf(Vn[q * R + k], src[q << sh], acc);
      dst[e] = n == NT - 1 ? acc * dg[e] : acc;
    }
    __syncthreads();
    cur = dst;
    nb ^= 1;
  }
#pragma unroll
  for (int n = NT - 1; n >= 0; --n) {                  // z = (x V_n) t
    const int sh = LR * (NT - 1 - n);
    float* dst = n == 0 ? z : bufs[nb];
    const float* Vn = Vs + n * RR;
    for (int e = threadIdx.x; e < d; e += KP_THREADS) {
      const int k = (e >> sh) & (R - 1);
      const float* src = cur + (e - (k << sh));
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < R; ++q) acc = fmaf(Vn[k * R + q], src[q << sh], acc);
      dst[e] = acc;
    }
    __syncthreads();
    cur = dst;
    nb ^= 1;
  }
}

// Which kron_precond_pow2 instance applies (0: none): equal ranks R = 2^LR,
// d = R^N, for (N, R) in {2, 3, 4} x {4, 8, 16} with d <= KP_BMAX * KP_THREADS.
__device__ __forceinline__ int precond_kind(int N, const int* R, int d) {
  for (int n = 1; n < N; ++n)
    if (R[n] != R[0]) return 0;
  const int lr = R[0] == 4 ? 2 : R[0] == 8 ? 3 : R[0] == 16 ? 4 : 0;
  if (lr == 0 || N < 2 || N > 4 || d != 1 << (lr * N) || d > KP_BMAX * KP_THREADS) return 0;
  return N * 8 + lr;
}

__device__ __forceinline__ void precond_any(int kind, int d, int N, const KpcgShared& sh,
                                            const float* Vs, const float* dg, const float* r,
                                            float* t0, float* t1, float* z) {
  switch (kind) {
    case 2 * 8 + 3: kron_precond_pow2<2, 3>(d, Vs, dg, r, t0, t1, z); break;
    case 2 * 8 + 4: kron_precond_pow2<2, 4>(d, Vs, dg, r, t0, t1, z); break;
    case 3 * 8 + 2: kron_precond_pow2<3, 2>(d, Vs, dg, r, t0, t1, z); break;
    case 3 * 8 + 3: kron_precond_pow2<3, 3>(d, Vs, dg, r, t0, t1, z); break;
    case 3 * 8 + 4: kron_precond_pow2<3, 4>(d, Vs, dg, r, t0, t1, z); break;
    case 4 * 8 + 2: kron_precond_pow2<4, 2>(d, Vs, dg, r, t0, t1, z); break;
    case 4 * 8 + 3: kron_precond_pow2<4, 3>(d, Vs, dg, r, t0, t1, z); break;
    default: kron_precond(d, N, sh, Vs, dg, r, t0, t1, z); break;
  }
}

// Shared-memory vectors of one CTA (d-vectors padded to dp, 16-byte slots).
struct KpcgVecs {
  float *r, *z, *p, *q, *x, *dg, *t0, *t1, *Vs;
};

__device__ __forceinline__ KpcgVecs kpcg_carve(float* base, int dp) {
  KpcgVecs v;
  v.r = base;
  v.z = v.r + dp;
  v.p = v.z + dp;
  v.q = v.p + dp;
  v.x = v.q + dp;
  v.dg = v.x + dp;
  v.t0 = v.dg + dp;
  v.t1 = v.t0 + dp;
  v.Vs = v.t1 + dp;                                   // sum_n R_n^2 floats
  return v;
}

// Set-up shared by both kernels: ranks and dividers in shared memory, the V_n
// in FP32, s and lbar, the diagonal 1 / (s prod ev + lbar), r = b and
// x = p = q = 0.  Returns ||b||^2 (the same in every CTA).
__device__ float kpcg_setup(const KpcgArgs& a, KpcgShared& sh, const KpcgVecs& v) {
  const int d = a.d, tid = threadIdx.x;
  if (tid < TUCKER_MAX_ORDER) {
    const bool on = tid < a.N;
    sh.R[tid] = on ? a.R[tid] : 1;
    sh.in[tid] = on ? (int)a.div_in[tid].q : 1;
    sh.div_in[tid] = a.div_in[tid];
    sh.div_r[tid] = a.div_r[tid];
  }
  {                                                    // V_n, ev_n into shared memory
    // one pass over all modes' entries, so that every load is in flight at once
    int off = 0, eoff = 0;
    int vo[TUCKER_MAX_ORDER + 1], eo[TUCKER_MAX_ORDER + 1];
    for (int n = 0; n < a.N; ++n) {
      vo[n] = off;
      eo[n] = eoff;
      off += a.R[n] * a.R[n];
      eoff += a.R[n];
    }
    vo[a.N] = off;
    eo[a.N] = eoff;
    for (int e = tid; e < off + eoff; e += KP_THREADS) {
      if (e < off) {
        int n = 0;
        while (e >= vo[n + 1]) ++n;
        v.Vs[e] = (float)a.V[n][e - vo[n]];
      } else {
        const int f = e - off;
        int n = 0;
        while (f >= eo[n + 1]) ++n;
        sh.ev[f] = fmaxf((float)a.ev[n][f - eo[n]], 0.f);
      }
    }
    if (tid < a.N) sh.evoff[tid] = eo[tid];
  }
  // one wave of global loads: the diagonal of M, lambda R and b (b stays in
  // registers: at most KP_BMAX entries per thread)
  float trm = 0.f, sreg = 0.f, bmax = 0.f;
  float bl[KP_BMAX];
#pragma unroll 4
  for (int t = 0; t < KP_BMAX; ++t) {
    const int j = tid + t * KP_THREADS;
    bl[t] = 0.f;
    if (j < d) {
      trm += a.M[(size_t)j * d + j];
      sreg += (float)a.regdiag[j];
      bl[t] = (float)a.rhs[j];
      bmax = fmaxf(bmax, fabsf(bl[t]));
    }
  }
  {                                                    // sums of the diagonals, max |b|
    const int lane = tid & 31, w = tid >> 5;
    trm = warp_sum(trm);
    sreg = warp_sum(sreg);
#pragma unroll
    for (int o = 16; o; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    if (lane == 0) {
      sh.part[0][w] = trm;
      sh.part[1][w] = sreg;
      sh.part[2][w] = bmax;
    }
    __syncthreads();                                   // (also publishes ev_n, V_n)
    if (w == 0) {
      float t0 = lane < KP_WARPS ? sh.part[0][lane] : 0.f;
      float t1 = lane < KP_WARPS ? sh.part[1][lane] : 0.f;
      float t2 = lane < KP_WARPS ? sh.part[2][lane] : 0.f;
      t0 = warp_sum(t0);
      t1 = warp_sum(t1);
#pragma unroll
      for (int o = 16; o; o >>= 1) t2 = fmaxf(t2, __shfl_xor_sync(0xffffffffu, t2, o));
      float trp = 1.f;                                 // prod_n tr(A^(n)T A^(n))
      for (int n = 0; n < a.N; ++n) {
        float t = 0.f;
        for (int k = lane; k < a.R[n]; k += 32) t += sh.ev[sh.evoff[n] + k];
        trp *= warp_sum(t);
      }
      if (lane == 0) {
        sh.sum[2] = trp > 0.f ? fmaxf(t0 - t1, 0.f) / trp : 0.f;   // s
        sh.sum[3] = t1 / d;                                        // lbar
        // b is scaled by a power of two, 1 / max|b| rounded down, so that the FP32
        // iteration sees |b_j| <= 1 (no overflow of squares for large weights)
        int ex = 0;
        frexpf(t2, &ex);
        sh.bscale = t2 > 0.f ? ldexp(1.0, ex) : 0.0;
      }
    }
    __syncthreads();
  }
  const float sc = sh.sum[2], lbar = sh.sum[3];
  for (int e = tid; e < d; e += KP_THREADS) {
    float prod = sc;
    uint32_t rem = (uint32_t)e;
    for (int n = a.N - 1; n >= 0; --n) {               // e = row-major (r_1 .. r_N)
      const uint32_t qn = fdiv(rem, sh.div_r[n]);
      prod *= sh.ev[sh.evoff[n] + (int)(rem - qn * (uint32_t)sh.R[n])];
      rem = qn;
    }
    const float den = prod + lbar;
    v.dg[e] = den > 0.f ? 1.f / den : 0.f;
  }
  const float inv = sh.bscale > 0.0 ? (float)(1.0 / sh.bscale) : 0.f;
  float bb = 0.f;
#pragma unroll
  for (int t = 0; t < KP_BMAX; ++t) {
    const int j = tid + t * KP_THREADS;
    if (j < d) {
      const float b = bl[t] * inv;
      v.r[j] = b;
      v.x[j] = 0.f;
      v.p[j] = 0.f;
      v.q[j] = 0.f;
      bb = fmaf(b, b, bb);
    }
  }
  block_sums<1>(sh, bb, 0.f, 0.f);
  __syncthreads();
  return sh.sum[0];
}

// After s = M z is complete in shared memory: the CG scalars (one thread, FP32)
// and the vector updates; returns ||r||^2 (the same in every CTA), or -1 on a
// breakdown (alpha not positive and finite; x is kept as it is).
__device__ float kpcg_step(KpcgShared& sh, const KpcgVecs& v, const float* s, int d, int it,
                           float& gamma_old, float& alpha_old) {
  const int tid = threadIdx.x;
  float gz = 0.f, zs = 0.f;
  for (int e = tid; e < d; e += KP_THREADS) {
    gz = fmaf(v.r[e], v.z[e], gz);
    zs = fmaf(v.z[e], s[e], zs);
  }
  block_sums<2>(sh, gz, zs, 0.f);
  if (tid == 0) {                                      // the CG scalars, once per CTA
    const float gamma = sh.sum[0], delta = sh.sum[1];
    float alpha, beta;
    if (it == 0) {
      beta = 0.f;
      alpha = delta != 0.f ? gamma / delta : 0.f;
    } else {
      beta = gamma / gamma_old;
      const float den = delta - beta * gamma / alpha_old;
      alpha = den != 0.f ? gamma / den : 0.f;
    }
    sh.stop = !(alpha > 0.f) || !isfinite(alpha);
    gamma_old = gamma;
    alpha_old = alpha;
    sh.coef[0] = alpha;
    sh.coef[1] = beta;
  }
  __syncthreads();
  if (sh.stop) return -1.f;
  const float fa = sh.coef[0], fb = sh.coef[1];
  float r2 = 0.f;
  for (int e = tid; e < d; e += KP_THREADS) {
    const float pe = fmaf(fb, v.p[e], v.z[e]);
    const float qe = fmaf(fb, v.q[e], s[e]);
    v.p[e] = pe;
    v.q[e] = qe;
    v.x[e] = fmaf(fa, pe, v.x[e]);
    const float re = fmaf(-fa, qe, v.r[e]);
    v.r[e] = re;
    r2 = fmaf(re, re, r2);
  }
  block_sums<1>(sh, r2, 0.f, 0.f);
  __syncthreads();
  return sh.sum[0];
}

// Dot products of nr <= 4 consecutive rows (stride ld floats; global or
// shared, 16-byte aligned when vec) with z by one warp, the four chains
// interleaved so that their loads and shuffles overlap; every lane gets the
// sums.  Rows past nr give 0 and are not read.
__device__ __forceinline__ float4 rows_dot4(const float* m0, size_t ld, int nr, const float* z,
                                            int d, bool vec, bool global) {
  const int lane = threadIdx.x & 31;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  if (vec) {
    const float4* z4 = reinterpret_cast<const float4*>(z);
    for (int c = lane; c < (d >> 2); c += 32) {
      const float4 zv = z4[c];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j < nr) {
          const float4* m4 = reinterpret_cast<const float4*>(m0 + (size_t)j * ld);
          const float4 mv = global ? __ldg(m4 + c) : m4[c];
          acc[j] = fmaf(mv.x, zv.x, acc[j]); acc[j] = fmaf(mv.y, zv.y, acc[j]);
          acc[j] = fmaf(mv.z, zv.z, acc[j]); acc[j] = fmaf(mv.w, zv.w, acc[j]);
        }
      }
    }
  } else {
    for (int c = lane; c < d; c += 32) {
      const float zc = z[c];
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < nr) {
          const float* mr = m0 + (size_t)j * ld;
          acc[j] = fmaf(global ? __ldg(mr + c) : mr[c], zc, acc[j]);
        }
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  }
  return make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// Outputs of this CTA's rows: out = x and/or upd += x; returns the partial
// (||x||^2, ||upd||^2) of those rows in FP64 (warp sums, then a fixed-order
// shuffle tree over the warps; valid in thread 0).  upd0: upd[lo + tid], loaded
// by the caller before the iterations (its latency off this tail).
__device__ double2 kpcg_write(const KpcgArgs& a, const KpcgShared& sh, const KpcgVecs& v, int lo,
                             int hi, double upd0) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  double so = 0.0, su = 0.0;
  const double sc = sh.bscale;                         // undo the scaling of b
  for (int i = lo + tid; i < hi; i += KP_THREADS) {
    const double xi = (double)v.x[i] * sc;
    if (a.out) a.out[i] = xi;
    if (a.upd) {
      const double gn = (i == lo + tid ? upd0 : a.upd[i]) + xi;
      a.upd[i] = gn;
      so = fma(xi, xi, so);
      su = fma(gn, gn, su);
    }
  }
  so = warp_sum(so);
  su = warp_sum(su);
  __shared__ double wpart[2][KP_WARPS];
  if (lane == 0) { wpart[0][w] = so; wpart[1][w] = su; }
  __syncthreads();
  double2 t = make_double2(0.0, 0.0);
  if (w == 0) {
    double x = lane < KP_WARPS ? wpart[0][lane] : 0.0, y = lane < KP_WARPS ? wpart[1][lane] : 0.0;
    x = warp_sum(x);
    y = warp_sum(y);
    t = make_double2(x, y);
  }
  return t;
}

// Grid-wide version: C CTAs of one cooperative launch, M read from global
// memory (L2) every iteration, s exchanged through global memory.
__global__ void __launch_bounds__(KP_THREADS, 1) k_kpcg(KpcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) float kp_sm[];
  __shared__ KpcgShared sh;
  const int d = a.d;
  const int dp = (d + 3) & ~3;
  const KpcgVecs v = kpcg_carve(kp_sm, dp);
  int vtot = 0;
  for (int n = 0; n < a.N; ++n) vtot += a.R[n] * a.R[n];
  float* s = v.Vs + ((vtot + 3) & ~3);                // d floats: s of this iteration
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int C = gridDim.x;
  const int rows = (d + C - 1) / C;
  const int lo = min(d, (int)blockIdx.x * rows), hi = min(d, lo + rows);
  const double upd0 = (a.upd && lo + tid < hi) ? a.upd[lo + tid] : 0.0;
  const float bnorm2 = kpcg_setup(a, sh, v);
  const int pkind = precond_kind(a.N, a.R, d);
  const float stop2 = (float)(a.tol * a.tol) * bnorm2;
  float rr = bnorm2, gamma_old = 1.f, alpha_old = 1.f;
  int it = 0;
  const bool vec = (d & 3) == 0;
  for (; it < a.max_iter && rr > stop2; ++it) {
    precond_any(pkind, d, a.N, sh, v.Vs, v.dg, v.r, v.t0, v.t1, v.z);   // ends with a barrier
    float* sgk = a.sg + (size_t)(it & 1) * d;
    for (int i = lo + 4 * w; i < hi; i += 4 * KP_WARPS) {
      const int nr = min(4, hi - i);
      const float4 acc = rows_dot4(a.M + (size_t)i * d, (size_t)d, nr, v.z, d, vec, true);
      if (lane < nr) sgk[i + lane] = lane == 0 ? acc.x : lane == 1 ? acc.y : lane == 2 ? acc.z : acc.w;
    }
    grid.sync();                                       // every block of s published
    for (int e = tid; e < d; e += KP_THREADS) s[e] = __ldcg(sgk + e);
    __syncthreads();
    const float r2 = kpcg_step(sh, v, s, d, it, gamma_old, alpha_old);
    if (r2 < 0.f) break;
    rr = r2;
  }
  // every CTA read rhs before the first barrier, and a barrier follows here in
  // any case (rhs may alias out)
  grid.sync();
  const double2 t = kpcg_write(a, sh, v, lo, hi, upd0);
  if (a.res && blockIdx.x == 0 && tid == 0) {
    a.res[0] = (double)it;
    a.res[1] = bnorm2 > 0.f ? sqrt((double)rr / (double)bnorm2) : 0.0;
  }
  if (a.upd && a.stats) {
    if (tid == 0) {
      a.part[2 * blockIdx.x] = t.x;
      a.part[2 * blockIdx.x + 1] = t.y;
    }
    grid.sync();
    if (blockIdx.x == 0 && tid == 0) {
      double u = 0.0, vv = 0.0;
      for (int k = 0; k < C; ++k) { u += a.part[2 * k]; vv += a.part[2 * k + 1]; }
      a.stats[0] = u;
      a.stats[1] = vv;
    }
  }
}

// One-cluster version (small d): the C CTAs of one thread-block cluster keep
// their rows of M in shared memory, and each pushes its block of s = M z into
// every CTA's shared memory (distributed shared memory, double-buffered by
// iteration parity); one cluster barrier per iteration replaces the grid
// barrier and M is read from L2 once per solve.
constexpr int KPCL_CTAS = 8;

__global__ void __launch_bounds__(KP_THREADS, 1) k_kpcg_cluster(KpcgArgs a) {
  pdl_wait();
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ __align__(16) float kp_sm[];
  __shared__ KpcgShared sh;
  __shared__ double cpart[KPCL_CTAS][2];
  const int d = a.d;
  const int dp = (d + 3) & ~3;
  const KpcgVecs v = kpcg_carve(kp_sm, dp);
  int vtot = 0;
  for (int n = 0; n < a.N; ++n) vtot += a.R[n] * a.R[n];
  float* s2 = v.Vs + ((vtot + 3) & ~3);               // 2 x dp: s by iteration parity
  float* Mr = s2 + 2 * dp;                            // this CTA's rows of M, stride dp
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int C = (int)cl.num_blocks();
  const int me = (int)cl.block_rank();
  const int rows = (d + C - 1) / C;
  const int lo = min(d, me * rows), hi = min(d, lo + rows);
  const bool vec = (d & 3) == 0;
  // rows lo..hi of M into shared memory: with 16-byte rows they are one
  // contiguous block, copied by one bulk TMA transfer that overlaps the set-up
  // below; otherwise plain loads
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t mbytes = (uint32_t)((size_t)(hi - lo) * d * sizeof(float));
  const bool tma = vec && mbytes > 0;
  if (tma) {
    if (tid == 0) {
      mbar_init(&mbar, 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      mbar_expect_tx(&mbar, mbytes);
      bulk_g2s(Mr, a.M + (size_t)lo * d, mbytes, &mbar);
    }
  } else {
    for (int i = lo + w; i < hi; i += KP_WARPS) {
      const float* src = a.M + (size_t)i * d;
      float* dst = Mr + (size_t)(i - lo) * dp;
      for (int c = lane; c < d; c += 32) dst[c] = __ldg(src + c);
    }
  }
  const double upd0 = (a.upd && lo + tid < hi) ? a.upd[lo + tid] : 0.0;
  const float bnorm2 = kpcg_setup(a, sh, v);           // ends with a barrier
  if (tma) {                                           // bounded wait for the rows
    bool ok = false;
    for (uint32_t k = 0; k < KP_WAIT_LIMIT && !ok; ++k) ok = mbar_try(&mbar, 0);
    if (!ok) set_status(a.status, DEV_INTERNAL);       // reported by the host; no barrier skipped
  }
  cl.sync();                                          // every CTA running before remote stores
  const int pkind = precond_kind(a.N, a.R, d);
  const float stop2 = (float)(a.tol * a.tol) * bnorm2;
  float rr = bnorm2, gamma_old = 1.f, alpha_old = 1.f;
  int it = 0;
  for (; it < a.max_iter && rr > stop2; ++it) {
    precond_any(pkind, d, a.N, sh, v.Vs, v.dg, v.r, v.t0, v.t1, v.z);   // ends with a barrier
    float* sk = s2 + (size_t)(it & 1) * dp;
    for (int i = lo + 4 * w; i < hi; i += 4 * KP_WARPS) {
      const int nr = min(4, hi - i);
      const float4 acc = rows_dot4(Mr + (size_t)(i - lo) * dp, (size_t)dp, nr, v.z, d, vec, false);
      // lane = 4 * target CTA + row: the rows' sums into every CTA's buffer
      const int tc = lane >> 2, j = lane & 3;
      if (tc < C && j < nr)
        *cl.map_shared_rank(sk + i + j, tc) = j == 0 ? acc.x : j == 1 ? acc.y : j == 2 ? acc.z : acc.w;
    }
    cl.sync();                                        // every block of s in every CTA
    const float r2 = kpcg_step(sh, v, sk, d, it, gamma_old, alpha_old);
    if (r2 < 0.f) break;
    rr = r2;
  }
  cl.sync();                                          // rhs read everywhere (it may alias out)
  const double2 t = kpcg_write(a, sh, v, lo, hi, upd0);
  if (a.res && me == 0 && tid == 0) {
    a.res[0] = (double)it;
    a.res[1] = bnorm2 > 0.f ? sqrt((double)rr / (double)bnorm2) : 0.0;
  }
  if (a.upd && a.stats) {
    if (tid == 0) {
      double* dst = cl.map_shared_rank(&cpart[0][0], 0);
      dst[2 * me] = t.x;
      dst[2 * me + 1] = t.y;
    }
    cl.sync();
    if (me == 0 && tid == 0) {
      double u = 0.0, vv = 0.0;
      for (int k = 0; k < C; ++k) { u += cpart[k][0]; vv += cpart[k][1]; }
      a.stats[0] = u;
      a.stats[1] = vv;
    }
  }
}

size_t kpcg_smem_bytes(int d, int N, const int* R) {
  const size_t dp = (size_t)((d + 3) & ~3);
  int vtot = 0;
  for (int n = 0; n < N; ++n) vtot += R[n] * R[n];
  return (9 * dp + ((vtot + 3) & ~3)) * sizeof(float) + 64;
}

// The one-cluster kernel also holds two s buffers and its ceil(d / 8) rows of M.
static size_t kpcg_cluster_smem_bytes(int d, int N, const int* R) {
  const size_t dp = (size_t)((d + 3) & ~3);
  const size_t rows = (size_t)((d + KPCL_CTAS - 1) / KPCL_CTAS);
  int vtot = 0;
  for (int n = 0; n < N; ++n) vtot += R[n] * R[n];
  return ((10 + rows) * dp + ((vtot + 3) & ~3)) * sizeof(float) + 64;
}

constexpr size_t KP_SMEM_MAX = 220 * 1024;

// Whether the solver fits (shared memory for the d-vectors and the V_n).
int kpcg_fits(int d, int N, const int* R) { return kpcg_smem_bytes(d, N, R) <= KP_SMEM_MAX; }

// CTAs of one grid-wide solve: about 16 rows of M each, at most one per SM.
int kpcg_grid(tucker_handle* h, int d) {
  int c = (d + 15) / 16;
  if (c < 1) c = 1;
  if (c > h->num_sms) c = h->num_sms;
  return c;
}

static cudaLaunchConfig_t cluster_cfg(cudaLaunchAttribute* at, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = KPCL_CTAS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(KPCL_CTAS);
  cfg.blockDim = dim3(KP_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Whether the one-cluster kernel takes order d: its rows of M fit in shared
// memory and the device can schedule the cluster (asked once per size).
static bool kpcg_cluster_ok(int d, int N, const int* R) {
  const size_t smem = kpcg_cluster_smem_bytes(d, N, R);
  if (smem > KP_SMEM_MAX) return false;
  static size_t checked_ok = 0, checked_bad = ~size_t(0);
  if (smem <= checked_ok) return true;
  if (smem >= checked_bad) return false;
  if (cudaFuncSetAttribute(k_kpcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem) != cudaSuccess) {
    cudaGetLastError();
    checked_bad = smem;
    return false;
  }
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = cluster_cfg(at, smem, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, k_kpcg_cluster, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    checked_bad = smem;
    return false;
  }
  checked_ok = smem;
  return true;
}

// x = M^-1 rhs to relative residual tol (into out, and/or upd += x with the
// norms of the correction and of upd in stats).  V, ev: the factor Gram
// eigendecompositions; sg: 2 d floats; part: 2 * kpcg_grid doubles; res:
// nullable, (iterations, final relative residual).  One cluster for small d,
// else a cooperative grid.
tucker_status launch_kpcg(tucker_handle* h, const float* M, const double* regdiag, int d, int N,
                          const int* R, const double* const* V, const double* const* ev,
                          const double* rhs, double* out, double* upd, double* stats,
                          double* part, float* sg, double* res, double tol, int max_iter,
                          bool dep) {
  KpcgArgs a;
  memset(&a, 0, sizeof(a));
  a.M = M; a.regdiag = regdiag; a.d = d; a.N = N;
  int in = 1;
  for (int n = N - 1; n >= 0; --n) {
    a.R[n] = R[n];
    a.div_in[n] = make_fastdiv((uint32_t)in);
    a.div_r[n] = make_fastdiv((uint32_t)R[n]);
    in *= R[n];
    a.V[n] = V[n];
    a.ev[n] = ev[n];
  }
  for (int n = N; n < TUCKER_MAX_ORDER; ++n) a.div_in[n] = a.div_r[n] = make_fastdiv(1);
  a.rhs = rhs; a.out = out; a.upd = upd; a.stats = stats; a.part = part; a.sg = sg; a.res = res;
  a.tol = tol; a.max_iter = max_iter;
  a.status = h->d_status;
  if (kpcg_cluster_ok(d, N, R)) {
    const size_t smem = kpcg_cluster_smem_bytes(d, N, R);
    TK_CUDA(h, cudaFuncSetAttribute(k_kpcg_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_cfg(at, smem, h->stream);
    if (dep) {            // programmatic dependent launch (the kernel waits first)
      at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      at[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.numAttrs = 2;
    }
    TK_COUNT(h);
    TK_CUDA(h, cudaLaunchKernelEx(&cfg, k_kpcg_cluster, a));
    return TUCKER_OK;
  }
  const size_t smem = kpcg_smem_bytes(d, N, R);
  const void* kern = (const void*)k_kpcg;
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, KP_THREADS, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return fail(h, TUCKER_ECUDA, "CG solve cannot be resident (d = %d)", d);
  }
  const int grid = kpcg_grid(h, d);
  void* args[] = {&a};
  TK_COUNT(h);
  TK_CUDA(h, cudaLaunchCooperativeKernel(kern, grid, KP_THREADS, args, smem, h->stream));
  return TUCKER_OK;
}

}  // namespace tk
