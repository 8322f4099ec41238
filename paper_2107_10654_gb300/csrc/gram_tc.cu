// Tensor-core (tcgen05) Gram of the implicit Kronecker rows of the sample:
//     G = sum_u x_u x_u^T,   x_u = sqrt(w_u) * A^(1)[i_1] (x) ... (x) A^(N)[i_N]
// (the normal-equation matrix of Alg. 1's sketched least squares, formed as
// a sum of outer products as in the proof of Thm 4.2).  The design matrix is
// never stored: operand tiles of x are generated in shared memory.
//
// Work unit: one 256 x 256 tile of the upper triangle of G (two 128 x 256
// tcgen05 accumulators in TMEM, 512 columns) and one contiguous range of
// sample chunks (64 samples for BF16, 32 for TF32).
//   pack kernel  : per chunk, the factor rows of its samples laid out
//                  entry-major [e][s] (e over (n, r_n)) in FP32, sqrt(w) folded
//                  into mode 1; for BF16 the samples of each 8-sample group
//                  are split into two 16-byte halves so that lanes reading
//                  consecutive groups hit consecutive shared-memory banks;
//   producer warp: 1-D bulk TMA (cp.async.bulk) of each chunk block into a
//                  ring of table stages (mbarrier transaction counts);
//   builder warps: the 512 operand rows (256 of B = the tile's columns, 256
//                  of A = its rows; A is B on diagonal tiles) are cut into
//                  groups of 8 rows and, inside a group, into runs of rows
//                  that share (r_1, ..., r_{N-1}); a thread owns one (group,
//                  8-sample octet), forms p = prod_{n<N} a_n over the octet once
//                  per run and writes x = p * a_N[r_N] rounded once to BF16
//                  (or TF32) into K-major, 128-byte-swizzled operand rows;
//   MMA thread   : per chunk 2 x 4 tcgen05.mma (M = 128, N = 256, K = 16 or 8)
//                  into the two TMEM accumulators; tcgen05.commit frees the
//                  operand stage;
//   epilogue     : tcgen05.ld of both accumulators, FP32 partial tile to global.
// A reduction kernel sums the sample splits in a fixed order into the
// symmetric FP64 G.
// Every wait is bounded: on timeout the kernel records TUCKER_EINTERNAL,
// waits (bounded) for its MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace tk {

constexpr int TC_M = 128;          // rows of one MMA (TMEM lanes)
constexpr int TC_N = 256;          // columns of one MMA
constexpr int TC_TILE = 256;       // output tile edge (two accumulators)
constexpr int TC_ROWB = 128;       // bytes of K per operand row (one swizzle atom)
constexpr int TC_STAGES = 2;       // operand stages
constexpr int TC_BUILD_WARPS = 16;
constexpr int TC_THREADS = (TC_BUILD_WARPS + 2) * 32;   // + MMA warp + TMA warp
constexpr int TC_GROUPS = 2 * TC_TILE / 8;               // 8-row groups of B then A
constexpr int TC_TMEM_COLS = 512;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;

template <int PREC> struct TcTraits;
template <> struct TcTraits<TUCKER_PREC_BF16> {
  static constexpr int CS = 64;        // samples per chunk (128 bytes of BF16)
  static constexpr uint32_t FMT = 1;   // BF16 in the instruction descriptor
  static constexpr int KSTEPS = 4;     // MMAs of K = 16 per chunk
};
template <> struct TcTraits<TUCKER_PREC_TF32> {
  static constexpr int CS = 32;
  static constexpr uint32_t FMT = 2;   // TF32
  static constexpr int KSTEPS = 4;     // MMAs of K = 8 per chunk
};

// One run of rows inside an 8-row group: rows row0 .. row0 + n - 1 of the
// group have a_N columns t0 .. t0 + n - 1 and share the product of modes
// 1..N-1, whose table rows start at po[0..N-2] (element offsets into a chunk
// block).  zero: rows beyond d.
struct TcRun {
  uint8_t row0, n, t0, zero;
  int po[TUCKER_MAX_ORDER - 1];
  int pad;                         // 36 bytes: the 4 groups a warp reads fall in distinct banks
};

struct TcArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  int off[TUCKER_MAX_ORDER];          // entry offset of mode n in a chunk block
  int sumR;
  int d;
  int Tt;                              // tiles along each edge
  int ntiles;
  int nsplit;
  int tstages;                         // chunk-table stages
  const float* pack;                   // [chunks][sumR][CS]
  const int* n_rows;
  float* partial;                      // [nsplit][ntiles][256][256]
  int* status;
  const int* cstart;                   // nullable: first chunk of each split (grouped Gram)
  const int* ccount;                   // chunks of each split
};

// ------------------------------------------------------------ PTX wrappers
// Bounded wait on phase `parity`; false (and the status set) on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* status,
                                          volatile int* abort_flag) {
  for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i) {
    if (mbar_try(b, parity)) return true;
    if (*abort_flag) return false;
  }
  set_status(status, DEV_INTERNAL);
  *abort_flag = 1;
  return false;
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);          // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused, 16 B)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1 << 46;                           // version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}
// Instruction descriptor: FP32 accumulate, A/B format `fmt`, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_N >> 3) << 17) |
         ((uint32_t)(TC_M >> 4) << 24);
}
template <int PREC>
__device__ __forceinline__ void mma(uint32_t dtm, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (PREC == TUCKER_PREC_BF16)
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(dtm), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
  else
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(dtm), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(smem_u32(b)) : "memory");
}
// AND of `pred` over the builder warps (named barrier 1); also a barrier.
__device__ __forceinline__ bool builders_all(bool pred) {
  uint32_t r;
  asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
               "bar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
               : "=r"(r) : "r"((uint32_t)pred), "r"(TC_BUILD_WARPS * 32) : "memory");
  return r != 0;
}
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// ------------------------------------------------------------------ pack
// pack[q][e][pos(s)] = value e (mode n, column r) of sample q*CS + s; mode 1
// scaled by sqrt(w).  BF16: within each 64-sample chunk, sample s = 8c + j is
// stored at 4c + j (j < 4) or 32 + 4c + (j - 4) (j >= 4).
struct PackArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  int off[TUCKER_MAX_ORDER];
  int sumR;
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  const uint32_t* idx[TUCKER_MAX_ORDER];
  const double* w;
  const int* n_rows;
  int CS;
  int perm;
  float* pack;
};

__device__ __forceinline__ int pack_pos(int s, int perm) {
  if (!perm) return s;
  const int c = s >> 3, j = s & 7;
  return j < 4 ? 4 * c + j : 32 + 4 * c + (j - 4);
}

// Thread = (chunk q, element e, sample slot s) with s fastest: a CTA covers
// blockDim / CS whole (q, e) rows, so the index arithmetic is one 32-bit
// division per output (the host keeps nch * sumR below 2^31).
__global__ void k_tc_pack(PackArgs a) {
  const int nrows = *a.n_rows;
  const int nch = (nrows + a.CS - 1) / a.CS;
  const int nrow_total = nch * a.sumR;                     // (chunk, element) rows
  const int per_cta = blockDim.x / a.CS;
  const int s = threadIdx.x % a.CS;
  for (int row = blockIdx.x * per_cta + threadIdx.x / a.CS; row < nrow_total;
       row += gridDim.x * per_cta) {
    const int q = row / a.sumR, e = row - q * a.sumR;
    const int64_t u = (int64_t)q * a.CS + s;
    float v = 0.f;
    if (u < nrows) {
      int n = 0;
      while (n + 1 < a.N && e >= a.off[n + 1]) ++n;
      const int r = e - a.off[n];
      const float f = (float)load_as_double(a.A[n], (int64_t)a.idx[n][u] * a.R[n] + r, a.is64);
      v = n == 0 ? sqrtf((float)a.w[u]) * f : f;     // FP32 is exact enough: rounded to BF16/TF32 next
    }
    a.pack[(int64_t)row * a.CS + pack_pos(s, a.perm)] = v;
  }
}

__device__ __forceinline__ void tile_of(int tile, int Tt, int* ti, int* tj) {
  // upper tiles (ti <= tj), column-major packed: tile = tj (tj + 1) / 2 + ti
  int j = (int)((sqrtf(8.0f * tile + 1.0f) - 1.0f) * 0.5f);
  while ((j + 1) * (j + 2) / 2 <= tile) ++j;
  while (j * (j + 1) / 2 > tile) --j;
  *tj = j;
  *ti = tile - j * (j + 1) / 2;
}

// ------------------------------------------ Gram grouped by the leading index
// With the sample sorted by key, rows of one i_1 are contiguous and
//   G = sum_u w_u k_u k_u^T = sum_{i_1} (a a^T) (x) M_{i_1},  a = A^(1)[i_1],
//   M_{i_1} = sum_{u: i_1(u) = i_1} w_u b_u b_u^T,  b_u = a_2 (x) ... (x) a_N
// (k_u = a (x) b_u, row-major vec with r_1 outermost).  The tensor-core kernel
// forms every M_{i_1} as its own split (operands from modes 2..N, d / R_1
// wide; each segment padded to whole chunks with zero rows), and a reduction
// forms G_{(r1,j),(r1',j')} = sum_{i_1} a_{r1} a_{r1'} M_{i_1}[j][j'].  The
// tensor-core work falls by R_1^2 for the price of the reduction's
// (d / R_1)^2 / 2 x I_1 x R_1^2 FP32 multiply-adds.

// Segment table of the sorted rows (seg_begin / seg_end zeroed beforehand).
__global__ void k_tcg_segments(const uint32_t* idx0, const int* n_rows, int* seg_begin,
                               int* seg_end) {
  const int n = *n_rows;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    const uint32_t v = idx0[u];
    if (u == 0 || idx0[u - 1] != v) seg_begin[v] = u;
    if (u == n - 1 || idx0[u + 1] != v) seg_end[v] = u + 1;
  }
}

// Chunks per segment, their exclusive prefix sum and the chunk -> segment map
// (one CTA; I_1 is bounded by the caller).
__global__ void __launch_bounds__(1024) k_tcg_chunks(const int* seg_begin, const int* seg_end,
                                                      int I1, int CS, int* cstart, int* ccount,
                                                      int* cseg) {
  __shared__ int64_t tmp[32];
  int64_t carry = 0;
  for (int base = 0; base < I1; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int c = i < I1 ? (seg_end[i] - seg_begin[i] + CS - 1) / CS : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan(c, tmp, &tot);
    if (i < I1) {
      cstart[i] = (int)(carry + ex);
      ccount[i] = c;
      for (int k = 0; k < c; ++k) cseg[carry + ex + k] = i;
    }
    carry += tot;
  }
}

// Operand table of the grouped Gram: chunk c of segment i_1 holds rows
// seg_begin + (c - cstart) CS + s (zero past the segment), modes 2..N, sqrt(w)
// folded into mode 2.  nch_max bounds the chunk count (the rest is not read).
__global__ void k_tc_pack_grouped(PackArgs a, const int* seg_begin, const int* seg_end,
                                  const int* cstart, const int* cseg, int nch_max) {
  const int nrow_total = nch_max * a.sumR;
  const int per_cta = blockDim.x / a.CS;
  const int s = threadIdx.x % a.CS;
  for (int row = blockIdx.x * per_cta + threadIdx.x / a.CS; row < nrow_total;
       row += gridDim.x * per_cta) {
    const int q = row / a.sumR, e = row - q * a.sumR;
    const int i1 = cseg[q];
    float v = 0.f;
    if (i1 >= 0) {
      const int64_t u = (int64_t)seg_begin[i1] + (int64_t)(q - cstart[i1]) * a.CS + s;
      if (u < seg_end[i1]) {
        int n = 0;
        while (n + 1 < a.N && e >= a.off[n + 1]) ++n;
        const int r = e - a.off[n];
        const float f = (float)load_as_double(a.A[n], (int64_t)a.idx[n][u] * a.R[n] + r, a.is64);
        v = n == 0 ? sqrtf((float)a.w[u]) * f : f;
      }
    }
    a.pack[(int64_t)row * a.CS + pack_pos(s, a.perm)] = v;
  }
}

// G_{(r1,j),(r1',j')} = sum_{i_1} a_{r1} a_{r1'} M_{i_1}[j][j'] on the tensor
// cores: with p = (r1, r1') and n = (j, j'), G_pairs = P M, where
// P[p][i_1] = a_{r1} a_{r1'} (R_1^2 x I_1) and M[i_1][n] are the FP32 partial
// tiles (I_1 x (d/R_1)^2), a contraction over i_1.  Work unit: one 16 x 16
// block (j, j') of M in the block-upper triangle (n = 16 jj + jj', the 256
// columns of one MMA) and 128 pairs p (one TMEM accumulator; R_1 = 16 takes
// two CTAs per block).  Per chunk of 32 values of i_1 the 256 threads stage,
// K-major with the 128-byte swizzle, the block's M entries and the pairs' P
// values, each split as x = hi + lo with hi = tf32(x) and lo = tf32(x - hi);
// one thread issues Ph Mh + Ph Ml + Pl Mh (the dropped Pl Ml is 2^-22
// relative).  P must not be rounded once: its error would repeat for every
// sample of one i_1 instead of averaging out like the Gram's own rounding.
// P is the same for (r1, r1') and (r1', r1).  Each entry of G is computed
// once and stored with its mirror: (r1, j; r1', j') for j < j', and for j = j'
// when r1 <= r1'.  The output goes through shared memory so that 16 lanes
// store 16 consecutive doubles, both for the entry and for its mirror.
constexpr int EX_THREADS = 256;
constexpr int EX_KC = 32;                        // i_1 values per chunk (128 bytes of TF32)
constexpr int EX_OP = TC_TILE * TC_ROWB;         // one 256-row operand: 32 KB
constexpr int EX_STAGE = 3 * EX_OP;              // M hi, M lo, P hi and P lo (16 KB each)
constexpr int EX_PS = 16 * 17 + 1;               // staged pair row: 16 rows of 17 floats, + 1

struct ExpandArgs {
  const float* partial;                          // [I1][ntiles][256][256]
  int I1, ntiles, nb, dp, R1, d;                 // nb: 16-blocks per edge of M
  const void* A1;
  int is64;
  double* G;
  int* status;
};

__device__ __forceinline__ bool ex_wait(uint64_t* b, uint32_t parity, int* status) {
  bool ok = false;
  for (uint32_t i = 0; i < TC_WAIT_LIMIT && !ok; ++i) ok = mbar_try(b, parity);
  if (!ok) set_status(status, DEV_INTERNAL);
  return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(EX_THREADS, 1) k_tcg_expand(ExpandArgs a) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const uint32_t base_u = smem_u32(smraw);
  unsigned char* sm = smraw + ((1024 - (base_u & 1023)) & 1023);
  float* a1s = reinterpret_cast<float*>(sm + 2 * EX_STAGE);     // [2][EX_KC][R1]
  __shared__ uint64_t bar_free[2], bar_done;
  __shared__ uint32_t tmem_slot;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  int bj, bjp;
  tile_of(blockIdx.x, a.nb, &bj, &bjp);                        // bj <= bjp
  const int ti = bj >> 4, tj = bjp >> 4;                       // the partial tile of the block
  const size_t tstride = (size_t)a.ntiles * (TC_TILE * TC_TILE);
  const float* src = a.partial + (size_t)(tj * (tj + 1) / 2 + ti) * (TC_TILE * TC_TILE) +
                     (size_t)((bj & 15) * 16) * TC_TILE + (bjp & 15) * 16;
  const int R1 = a.R1, P2 = R1 * R1;
  const int mb = blockIdx.y;                                   // pairs 128 mb .. 128 mb + 127
  constexpr uint32_t ncols = 256u;
  if (t == 0) {
    mbar_init(&bar_free[0], 1);
    mbar_init(&bar_free[1], 1);
    mbar_init(&bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // staging map: rows n = 16 jj + 4 jq + k (k < 4), i_1 = 8 ig + i (i < 8) of the chunk
  const int jq = t & 3, ig = (t >> 2) & 3, jj = t >> 4;
  const float* srow = src + (size_t)jj * TC_TILE + 4 * jq;
  const int nk = (a.I1 + EX_KC - 1) / EX_KC;
  float4 cur[8], nxt[8];
  float acur[2], anxt[2];
  auto load_chunk = [&](int k, float4* v, float* av) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int i1 = k * EX_KC + 8 * ig + i;
      v[i] = i1 < a.I1 ? __ldg(reinterpret_cast<const float4*>(srow + (size_t)i1 * tstride))
                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {                              // A^(1) rows of the chunk
      const int e = t + q * EX_THREADS, i1 = k * EX_KC + e / R1;
      av[q] = e < EX_KC * R1 && i1 < a.I1
                  ? (float)load_as_double(a.A1, (int64_t)i1 * R1 + e % R1, a.is64) : 0.f;
    }
  };
  load_chunk(0, cur, acur);
  bool ok = true;
  for (int k = 0; k < nk && ok; ++k) {
    const int s = k & 1;
    unsigned char* hi = sm + (size_t)s * EX_STAGE;
    unsigned char* lo = hi + EX_OP;
    unsigned char* pp = lo + EX_OP;
    float* as = a1s + s * EX_KC * R1;
    if (k >= 2) ok = ex_wait(&bar_free[s], ((k - 2) >> 1) & 1, a.status);   // MMAs of chunk k - 2
    if (!ok) break;
    if (k + 1 < nk) load_chunk(k + 1, nxt, anxt);
#pragma unroll
    for (int q = 0; q < 2; ++q)
      if (t + q * EX_THREADS < EX_KC * R1) as[t + q * EX_THREADS] = acur[q];
    // M rows: 4 rows x 8 consecutive i_1 = two 16-byte chunks of each row, hi and lo
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int n = 16 * jj + 4 * jq + r;
      const size_t rowoff = (size_t)(n >> 3) * 1024 + (n & 7) * TC_ROWB;
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 c = cur[4 * h2 + i];
          v[i] = r == 0 ? c.x : r == 1 ? c.y : r == 2 ? c.z : c.w;
        }
        uint4 vh, vl;
        vh.x = to_tf32(v[0]); vl.x = to_tf32(v[0] - __uint_as_float(vh.x));
        vh.y = to_tf32(v[1]); vl.y = to_tf32(v[1] - __uint_as_float(vh.y));
        vh.z = to_tf32(v[2]); vl.z = to_tf32(v[2] - __uint_as_float(vh.z));
        vh.w = to_tf32(v[3]); vl.w = to_tf32(v[3] - __uint_as_float(vh.w));
        const int chunk = (2 * ig + h2) ^ (n & 7);
        *reinterpret_cast<uint4*>(hi + rowoff + (chunk << 4)) = vh;
        *reinterpret_cast<uint4*>(lo + rowoff + (chunk << 4)) = vl;
      }
    }
    __syncthreads();                                           // A^(1) rows of the chunk
    // P rows: pair p = 128 mb + (t % 128) (zero past R1^2), 16-byte chunks 4 (t / 128) ..
    {
      const int pl = t & 127, p = mb * 128 + pl;
      const size_t rowoff = (size_t)(pl >> 3) * 1024 + (pl & 7) * TC_ROWB;
      const int r1 = p / R1, r2 = p - r1 * R1;
#pragma unroll
      for (int c = 4 * (t >> 7); c < 4 * (t >> 7) + 4; ++c) {
        uint4 oh = make_uint4(0u, 0u, 0u, 0u), ol = oh;
        if (p < P2) {
          const float* a0 = as + (4 * c) * R1;
          float v[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) v[i] = a0[i * R1 + r1] * a0[i * R1 + r2];
          oh.x = to_tf32(v[0]); ol.x = to_tf32(v[0] - __uint_as_float(oh.x));
          oh.y = to_tf32(v[1]); ol.y = to_tf32(v[1] - __uint_as_float(oh.y));
          oh.z = to_tf32(v[2]); ol.z = to_tf32(v[2] - __uint_as_float(oh.z));
          oh.w = to_tf32(v[3]); ol.w = to_tf32(v[3] - __uint_as_float(oh.w));
        }
        const size_t o = rowoff + ((c ^ (pl & 7)) << 4);
        *reinterpret_cast<uint4*>(pp + o) = oh;
        *reinterpret_cast<uint4*>(pp + TC_M * TC_ROWB + o) = ol;
      }
    }
    fence_proxy_async();                                       // generic writes -> tensor core
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t id = idesc(2u);                           // TF32, M = 128, N = 256
      const uint32_t bh = smem_u32(hi), bl = smem_u32(lo), ph = smem_u32(pp);
      const uint32_t pl = ph + (uint32_t)(TC_M * TC_ROWB);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {                         // 8 values of i_1 per MMA
        mma<TUCKER_PREC_TF32>(tmem, sw128_desc(ph + 32 * kk), sw128_desc(bh + 32 * kk), id,
                              (k > 0 || kk > 0) ? 1u : 0u);
        mma<TUCKER_PREC_TF32>(tmem, sw128_desc(ph + 32 * kk), sw128_desc(bl + 32 * kk), id, 1u);
        mma<TUCKER_PREC_TF32>(tmem, sw128_desc(pl + 32 * kk), sw128_desc(bh + 32 * kk), id, 1u);
      }
      mma_commit(&bar_free[s]);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) cur[i] = nxt[i];
    acur[0] = anxt[0];
    acur[1] = anxt[1];
  }
  if (t == 0) mma_commit(&bar_done);                           // tracks every MMA issued
  const bool done = ex_wait(&bar_done, 0, a.status);
  tc_fence_after();
  // ---------------- epilogue through shared memory
  float* S = reinterpret_cast<float*>(sm);                     // [128 pairs][EX_PS]
  const bool diagb = bj == bjp;
  if (done && ok) {
    // TMEM -> S: warp w reads lanes 32 (w % 4).. and column half (w / 4) * 128..
    const int quad = warp & 3, half = warp >> 2;
    const int pl = quad * 32 + lane;
#pragma unroll 1
    for (int cb = 0; cb < 128; cb += 16) {
      const int col = half * 128 + cb;                         // = 16 jj: one row of the block
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                     "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                     "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                   : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float* dst = S + (size_t)pl * EX_PS + (col >> 4) * 17;
#pragma unroll
      for (int i = 0; i < 16; ++i) dst[i] = __uint_as_float(v[i]);
    }
    __syncthreads();
    // S -> G: item (pair, row) with 16 lanes along the row; entry rows jj, mirror rows jj'
    const int sub = lane >> 4, l16 = lane & 15;
    for (int item = warp * 2 + sub; item < 128 * 16 * 2; item += (EX_THREADS / 32) * 2) {
      const int pl2 = item >> 5, mode = (item >> 4) & 1, q = item & 15;
      const int p = mb * 128 + pl2;
      if (p >= P2) continue;
      const int r1 = p / R1, r2 = p - r1 * R1;
      // mode 0: jj = q, jj' = l16 (the entry); mode 1: jj' = q, jj = l16 (the mirror)
      const int jjv = mode ? l16 : q, jjp = mode ? q : l16;
      const int j = 16 * bj + jjv, jp = 16 * bjp + jjp;
      if (j >= a.dp || jp >= a.dp) continue;
      if (diagb && (jjv > jjp || (jjv == jjp && r1 > r2))) continue;
      const double v = (double)S[(size_t)pl2 * EX_PS + jjv * 17 + jjp];
      const size_t A = (size_t)r1 * a.dp + j, B = (size_t)r2 * a.dp + jp;
      if (mode == 0) a.G[A * a.d + B] = v;
      else a.G[B * a.d + A] = v;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols)
                 : "memory");
  }
}

// ------------------------------- the grouped Gram with narrow M_{i_1} (d / R_1 <= 64)
// Same decomposition, G = sum_{i_1} (a a^T) (x) M_{i_1}, for d' = d / R_1 <= 64,
// where a 256-wide tile would be mostly padding.  The rows of each i_1 segment
// are cut into pieces of at most 256 rows, and one CTA per piece forms the
// piece's share of M_{i_1} on the tensor cores from its rows
// b_u = sqrt(w_u) a_2 (x) ... (x) a_N (built in FP32), each split as
// b = b_hi + b_lo (TF32 both): with
//   A = [B_hi^T; B_lo^T] (128 x K: rows j and 64 + j),  B = B_hi^T (64 x K)
// one M = 128, N = 64 MMA per 8 samples gives D = [B_hi^T B_hi; B_lo^T B_hi] and
//   M[j][j'] = D[j][j'] + D[64 + j][j'] + D[64 + j'][j]
// (the dropped B_lo^T B_lo is 2^-22 relative), as accurate as an FP32 Gram.
// The piece's factor rows and weights are loaded into shared memory at once
// (every load of the piece in flight together), so a piece costs about one
// memory latency plus its MMAs, and no CTA waits on a long segment.  The
// expansion by a_{r1} a_{r1'} is a small contraction over the pieces
// (I_1 R_1^2 d'^2 / 2 multiply-adds and then some), done on the CUDA cores in FP32.
constexpr int NR_THREADS = 256;
constexpr int NR_WARPS = NR_THREADS / 32;
constexpr int NR_KC = 32;                        // samples per chunk (128 bytes of TF32)
constexpr int NR_PR = 256;                       // rows of one piece (8 chunks)
constexpr int NR_OP = TC_M * TC_ROWB;            // one 128-row operand stage: 16 KB
constexpr int NR_COLS = 64;                      // TMEM columns (N of the MMA)
constexpr int NR_DS = 65;                        // epilogue row stride (floats)
constexpr int NR_MAXE = 96;                      // table row: sum R_n (n >= 2) + 1 <= 3 x 32

struct NarrowArgs {
  int nm;                                        // modes 2..N: nm = N - 1 of them
  int R[TUCKER_MAX_ORDER];
  int off[TUCKER_MAX_ORDER];                     // entry offset of mode n in a table row
  int sumR;                                      // table row: sumR factor values + sqrt(w)
  int dp;
  const void* A[TUCKER_MAX_ORDER];
  const uint32_t* idx[TUCKER_MAX_ORDER];
  int is64;
  const double* w;
  const int* prow0;                              // [pieces] first row of each piece
  const int* prow1;                              // [pieces] end row
  const int* npieces;                            // [1]
  float* Mp;                                     // [pieces][dp][dp]
  int* status;
};

static size_t narrow_smem_bytes(int sumR, int nm) {
  const size_t body = 2 * (size_t)NR_OP + (size_t)NR_PR * (sumR + 1) * 4 + (size_t)nm * NR_PR * 4;
  const size_t epi = (size_t)TC_M * NR_DS * 4;
  return std::max(body, epi) + 1024;
}

// Pieces of at most NR_PR rows of every i_1 segment, in order of i_1 (one CTA).
__global__ void __launch_bounds__(1024) k_tcg_pieces(const int* seg_begin, const int* seg_end,
                                                      int I1, int* prow0, int* prow1, int* pseg,
                                                      int* npieces) {
  pdl_wait();
  __shared__ int64_t tmp[32];
  int64_t carry = 0;
  for (int base = 0; base < I1; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int b0 = i < I1 ? seg_begin[i] : 0, b1 = i < I1 ? seg_end[i] : 0;
    const int c = (b1 - b0 + NR_PR - 1) / NR_PR;
    int64_t tot;
    const int64_t ex = block_exclusive_scan(c, tmp, &tot);
    for (int k = 0; k < c; ++k) {
      const int64_t q = carry + ex + k;
      prow0[q] = b0 + k * NR_PR;
      prow1[q] = min(b1, b0 + (k + 1) * NR_PR);
      pseg[q] = i;
    }
    carry += tot;
  }
  if (threadIdx.x == 0) *npieces = (int)carry;
}

// NMT: the number of trailing modes when known at compile time (2 or 3), else 0.
template <int NMT>
__global__ void __launch_bounds__(NR_THREADS, 4) k_tcg_narrow(NarrowArgs a) {
  pdl_wait();
  constexpr int NMX = NMT > 0 ? NMT : TUCKER_MAX_ORDER - 1;
  extern __shared__ __align__(1024) unsigned char smraw[];
  const uint32_t base_u = smem_u32(smraw);
  unsigned char* sm = smraw + ((1024 - (base_u & 1023)) & 1023);
  const int E = a.sumR + 1, dp = a.dp;
  float* tab = reinterpret_cast<float*>(sm + 2 * NR_OP);        // [NR_PR][E]
  __shared__ uint64_t bar_free[2], bar_done;
  __shared__ uint32_t tmem_slot;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int p = blockIdx.x;
  if (p >= *a.npieces) return;                                 // the grid is an upper bound
  const int b0 = a.prow0[p], b1 = a.prow1[p];
  const int nk = (b1 - b0 + NR_KC - 1) / NR_KC;                // 1 .. NR_PR / NR_KC
  float* Mo = a.Mp + (size_t)p * dp * dp;
  if (t == 0) {
    mbar_init(&bar_free[0], 1);
    mbar_init(&bar_free[1], 1);
    mbar_init(&bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"((uint32_t)NR_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the table of the piece: row s (sample b0 + s) holds the factor entries of
  // modes 2..N and sqrt(w).  Two rounds of loads: the rows' indices into shared
  // memory (one per thread and mode), then every entry at once (lane = entry,
  // warp = rows w + 8 i, all 32 rows of a warp in flight together).
  {
    uint32_t* sidx = reinterpret_cast<uint32_t*>(sm + 2 * NR_OP + (size_t)NR_PR * E * 4);
    const int nrow = nk * NR_KC;
    for (int q = t; q < a.nm * NR_PR; q += NR_THREADS) {
      const int n = q / NR_PR, s = q - n * NR_PR;
      const int u = b0 + s;
      sidx[q] = (s < nrow && u < b1) ? __ldg(a.idx[n] + u) : 0u;
    }
    __syncthreads();
    for (int z = 0; z * 32 < E; ++z) {
      const int e = lane + 32 * z;
      const bool on = e < E, isw = e == a.sumR;
      int n = 0;
      while (n + 1 < a.nm && e >= a.off[n + 1]) ++n;
      const void* ap = a.A[n];
      const int rn = a.R[n], rr = e - a.off[n];
      const uint32_t* si = sidx + n * NR_PR;
      float xv[NR_PR / NR_WARPS];
#pragma unroll
      for (int i = 0; i < NR_PR / NR_WARPS; ++i) {
        const int s = warp + NR_WARPS * i, u = b0 + s;
        float x = 0.f;
        if (on && s < nrow && u < b1)
          x = isw ? sqrtf((float)__ldg(a.w + u))
                  : (float)load_as_double(ap, (int64_t)si[s] * rn + rr, a.is64);
        xv[i] = x;
      }
#pragma unroll
      for (int i = 0; i < NR_PR / NR_WARPS; ++i) {
        const int s = warp + NR_WARPS * i;
        if (on && s < nrow) tab[s * E + e] = xv[i];
      }
    }
  }
  tc_fence_before();
  __syncthreads();                                             // the table, TMEM address
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // the two build units of this thread: operand row j (and 64 + j), 16-byte chunk q
  int eo[2][NMX];
  bool live[2];
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    int j = (t + NR_THREADS * h2) & 63;
    live[h2] = j < dp;
#pragma unroll
    for (int n = NMX - 1; n >= 0; --n) {
      eo[h2][n] = 0;
      if (NMT > 0 || n < a.nm) {
        eo[h2][n] = a.off[n] + j % a.R[n];
        j /= a.R[n];
      }
    }
  }
  const uint32_t id = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NR_COLS >> 3) << 17) |
                      ((uint32_t)(TC_M >> 4) << 24);           // TF32, M = 128, N = 64
  bool ok = true;
  for (int k = 0; k < nk && ok; ++k) {
    const int st = k & 1;
    unsigned char* op = sm + (size_t)st * NR_OP;
    if (k >= 2) ok = ex_wait(&bar_free[st], ((k - 2) >> 1) & 1, a.status);  // chunk k - 2's MMAs
    if (!ok) break;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int uu = t + NR_THREADS * h2, j = uu & 63, q = uu >> 6;
      uint4 vh = make_uint4(0u, 0u, 0u, 0u), vl = vh;
      if (live[h2]) {
        float x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float* row = tab + (k * NR_KC + 4 * q + i) * E;
          float pr = row[a.sumR];
#pragma unroll
          for (int n = 0; n < NMX; ++n)
            if (NMT > 0 || n < a.nm) pr *= row[eo[h2][n]];
          x[i] = pr;
        }
        vh.x = to_tf32(x[0]); vl.x = to_tf32(x[0] - __uint_as_float(vh.x));
        vh.y = to_tf32(x[1]); vl.y = to_tf32(x[1] - __uint_as_float(vh.y));
        vh.z = to_tf32(x[2]); vl.z = to_tf32(x[2] - __uint_as_float(vh.z));
        vh.w = to_tf32(x[3]); vl.w = to_tf32(x[3] - __uint_as_float(vh.w));
      }
      const int rl = 64 + j;                                   // j & 7 == rl & 7
      const int c = (q ^ (j & 7)) << 4;
      *reinterpret_cast<uint4*>(op + (size_t)(j >> 3) * 1024 + (j & 7) * TC_ROWB + c) = vh;
      *reinterpret_cast<uint4*>(op + (size_t)(rl >> 3) * 1024 + (rl & 7) * TC_ROWB + c) = vl;
    }
    fence_proxy_async();                                       // generic writes -> tensor core
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t ob = smem_u32(op);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk)                           // 8 samples per MMA
        mma<TUCKER_PREC_TF32>(tmem, sw128_desc(ob + 32 * kk), sw128_desc(ob + 32 * kk), id,
                              (k > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&bar_free[st]);
    }
  }
  if (t == 0) mma_commit(&bar_done);                           // tracks every MMA issued
  const bool done = ex_wait(&bar_done, 0, a.status);
  tc_fence_after();
  float* D = reinterpret_cast<float*>(sm);                     // [128][NR_DS]
  if (done && ok) {
    // TMEM -> D: warp w reads lanes 32 (w % 4) .. and columns 32 (w / 4) ..
    const int quad = warp & 3, half = warp >> 2, row = quad * 32 + lane;
#pragma unroll
    for (int cb = 0; cb < 32; cb += 16) {
      const int col = half * 32 + cb;
      uint32_t v[16];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                   "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                   : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                     "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                     "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                   : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) D[row * NR_DS + col + i] = __uint_as_float(v[i]);
    }
    __syncthreads();
    for (int j = warp; j < dp; j += NR_WARPS)                  // row j of M: lanes along j'
      for (int jp = lane; jp < dp; jp += 32)
        Mo[j * dp + jp] = D[j * NR_DS + jp] + D[(64 + j) * NR_DS + jp] + D[(64 + jp) * NR_DS + j];
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;"
                 ::"r"(tmem), "r"((uint32_t)NR_COLS) : "memory");
  }
}

// G_{(r1,j),(r2,j')} = sum_{pieces} a_{r1} a_{r2} M_piece[j][j'] (a = A^(1) row of
// the piece's i_1) in FP32 on the CUDA cores.  CTA: 32 entries (j <= j', the
// upper triangle of M in row-major order) x 32 pairs (r1, r2) (pairs 32 y ..
// 32 y + 31); warp w sums the w-th of 16 contiguous ranges of pieces, sixteen
// pieces' loads in flight, and the 16 partials are added in a fixed order, so
// the result does not depend on scheduling.  Writes each entry of G and its
// mirror (for j = j' only the pairs r1 <= r2, so G is exactly symmetric).
constexpr int XN_WARPS = 16;

template <int R1>
__global__ void __launch_bounds__(XN_WARPS * 32) k_tcg_expand_narrow(const float* Mp,
                                                                     const int* pseg,
                                                                     const int* npieces, int I1,
                                                                     int dp, const void* A1,
                                                                     int is64, int d, double* G) {
  pdl_wait();
  extern __shared__ float xs[];
  float* a1 = xs;                                              // [I1][R1]
  float* red = xs + ((I1 * R1 + 3) & ~3);                      // [16][32][32]
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int i = t; i < I1 * R1; i += XN_WARPS * 32)
    a1[i] = (float)load_as_double(A1, i, is64);
  // entry e -> (j, j'): rows j hold dp - j entries
  const int ne = dp * (dp + 1) / 2;
  const int e = blockIdx.x * 32 + lane;
  int j = 0, jp = 0;
  if (e < ne) {
    int start = 0;
    while (start + (dp - j) <= e) { start += dp - j; ++j; }
    jp = j + (e - start);
  }
  constexpr int NP = R1 * R1 < 32 ? R1 * R1 : 32;              // pairs of this CTA
  constexpr int NR = NP / R1 > 0 ? NP / R1 : 1;                // values of r1 among them
  const int r1b = blockIdx.y * 32 / R1;
  const int P = *npieces;
  __syncthreads();
  float acc[NP];
#pragma unroll
  for (int c = 0; c < NP; ++c) acc[c] = 0.f;
  const int pb = (int)((int64_t)P * warp / XN_WARPS), pe = (int)((int64_t)P * (warp + 1) / XN_WARPS);
  const size_t msz = (size_t)dp * dp;
  const float* mp = Mp + (size_t)j * dp + jp;
  constexpr int XB = 16;                                       // pieces' loads in flight
  for (int p0 = pb; p0 < pe; p0 += XB) {
    float m[XB];
    int seg[XB];
#pragma unroll
    for (int q = 0; q < XB; ++q) {
      const int pq = p0 + q;
      seg[q] = pq < pe ? __ldg(pseg + pq) : 0;
      m[q] = (pq < pe && e < ne) ? __ldg(mp + (size_t)pq * msz) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < XB; ++q) {
      if (p0 + q >= pe) break;
      const float* ar = a1 + seg[q] * R1;
      float tq[R1];
#pragma unroll
      for (int r = 0; r < R1; ++r) tq[r] = ar[r] * m[q];
      float ap[NR];
#pragma unroll
      for (int r = 0; r < NR; ++r) ap[r] = ar[r1b + r];
#pragma unroll
      for (int c = 0; c < NP; ++c) acc[c] = fmaf(ap[c / R1], tq[c % R1], acc[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < NP; ++c) red[(warp * 32 + c) * 32 + lane] = acc[c];
  __syncthreads();
  for (int o = t; o < NP * 32; o += XN_WARPS * 32) {
    const int c = o >> 5, le = o & 31;
    const int eo = blockIdx.x * 32 + le;
    if (eo >= ne) continue;
    float v = 0.f;
    for (int w = 0; w < XN_WARPS; ++w) v += red[(w * 32 + c) * 32 + le];
    int jj = 0, start = 0;
    while (start + (dp - jj) <= eo) { start += dp - jj; ++jj; }
    const int jjp = jj + (eo - start);
    const int r1 = r1b + c / R1, r2 = c % R1;
    if (jj == jjp && r1 > r2) continue;
    const size_t A = (size_t)r1 * dp + jj, B = (size_t)r2 * dp + jjp;
    G[A * d + B] = (double)v;
    G[B * d + A] = (double)v;
  }
}

// --------------------------------------------------------------- the SYRK

template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_syrk_tc(TcArgs a) {
  using Tr = TcTraits<PREC>;
  constexpr int CS = Tr::CS;
  extern __shared__ __align__(1024) unsigned char smraw[];
  const uint32_t base_u = smem_u32(smraw);
  unsigned char* sm = smraw + ((1024 - (base_u & 1023)) & 1023);
  unsigned char* opA = sm;                                          // STAGES x 256 rows x 128 B
  unsigned char* opB = opA + TC_STAGES * TC_TILE * TC_ROWB;         // STAGES x 256 rows x 128 B
  float* tab = reinterpret_cast<float*>(opB + TC_STAGES * TC_TILE * TC_ROWB);
  const int tab_elems = a.sumR * CS;
  TcRun* runs = reinterpret_cast<TcRun*>(tab + (size_t)a.tstages * tab_elems);   // [groups][8]
  uint8_t* nruns = reinterpret_cast<uint8_t*>(runs + TC_GROUPS * 8);             // [groups]
  __shared__ uint64_t bar_tfull[4], bar_tempty[4];
  __shared__ uint64_t bar_ofull[TC_STAGES], bar_oempty[TC_STAGES], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int ti, tj;
  tile_of(blockIdx.x % a.ntiles, a.Tt, &ti, &tj);
  const int split = blockIdx.x / a.ntiles;
  const int nrows = *a.n_rows;
  int c0, c1;
  if (a.cstart) {                                 // grouped Gram: one split per leading index
    c0 = a.cstart[split];
    c1 = c0 + a.ccount[split];
  } else {
    const int nch = (nrows + CS - 1) / CS;
    const int cps = (nch + a.nsplit - 1) / a.nsplit;
    c0 = split * cps;
    c1 = min(nch, c0 + cps);
  }
  const int nchunks = max(0, c1 - c0);
  const int row0 = ti * TC_TILE, col0 = tj * TC_TILE;
  const bool diag = ti == tj;                     // A rows are the B rows
  const int ngroups = diag ? TC_GROUPS / 2 : TC_GROUPS;
  const int RN = a.R[a.N - 1];

  // runs of each 8-row group (group g < 32: B rows col0 + 8g.., else A rows)
  for (int g = threadIdx.x; g < ngroups; g += blockDim.x) {
    const int gbase = g < TC_GROUPS / 2 ? col0 + 8 * g : row0 + 8 * (g - TC_GROUPS / 2);
    int cnt = 0, i = 0;
    while (i < 8) {
      TcRun run;
      const int grow = gbase + i;
      run.row0 = (uint8_t)i;
      if (grow >= a.d) {
        run.n = (uint8_t)(8 - i); run.t0 = 0; run.zero = 1;
        for (int n = 0; n < TUCKER_MAX_ORDER - 1; ++n) run.po[n] = 0;
      } else {
        const int rho = grow / RN, t = grow - rho * RN;
        int n = min(8 - i, RN - t);
        if (grow + n > a.d) n = a.d - grow;
        run.n = (uint8_t)n; run.t0 = (uint8_t)t; run.zero = 0;
        int rr = rho;
        for (int m = a.N - 2; m >= 0; --m) {
          run.po[m] = (a.off[m] + rr % a.R[m]) * CS;
          rr /= a.R[m];
        }
        for (int m = a.N - 1; m < TUCKER_MAX_ORDER - 1; ++m) run.po[m] = 0;
      }
      runs[g * 8 + cnt++] = run;
      i += run.n;
    }
    nruns[g] = (uint8_t)cnt;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < a.tstages; ++i) {
      mbar_init(&bar_tfull[i], 1);
      mbar_init(&bar_tempty[i], TC_BUILD_WARPS * 32);
    }
    for (int i = 0; i < TC_STAGES; ++i) {
      mbar_init(&bar_ofull[i], TC_BUILD_WARPS * 32);
      mbar_init(&bar_oempty[i], 1);
    }
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_BUILD_WARPS) {     // TMEM allocation: two 256-column FP32 accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == TC_BUILD_WARPS + 1) {
    // ---------------- producer: bulk TMA of the chunk tables
    if (lane == 0) {
      const uint32_t bytes = (uint32_t)tab_elems * 4u;
      for (int it = 0; it < nchunks; ++it) {
        const int ts = it % a.tstages;
        if (it >= a.tstages &&
            !mbar_wait(&bar_tempty[ts], ((it / a.tstages) - 1) & 1, a.status, &abort_flag))
          break;
        mbar_expect_tx(&bar_tfull[ts], bytes);
        bulk_g2s(tab + (size_t)ts * tab_elems, a.pack + (size_t)(c0 + it) * tab_elems, bytes,
                 &bar_tfull[ts]);
      }
    }
  } else if (warp == TC_BUILD_WARPS) {
    // ---------------- MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc(Tr::FMT);
      for (int it = 0; it < nchunks; ++it) {
        const int os = it % TC_STAGES;
        if (!mbar_wait(&bar_ofull[os], (it / TC_STAGES) & 1, a.status, &abort_flag)) break;
        tc_fence_after();
        const uint32_t bB = smem_u32(opB + (size_t)os * TC_TILE * TC_ROWB);
        const uint32_t bA = diag ? bB : smem_u32(opA + (size_t)os * TC_TILE * TC_ROWB);
#pragma unroll
        for (int mb = 0; mb < 2; ++mb) {
          const uint32_t aA = bA + (uint32_t)(mb * TC_M * TC_ROWB);
#pragma unroll
          for (int k = 0; k < Tr::KSTEPS; ++k)     // 32 bytes of K per MMA
            mma<PREC>(tmem + (uint32_t)(mb * TC_N), sw128_desc(aA + 32 * k),
                      sw128_desc(bB + 32 * k), id, (it > 0 || k > 0) ? 1u : 0u);
        }
        mma_commit(&bar_oempty[os]);
      }
      mma_commit(&bar_done);
    }
  } else {
    // ---------------- builders (warps 0..15): item = (8-row group, 16-byte octet)
    const int bt = threadIdx.x;
    const int aNoff = a.off[a.N - 1] * CS;
    for (int it = 0; it < nchunks; ++it) {
      const int ts = it % a.tstages, os = it % TC_STAGES;
      const bool ok1 = mbar_wait(&bar_tfull[ts], (it / a.tstages) & 1, a.status, &abort_flag);
      const bool ok2 = it < TC_STAGES ||
                       mbar_wait(&bar_oempty[os], ((it / TC_STAGES) - 1) & 1, a.status, &abort_flag);
      if (!builders_all(ok1 && ok2)) break;            // uniform
      const float* T = tab + (size_t)ts * tab_elems;
      unsigned char* sB = opB + (size_t)os * TC_TILE * TC_ROWB;
      unsigned char* sA = opA + (size_t)os * TC_TILE * TC_ROWB;
      for (int item = bt; item < ngroups * 8; item += TC_BUILD_WARPS * 32) {
        const int g = item >> 3, c = item & 7;
        unsigned char* op = g < TC_GROUPS / 2 ? sB + (size_t)(8 * g) * TC_ROWB
                                              : sA + (size_t)(8 * (g - TC_GROUPS / 2)) * TC_ROWB;
        const int nr = nruns[g];
        for (int j = 0; j < nr; ++j) {
          const TcRun& run = runs[g * 8 + j];
          const int gr0 = 8 * (g & (TC_GROUPS / 2 - 1)) + run.row0;   // row inside the operand
          if (PREC == TUCKER_PREC_BF16) {
            // octet c: samples 8c..8c+7 at 4c..4c+3 and 32+4c..32+4c+3
            float4 p0 = make_float4(1.f, 1.f, 1.f, 1.f), p1 = p0;
            for (int m = 0; m < a.N - 1; ++m) {
              const float4 v0 = *reinterpret_cast<const float4*>(T + run.po[m] + 4 * c);
              const float4 v1 = *reinterpret_cast<const float4*>(T + run.po[m] + 32 + 4 * c);
              p0.x *= v0.x; p0.y *= v0.y; p0.z *= v0.z; p0.w *= v0.w;
              p1.x *= v1.x; p1.y *= v1.y; p1.z *= v1.z; p1.w *= v1.w;
            }
            if (run.n == 8 && !run.zero) {           // whole group: rows gr0 .. gr0 + 7
              const float* aN = T + aNoff + run.t0 * CS + 4 * c;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const float4 q0 = *reinterpret_cast<const float4*>(aN + q * CS);
                const float4 q1 = *reinterpret_cast<const float4*>(aN + q * CS + 32);
                uint4 out;
                out.x = pack_bf16(p0.x * q0.x, p0.y * q0.y);
                out.y = pack_bf16(p0.z * q0.z, p0.w * q0.w);
                out.z = pack_bf16(p1.x * q1.x, p1.y * q1.y);
                out.w = pack_bf16(p1.z * q1.z, p1.w * q1.w);
                *reinterpret_cast<uint4*>(op + q * TC_ROWB + ((c ^ q) << 4)) = out;
              }
              continue;
            }
            for (int q = 0; q < run.n; ++q) {
              const int row = gr0 + q;
              uint4 out = make_uint4(0, 0, 0, 0);
              if (!run.zero) {
                const float* aN = T + aNoff + (run.t0 + q) * CS;
                const float4 q0 = *reinterpret_cast<const float4*>(aN + 4 * c);
                const float4 q1 = *reinterpret_cast<const float4*>(aN + 32 + 4 * c);
                out.x = pack_bf16(p0.x * q0.x, p0.y * q0.y);
                out.y = pack_bf16(p0.z * q0.z, p0.w * q0.w);
                out.z = pack_bf16(p1.x * q1.x, p1.y * q1.y);
                out.w = pack_bf16(p1.z * q1.z, p1.w * q1.w);
              }
              *reinterpret_cast<uint4*>(op + (size_t)(row - 8 * (g & (TC_GROUPS / 2 - 1))) * TC_ROWB +
                                        ((c ^ (row & 7)) << 4)) = out;
            }
          } else {
            float4 p0 = make_float4(1.f, 1.f, 1.f, 1.f);
            for (int m = 0; m < a.N - 1; ++m) {
              const float4 v0 = *reinterpret_cast<const float4*>(T + run.po[m] + 4 * c);
              p0.x *= v0.x; p0.y *= v0.y; p0.z *= v0.z; p0.w *= v0.w;
            }
            if (run.n == 8 && !run.zero) {           // whole group: rows gr0 .. gr0 + 7
              const float* aN = T + aNoff + run.t0 * CS + 4 * c;
#pragma unroll
              for (int q = 0; q < 8; ++q) {
                const float4 q0 = *reinterpret_cast<const float4*>(aN + q * CS);
                uint4 out;
                out.x = to_tf32(p0.x * q0.x);
                out.y = to_tf32(p0.y * q0.y);
                out.z = to_tf32(p0.z * q0.z);
                out.w = to_tf32(p0.w * q0.w);
                *reinterpret_cast<uint4*>(op + q * TC_ROWB + ((c ^ q) << 4)) = out;
              }
              continue;
            }
            for (int q = 0; q < run.n; ++q) {
              const int row = gr0 + q;
              uint4 out = make_uint4(0, 0, 0, 0);
              if (!run.zero) {
                const float4 q0 = *reinterpret_cast<const float4*>(T + aNoff + (run.t0 + q) * CS + 4 * c);
                out.x = to_tf32(p0.x * q0.x);
                out.y = to_tf32(p0.y * q0.y);
                out.z = to_tf32(p0.z * q0.z);
                out.w = to_tf32(p0.w * q0.w);
              }
              *reinterpret_cast<uint4*>(op + (size_t)(row - 8 * (g & (TC_GROUPS / 2 - 1))) * TC_ROWB +
                                        ((c ^ (row & 7)) << 4)) = out;
            }
          }
        }
      }
      fence_proxy_async();          // generic-proxy writes -> visible to the tensor core
      mbar_arrive(&bar_tempty[ts]);
      mbar_arrive(&bar_ofull[os]);
    }
  }

  // ---------------- epilogue: warps 0..15, four per TMEM lane quadrant
  __syncthreads();
  float* outp = a.partial + ((size_t)split * a.ntiles + (blockIdx.x % a.ntiles)) * (TC_TILE * TC_TILE);
  if (warp < TC_BUILD_WARPS) {
    bool ok = true;
    if (nchunks > 0) ok = mbar_wait(&bar_done, 0, a.status, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    const int quad = warp & 3, cg = warp >> 2;            // lanes 32*quad.., TMEM columns cg*128..
    const int mb = cg >> 1;                                // accumulator
    const int row = mb * TC_M + quad * 32 + lane;          // row of the 256 x 256 tile
    for (int cb = 0; cb < 128; cb += 16) {
      const int tcol = cg * 128 + cb;                      // TMEM column
      const int col = (cg & 1) * 128 + cb;                 // column of the tile
      uint32_t v[16];
      if (nchunks > 0 && ok) {
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)tcol;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                       "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                       "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                     : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0u;
      }
      float4* dst = reinterpret_cast<float4*>(outp + (size_t)row * TC_TILE + col);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        dst[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                             __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_BUILD_WARPS) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

// G[r][c] = G[c][r] = sum over splits of the partial tiles (upper instances only).
// Thread = four consecutive columns of a tile row (16-byte loads), eight
// independent chains over the splits so that many loads are in flight (the
// partial tiles were just written and are mostly still in L2); the chains are
// combined in FP64 in a fixed order, so the result does not depend on timing.
__global__ void __launch_bounds__(256) k_tc_reduce(const float* partial, int nsplit, int ntiles,
                                                   int Tt, int d, double* G) {
  int ti, tj;
  tile_of(blockIdx.y, Tt, &ti, &tj);
  constexpr int Q = TC_TILE / 4;                        // 16-byte groups per tile row
  const size_t stride4 = (size_t)ntiles * (TC_TILE * TC_TILE) / 4;
  for (int e4 = blockIdx.x * blockDim.x + threadIdx.x; e4 < TC_TILE * Q;
       e4 += gridDim.x * blockDim.x) {
    const int lr = e4 / Q, lc = 4 * (e4 % Q);
    const int r = ti * TC_TILE + lr, c0 = tj * TC_TILE + lc;
    if (r >= d || c0 >= d || c0 + 3 < r) continue;     // nothing of the upper triangle here
    const float4* src = reinterpret_cast<const float4*>(partial) +
                        ((size_t)blockIdx.y * (TC_TILE * TC_TILE) + (size_t)lr * TC_TILE + lc) / 4;
    float4 acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int sp = 0; sp < nsplit; sp += 8) {             // chain j takes splits j, j + 8, ...
      float4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j)
        v[j] = sp + j < nsplit ? src[(size_t)(sp + j) * stride4] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        acc[j].x += v[j].x; acc[j].y += v[j].y; acc[j].z += v[j].z; acc[j].w += v[j].w;
      }
    }
    double o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double t[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) t[j] = q == 0 ? acc[j].x : q == 1 ? acc[j].y : q == 2 ? acc[j].z : acc[j].w;
      o[q] = ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + q;
      if (c < d && c >= r) {
        G[(size_t)r * d + c] = o[q];
        G[(size_t)c * d + r] = o[q];
      }
    }
  }
}

// ------------------------------------------------------------------ host side
static int tiles_of(int d, int* Tt) {
  *Tt = (d + TC_TILE - 1) / TC_TILE;
  return *Tt * (*Tt + 1) / 2;
}

static int chunk_samples(int prec) { return prec == TUCKER_PREC_BF16 ? 64 : 32; }

static int pick_splits(int ntiles, int64_t nch, int sms) {
  int best = 1;
  double best_eff = 0.0;
  for (int s = 1; s <= 64; ++s) {
    if ((int64_t)s > nch) break;
    const int ctas = ntiles * s;
    const int waves = (ctas + sms - 1) / sms;
    double eff = double(ctas) / double(waves * sms);
    // small penalty per split for the partial-tile traffic
    eff -= 0.002 * s;
    if (eff > best_eff + 1e-9) { best_eff = eff; best = s; }
  }
  return best;
}

int gram_tc_supported(int prec, int d) {
  return (prec == TUCKER_PREC_BF16 || prec == TUCKER_PREC_TF32) && d >= 1 && d <= 8192;
}

static size_t tc_smem_bytes(int sumR, int CS, int tstages) {
  const size_t ops = (size_t)TC_STAGES * 2 * TC_TILE * TC_ROWB;
  const size_t tab = (size_t)tstages * sumR * CS * 4;
  const size_t runs = (size_t)TC_GROUPS * 8 * sizeof(TcRun) + TC_GROUPS;
  return ops + tab + runs + 1024;
}

// Whether the leading-index-grouped Gram applies: order >= 3, R_1 in {1, 2, 4,
// 8, 16}, d / R_1 >= 128, and at most 8192 (segment, tile) splits of FP32
// partial tiles.
int gram_tc_grouped_ok(int N, int d, int R1, int64_t I1) {
  if (N < 3 || R1 < 1 || R1 > 16 || (R1 & (R1 - 1)) || d % R1) return 0;
  const int dp = d / R1;
  if (dp < 128) return 0;
  int Tt;
  const int nt = tiles_of(dp, &Tt);
  return I1 >= 1 && I1 * nt <= 8192 && I1 * R1 * 4 <= 200 * 1024;   // A^(1) staged in the reduction
}

// Whether the narrow grouped Gram applies: order >= 3, R_1 in {2, 4, 8, 16},
// d / R_1 <= 64, at least 2 rows per value of i_1 on average (else the full-width
// Gram is as cheap), and A^(1) small enough to stage in shared memory.
int gram_tc_narrow_ok(int N, int d, int R1, int64_t I1, int64_t cap) {
  if (N < 3 || R1 < 2 || R1 > 16 || (R1 & (R1 - 1)) || d % R1) return 0;
  const int dp = d / R1;
  return dp <= 64 && I1 >= 1 && cap >= 2 * I1 && I1 * R1 * 4 <= 96 * 1024;
}

static int64_t narrow_max_pieces(int64_t I1, int64_t cap) { return I1 + (cap + NR_PR - 1) / NR_PR; }

static size_t gram_tc_narrow_bytes(int d, int R1, int64_t I1, int64_t cap) {
  const int dp = d / R1;
  const int64_t P = narrow_max_pieces(I1, cap);
  return (size_t)P * dp * dp * 4 + 4096 + (size_t)(2 * I1 + 3 * P + 1) * 4 + 4096;
}

static size_t gram_tc_grouped_bytes(int prec, int d, int sumR, int R1, int64_t I1, int64_t cap) {
  const int dp = d / R1;
  int Tt;
  const int nt = tiles_of(dp, &Tt);
  const int CS = chunk_samples(prec);
  const int64_t nchm = (cap + CS - 1) / CS + I1;
  return (size_t)nchm * CS * (sumR - R1) * 4 + 4096 + (size_t)I1 * nt * TC_TILE * TC_TILE * 4 +
         4096 + (size_t)(4 * I1 + nchm) * 4 + 4096;
}

size_t gram_tc_workspace(tucker_handle* h, int prec, int d, int sumR, int64_t cap, int N, int R1,
                         int64_t I1) {
  int Tt;
  const int ntiles = tiles_of(d, &Tt);
  const int CS = chunk_samples(prec);
  const int64_t nch = (cap + CS - 1) / CS;
  const int ns = pick_splits(ntiles, nch, h->num_sms);
  // pack (sum R_n entries per sample) + partial tiles
  size_t b = (size_t)nch * CS * sumR * 4 + 4096 + (size_t)ns * ntiles * TC_TILE * TC_TILE * 4 + 4096;
  if (gram_tc_grouped_ok(N, d, R1, I1))
    b = std::max(b, gram_tc_grouped_bytes(prec, d, sumR, R1, I1, cap));
  if (gram_tc_narrow_ok(N, d, R1, I1, cap)) b = std::max(b, gram_tc_narrow_bytes(d, R1, I1, cap));
  return b;
}

static size_t expand_smem_bytes() { return 2 * (size_t)EX_STAGE + 2 * EX_KC * 16 * 4 + 1024; }

static tucker_status launch_expand(tucker_handle* h, const float* partial, int I1, int ntiles,
                                   int dp, const void* A1, int is64, int R1, int d, double* G) {
  ExpandArgs e;
  e.partial = partial;
  e.I1 = I1;
  e.ntiles = ntiles;
  e.nb = (dp + 15) / 16;
  e.dp = dp;
  e.R1 = R1;
  e.d = d;
  e.A1 = A1;
  e.is64 = is64;
  e.G = G;
  e.status = h->d_status;
  const size_t smem = expand_smem_bytes();
  TK_CUDA(h, cudaFuncSetAttribute(k_tcg_expand, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TK_COUNT(h);
  k_tcg_expand<<<dim3(e.nb * (e.nb + 1) / 2, (R1 * R1 + TC_M - 1) / TC_M), EX_THREADS, smem,
                 h->stream>>>(e);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// The Gram grouped by the leading index (sorted sample, s.idx[0] non-decreasing).
tucker_status launch_gram_tc_grouped(tucker_handle* h, const RowSet& s, int prec, int64_t cap,
                                     int64_t I1, char* ws, size_t ws_bytes, double* G) {
  const int R1 = s.R[0], dp = s.d / R1;
  int Tt;
  const int ntiles = tiles_of(dp, &Tt);
  const int CS = chunk_samples(prec);
  const int64_t nchm = (cap + CS - 1) / CS + I1;
  int sumR = 0;
  for (int n = 0; n < s.N; ++n) sumR += s.R[n];
  const int sumRp = sumR - R1;
  if (gram_tc_grouped_bytes(prec, s.d, sumR, R1, I1, cap) > ws_bytes)
    return fail(h, TUCKER_EINTERNAL, "grouped tc workspace too small");
  if ((size_t)sumRp * CS * 4 % 16 != 0) return fail(h, TUCKER_EINTERNAL, "pack block not 16-byte sized");
  if (nchm * sumRp >= (int64_t)1 << 31)
    return fail(h, TUCKER_ENOTSUP, "tensor-core Gram of %lld rows too large", (long long)cap);
  const size_t pack_bytes = (size_t)nchm * sumRp * CS * 4;
  float* pack = reinterpret_cast<float*>(ws);
  char* q = ws + ((pack_bytes + 255) & ~size_t(255));
  float* partial = reinterpret_cast<float*>(q);
  q += ((size_t)I1 * ntiles * TC_TILE * TC_TILE * 4 + 255) & ~size_t(255);
  int* seg_begin = reinterpret_cast<int*>(q);
  int* seg_end = seg_begin + I1;
  int* cstart = seg_end + I1;
  int* ccount = cstart + I1;
  int* cseg = ccount + I1;
  TK_CUDA(h, cudaMemsetAsync(seg_begin, 0, sizeof(int) * 2 * I1, h->stream));
  TK_CUDA(h, cudaMemsetAsync(cseg, 0xff, sizeof(int) * nchm, h->stream));
  int gs = (int)std::min<int64_t>((cap + 255) / 256, (int64_t)h->num_sms * 8);
  if (gs < 1) gs = 1;
  TK_COUNT(h);
  k_tcg_segments<<<gs, 256, 0, h->stream>>>(s.idx[0], s.n_rows, seg_begin, seg_end);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_tcg_chunks<<<1, 1024, 0, h->stream>>>(seg_begin, seg_end, (int)I1, CS, cstart, ccount, cseg);
  TK_LAUNCH(h);
  PackArgs p;
  memset(&p, 0, sizeof(p));
  TcArgs a;
  memset(&a, 0, sizeof(a));
  a.N = p.N = s.N - 1;
  int off = 0;
  for (int n = 1; n < s.N; ++n) {
    a.R[n - 1] = p.R[n - 1] = s.R[n];
    a.off[n - 1] = p.off[n - 1] = off;
    off += s.R[n];
    p.A[n - 1] = s.A[n];
    p.idx[n - 1] = s.idx[n];
  }
  a.sumR = p.sumR = sumRp;
  p.is64 = s.is64;
  p.w = s.w;
  p.n_rows = s.n_rows;
  p.CS = CS;
  p.perm = prec == TUCKER_PREC_BF16;
  p.pack = pack;
  int pg = (int)std::min<int64_t>((nchm * sumRp * CS + 255) / 256, (int64_t)h->num_sms * 16);
  if (pg < 1) pg = 1;
  TK_COUNT(h);
  k_tc_pack_grouped<<<pg, 256, 0, h->stream>>>(p, seg_begin, seg_end, cstart, cseg, (int)nchm);
  TK_LAUNCH(h);
  a.d = dp;
  a.Tt = Tt;
  a.ntiles = ntiles;
  a.nsplit = (int)I1;
  a.n_rows = s.n_rows;
  a.status = h->d_status;
  a.pack = pack;
  a.partial = partial;
  a.cstart = cstart;
  a.ccount = ccount;
  int tst = 4;
  while (tst > 2 && tc_smem_bytes(sumRp, CS, tst) > 227 * 1024) --tst;
  const size_t smem = tc_smem_bytes(sumRp, CS, tst);
  if (smem > 227 * 1024) return fail(h, TUCKER_ENOTSUP, "grouped tensor-core Gram: shared memory");
  a.tstages = tst;
  auto kern = prec == TUCKER_PREC_BF16 ? k_syrk_tc<TUCKER_PREC_BF16> : k_syrk_tc<TUCKER_PREC_TF32>;
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (h->timing) cudaEventRecord(h->ev[10], h->stream);
  TK_COUNT(h);
  kern<<<(int)(ntiles * I1), TC_THREADS, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  if (h->timing) cudaEventRecord(h->ev[11], h->stream);
  return launch_expand(h, partial, (int)I1, ntiles, dp, s.A[0], s.is64, R1, s.d, G);
}

// The narrow grouped Gram (sorted sample, s.idx[0] non-decreasing, d / R_1 <= 64).
template <int R1>
static tucker_status launch_expand_narrow(tucker_handle* h, const float* Mp, const int* pseg,
                                          const int* npieces, int I1, int dp, const void* A1,
                                          int is64, int d, double* G) {
  const int ne = dp * (dp + 1) / 2;
  const size_t smem = (size_t)(((I1 * R1 + 3) & ~3) + XN_WARPS * 32 * 32) * 4;
  if (smem > 227 * 1024) return fail(h, TUCKER_ENOTSUP, "narrow grouped Gram: shared memory");
  TK_CUDA(h, cudaFuncSetAttribute(k_tcg_expand_narrow<R1>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TK_CUDA(h, launch_dep(h, k_tcg_expand_narrow<R1>, dim3((ne + 31) / 32, (R1 * R1 + 31) / 32),
                        XN_WARPS * 32, smem, Mp, pseg, npieces, I1, dp, A1, is64, d, G));
  return TUCKER_OK;
}

tucker_status launch_gram_tc_narrow(tucker_handle* h, const RowSet& s, int64_t I1, int64_t cap,
                                    char* ws, size_t ws_bytes, double* G) {
  const int R1 = s.R[0], dp = s.d / R1;
  if (gram_tc_narrow_bytes(s.d, R1, I1, cap) > ws_bytes)
    return fail(h, TUCKER_EINTERNAL, "narrow grouped Gram workspace too small");
  const int64_t P = narrow_max_pieces(I1, cap);
  if (P >= (int64_t)1 << 31) return fail(h, TUCKER_ENOTSUP, "narrow grouped Gram: %lld rows", (long long)cap);
  NarrowArgs a;
  memset(&a, 0, sizeof(a));
  a.nm = s.N - 1;
  int off = 0;
  for (int n = 1; n < s.N; ++n) {
    a.R[n - 1] = s.R[n];
    a.off[n - 1] = off;
    off += s.R[n];
    a.A[n - 1] = s.A[n];
    a.idx[n - 1] = s.idx[n];
  }
  a.sumR = off;
  if (a.sumR + 1 > NR_MAXE)
    return fail(h, TUCKER_ENOTSUP, "narrow grouped Gram: sum of ranks %d too large", a.sumR);
  a.dp = dp;
  a.is64 = s.is64;
  a.w = s.w;
  float* Mp = reinterpret_cast<float*>(ws);
  int* seg_begin = reinterpret_cast<int*>(ws + (((size_t)P * dp * dp * 4 + 255) & ~size_t(255)));
  int* seg_end = seg_begin + I1;
  int* prow0 = seg_end + I1;
  int* prow1 = prow0 + P;
  int* pseg = prow1 + P;
  int* npieces = pseg + P;
  a.prow0 = prow0;
  a.prow1 = prow1;
  a.npieces = npieces;
  a.Mp = Mp;
  a.status = h->d_status;
  TK_CUDA(h, cudaMemsetAsync(seg_begin, 0, sizeof(int) * 2 * I1, h->stream));
  int gs = (int)std::min<int64_t>((cap + 255) / 256, (int64_t)h->num_sms * 8);
  if (gs < 1) gs = 1;
  TK_COUNT(h);
  k_tcg_segments<<<gs, 256, 0, h->stream>>>(s.idx[0], s.n_rows, seg_begin, seg_end);
  TK_LAUNCH(h);
  TK_CUDA(h, launch_dep(h, k_tcg_pieces, 1, 1024, 0, seg_begin, seg_end, (int)I1, prow0, prow1,
                        pseg, npieces));
  const size_t smem = narrow_smem_bytes(a.sumR, a.nm);
  auto kern = a.nm == 2 ? k_tcg_narrow<2> : a.nm == 3 ? k_tcg_narrow<3> : k_tcg_narrow<0>;
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (h->timing) cudaEventRecord(h->ev[10], h->stream);
  TK_CUDA(h, launch_dep(h, kern, (int)P, NR_THREADS, smem, a));
  if (h->timing) cudaEventRecord(h->ev[11], h->stream);
  switch (R1) {
    case 2: return launch_expand_narrow<2>(h, Mp, pseg, npieces, (int)I1, dp, s.A[0], s.is64, s.d, G);
    case 4: return launch_expand_narrow<4>(h, Mp, pseg, npieces, (int)I1, dp, s.A[0], s.is64, s.d, G);
    case 8: return launch_expand_narrow<8>(h, Mp, pseg, npieces, (int)I1, dp, s.A[0], s.is64, s.d, G);
    case 16: return launch_expand_narrow<16>(h, Mp, pseg, npieces, (int)I1, dp, s.A[0], s.is64, s.d, G);
    default: return fail(h, TUCKER_EINTERNAL, "narrow grouped Gram: R_1 = %d", R1);
  }
}

tucker_status launch_gram_tc(tucker_handle* h, const RowSet& s, int prec, int64_t cap, char* ws,
                             size_t ws_bytes, double* G) {
  int Tt;
  const int ntiles = tiles_of(s.d, &Tt);
  const int CS = chunk_samples(prec);
  const int64_t nch = (cap + CS - 1) / CS;
  const int ns = pick_splits(ntiles, nch, h->num_sms);
  TcArgs a;
  memset(&a, 0, sizeof(a));
  PackArgs p;
  memset(&p, 0, sizeof(p));
  a.N = p.N = s.N;
  int sumR = 0;
  for (int n = 0; n < s.N; ++n) {
    a.R[n] = p.R[n] = s.R[n];
    a.off[n] = p.off[n] = sumR;
    sumR += s.R[n];
    p.A[n] = s.A[n];
    p.idx[n] = s.idx[n];
  }
  a.sumR = p.sumR = sumR;
  if ((size_t)sumR * CS * 4 % 16 != 0) return fail(h, TUCKER_EINTERNAL, "pack block not 16-byte sized");
  a.d = s.d;
  a.Tt = Tt; a.ntiles = ntiles; a.nsplit = ns;
  a.n_rows = p.n_rows = s.n_rows;
  a.status = h->d_status;
  const size_t pack_bytes = (size_t)nch * sumR * CS * 4;
  const size_t part_bytes = (size_t)ns * ntiles * TC_TILE * TC_TILE * 4;
  if (pack_bytes + part_bytes + 512 > ws_bytes) return fail(h, TUCKER_EINTERNAL, "tc workspace too small");
  float* pack = reinterpret_cast<float*>(ws);
  float* partial = reinterpret_cast<float*>(ws + ((pack_bytes + 255) & ~size_t(255)));
  p.is64 = s.is64;
  p.w = s.w;
  p.CS = CS;
  p.perm = prec == TUCKER_PREC_BF16;
  p.pack = pack;
  a.pack = pack;
  a.partial = partial;
  // as many chunk-table stages (2..4) as shared memory allows
  int tst = 4;
  while (tst > 2 && tc_smem_bytes(sumR, CS, tst) > 227 * 1024) --tst;
  const size_t smem = tc_smem_bytes(sumR, CS, tst);
  if (smem > 227 * 1024)
    return fail(h, TUCKER_ENOTSUP, "tensor-core Gram needs %zu bytes of shared memory "
                "(sum R_n = %d)", smem, sumR);
  a.tstages = tst;
  if (nch * sumR >= (int64_t)1 << 31)
    return fail(h, TUCKER_ENOTSUP, "tensor-core Gram of %lld rows too large", (long long)cap);
  int pg = (int)std::min<int64_t>((nch * sumR * CS + 255) / 256, (int64_t)h->num_sms * 16);
  if (pg < 1) pg = 1;
  TK_COUNT(h);
  k_tc_pack<<<pg, 256, 0, h->stream>>>(p);
  TK_LAUNCH(h);
  auto kern = prec == TUCKER_PREC_BF16 ? k_syrk_tc<TUCKER_PREC_BF16> : k_syrk_tc<TUCKER_PREC_TF32>;
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (h->timing) cudaEventRecord(h->ev[10], h->stream);
  TK_COUNT(h);
  kern<<<ntiles * ns, TC_THREADS, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  if (h->timing) cudaEventRecord(h->ev[11], h->stream);
  TK_COUNT(h);
  k_tc_reduce<<<dim3(64, ntiles), 256, 0, h->stream>>>(partial, ns, ntiles, Tt, s.d, G);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
