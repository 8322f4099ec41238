// Tensor-core (tcgen05) Gram of the implicit Kronecker rows of the sample:
//     G = sum_u x_u x_u^T,   x_u = sqrt(w_u) * A^(1)[i_1] (x) ... (x) A^(N)[i_N]
// (the normal-equation matrix of Alg. 1's sketched least squares, formed as
// a sum of outer products as in the proof of Thm 4.2).  The design matrix is
// never stored: operand tiles of x are generated in shared memory.
//
// Pipeline per CTA (one 128 x 256 output tile of the upper triangle of G and
// one contiguous range of 64-sample chunks):
//   pack kernel  : per chunk, the factor rows of its samples are laid out
//                  entry-major [e][s] (e over (n, r_n), s over 64 samples) in
//                  FP32, with sqrt(w) folded into mode 1 -> one contiguous block;
//   producer warp: 1-D bulk TMA (cp.async.bulk) of each chunk block into a
//                  4-deep shared-memory ring (mbarrier transaction counts);
//   builder warps: P[rho][s] = prod_{n<N} a_n[s][r_n] (rho = r / R_N) for the
//                  tile's row ranges, then x[r][s] = P[rho(r)][s] * a_N[s][r mod R_N]
//                  rounded to BF16 (or TF32) into K-major, 128-byte-swizzled
//                  operand tiles (rows = d index, 128 bytes of samples per row);
//   MMA thread   : tcgen05.mma.cta_group::1 (M = 128, N = 256) accumulating in
//                  TMEM (FP32), tcgen05.commit frees the operand stage;
//   epilogue     : tcgen05.ld of the accumulator, FP32 partial tile to global.
// A reduction kernel sums the sample splits in a fixed order into the
// symmetric FP64 G.  Tiles whose row range lies inside their column range
// reuse the B operand rows as A (no second build).
// Every wait is bounded: on timeout the kernel records TUCKER_EINTERNAL,
// waits (bounded) for its MMAs, frees TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace tk {

constexpr int TC_M = 128;          // rows of an output tile (TMEM lanes)
constexpr int TC_N = 256;          // columns of an output tile (TMEM columns)
constexpr int TC_ROWB = 128;       // bytes of K per operand row (one swizzle atom)
constexpr int TC_STAGES = 2;       // operand stages
constexpr int TC_TSTAGES = 4;      // sample-table stages
constexpr int TC_BUILD_WARPS = 8;
constexpr int TC_THREADS = (TC_BUILD_WARPS + 2) * 32;   // + MMA warp + TMA warp
constexpr uint32_t TC_WAIT_LIMIT = 1u << 24;

template <int PREC> struct TcTraits;
template <> struct TcTraits<TUCKER_PREC_BF16> {
  static constexpr int CS = 64;        // samples per chunk (128 bytes of BF16)
  static constexpr int PER16 = 8;      // samples per 16-byte unit
  static constexpr uint32_t FMT = 1;   // BF16 in the instruction descriptor
};
template <> struct TcTraits<TUCKER_PREC_TF32> {
  static constexpr int CS = 32;
  static constexpr int PER16 = 4;
  static constexpr uint32_t FMT = 2;   // TF32
};

struct TcArgs {
  int N;
  int R[TUCKER_MAX_ORDER];
  int off[TUCKER_MAX_ORDER];          // entry offset of mode n in a chunk block
  int sumR;
  int d;
  int RN;                              // R_N
  int Ti, Tj;                          // tiles along rows (128) and columns (256)
  int ntiles;
  int nsplit;
  const float* pack;                   // [chunks][sumR][CS]
  const int* n_rows;
  float* partial;                      // [nsplit][ntiles][128][256]
  int* status;
};

// ------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}"
               ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
  return ok != 0;
}
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
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
// pack[q][e][s] = value e (mode n, column r) of sample q*CS + s; mode 1 scaled by sqrt(w).
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
  int64_t cap_chunks;
  float* pack;
};

__global__ void k_tc_pack(PackArgs a) {
  const int nrows = *a.n_rows;
  const int64_t nch = (nrows + a.CS - 1) / a.CS;
  const int64_t total = nch * a.sumR * a.CS;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(t % a.CS);
    const int e = (int)((t / a.CS) % a.sumR);
    const int64_t q = t / ((int64_t)a.CS * a.sumR);
    const int64_t u = q * a.CS + s;
    float v = 0.f;
    if (u < nrows) {
      int n = 0;
      while (n + 1 < a.N && e >= a.off[n + 1]) ++n;
      const int r = e - a.off[n];
      v = (float)load_as_double(a.A[n], (int64_t)a.idx[n][u] * a.R[n] + r, a.is64);
      if (n == 0) v = (float)(sqrt(a.w[u]) * load_as_double(a.A[n], (int64_t)a.idx[n][u] * a.R[n] + r, a.is64));
    }
    a.pack[t] = v;
  }
}

// --------------------------------------------------------------- the SYRK
template <int PREC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_syrk_tc(TcArgs a) {
  using Tr = TcTraits<PREC>;
  constexpr int CS = Tr::CS;
  extern __shared__ __align__(1024) unsigned char smraw[];
  // carve shared memory (1024-byte aligned operand stages first)
  const uint32_t base_u = smem_u32(smraw);
  unsigned char* sm = smraw + ((1024 - (base_u & 1023)) & 1023);
  unsigned char* opA = sm;                                   // STAGES x 128 rows x 128 B
  unsigned char* opB = opA + TC_STAGES * TC_M * TC_ROWB;      // STAGES x 256 rows x 128 B
  float* tab = reinterpret_cast<float*>(opB + TC_STAGES * TC_N * TC_ROWB);   // TSTAGES x sumR x CS
  const int tab_elems = a.sumR * CS;
  float* Ptab = tab + TC_TSTAGES * tab_elems;                 // (N/RN + 2 + M/RN + 2) x CS
  const int nPB = TC_N / a.RN + 2, nPA = TC_M / a.RN + 2;
  // decode tables (fixed per tile): T entry offsets of each P row, and for
  // each operand row its P row and its column of a_N (0xffff: beyond d)
  int* Poff = reinterpret_cast<int*>(Ptab + (nPB + nPA) * CS);           // (nPB+nPA) x (N-1)
  uint32_t* rowinfo = reinterpret_cast<uint32_t*>(Poff + (nPB + nPA) * TUCKER_MAX_ORDER);  // 384
  __shared__ uint64_t bar_tfull[TC_TSTAGES], bar_tempty[TC_TSTAGES];
  __shared__ uint64_t bar_ofull[TC_STAGES], bar_oempty[TC_STAGES], bar_done;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tile (ti, tj) of the upper triangle and the chunk range of this split
  int rem = blockIdx.x % a.ntiles, tj = 0;
  while (true) {
    const int cnt = min(2 * tj + 2, a.Ti);
    if (rem < cnt) break;
    rem -= cnt;
    ++tj;
  }
  const int ti = rem;
  const int split = blockIdx.x / a.ntiles;
  const int nrows = *a.n_rows;
  const int nch = (nrows + CS - 1) / CS;
  const int cps = (nch + a.nsplit - 1) / a.nsplit;
  const int c0 = split * cps, c1 = min(nch, c0 + cps);
  const int nchunks = max(0, c1 - c0);
  const int row0 = ti * TC_M, col0 = tj * TC_N;
  const bool a_in_b = row0 >= col0 && row0 + TC_M <= col0 + TC_N;
  const int rho0B = col0 / a.RN, rho0A = row0 / a.RN;

  for (int pr = threadIdx.x; pr < nPB + nPA; pr += blockDim.x) {
    int rr = pr < nPB ? rho0B + pr : rho0A + (pr - nPB);
    for (int n = a.N - 2; n >= 0; --n) {
      Poff[pr * TUCKER_MAX_ORDER + n] = (a.off[n] + rr % a.R[n]) * CS;
      rr /= a.R[n];
    }
  }
  for (int r = threadIdx.x; r < TC_N + TC_M; r += blockDim.x) {
    const bool isB = r < TC_N;
    const int grow = isB ? col0 + r : row0 + (r - TC_N);
    uint32_t info = 0xffffffffu;
    if (grow < a.d) {
      const int rho = grow / a.RN, t = grow - rho * a.RN;
      const int prow = isB ? rho - rho0B : nPB + (rho - rho0A);
      info = ((uint32_t)prow << 16) | (uint32_t)t;
    }
    rowinfo[r] = info;
  }
  if (threadIdx.x == 0) {
    for (int i = 0; i < TC_TSTAGES; ++i) { mbar_init(&bar_tfull[i], 1); mbar_init(&bar_tempty[i], TC_BUILD_WARPS * 32); }
    for (int i = 0; i < TC_STAGES; ++i) { mbar_init(&bar_ofull[i], TC_BUILD_WARPS * 32); mbar_init(&bar_oempty[i], 1); }
    mbar_init(&bar_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_BUILD_WARPS) {     // TMEM allocation: 256 FP32 columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(smem_u32(&tmem_slot)), "r"(TC_N) : "memory");
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
        const int ts = it % TC_TSTAGES;
        if (it >= TC_TSTAGES &&
            !mbar_wait(&bar_tempty[ts], ((it / TC_TSTAGES) - 1) & 1, a.status, &abort_flag))
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
        const uint32_t bB = smem_u32(opB + (size_t)os * TC_N * TC_ROWB);
        const uint32_t bA = a_in_b ? bB + (uint32_t)(row0 - col0) * TC_ROWB
                                   : smem_u32(opA + (size_t)os * TC_M * TC_ROWB);
#pragma unroll
        for (int k = 0; k < 4; ++k)     // 4 x 32 bytes of K per 128-byte row
          mma<PREC>(tmem, sw128_desc(bA + 32 * k), sw128_desc(bB + 32 * k), id,
                    (it > 0 || k > 0) ? 1u : 0u);
        mma_commit(&bar_oempty[os]);
      }
      mma_commit(&bar_done);
    }
  } else {
    // ---------------- builders (warps 0..7)
    const int bt = threadIdx.x;                       // 0..255
    for (int it = 0; it < nchunks; ++it) {
      const int ts = it % TC_TSTAGES, os = it % TC_STAGES;
      const bool ok1 = mbar_wait(&bar_tfull[ts], (it / TC_TSTAGES) & 1, a.status, &abort_flag);
      const float* T = tab + (size_t)ts * tab_elems;
      if (ok1) {
        // P[rho][s] = prod over modes 1..N-1 of the factor entries of rho
        for (int e = bt; e < (nPB + nPA) * CS; e += TC_BUILD_WARPS * 32) {
          const int pr = e / CS, s = e % CS;          // CS is a power of two
          const int* po = Poff + pr * TUCKER_MAX_ORDER;
          float v = 1.f;
          for (int n = 0; n < a.N - 1; ++n) v *= T[po[n] + s];
          Ptab[pr * CS + s] = v;
        }
      }
      // the operand stage must be free (MMAs of chunk it - STAGES done)
      const bool ok2 = it < TC_STAGES ||
                       mbar_wait(&bar_oempty[os], ((it / TC_STAGES) - 1) & 1, a.status, &abort_flag);
      if (!builders_all(ok1 && ok2)) break;            // uniform; also publishes Ptab
      const float* aN = T + a.off[a.N - 1] * CS;
      unsigned char* sB = opB + (size_t)os * TC_N * TC_ROWB;
      unsigned char* sA = opA + (size_t)os * TC_M * TC_ROWB;
      const int units = (TC_N + (a_in_b ? 0 : TC_M)) * 8;
      for (int uidx = bt; uidx < units; uidx += TC_BUILD_WARPS * 32) {
        const bool isB = uidx < TC_N * 8;
        const int ul = isB ? uidx : uidx - TC_N * 8;
        const int r = ul >> 3, c = ul & 7;
        const uint32_t info = rowinfo[isB ? r : TC_N + r];
        uint4 out = make_uint4(0, 0, 0, 0);
        if (info != 0xffffffffu) {
          const int t = (int)(info & 0xffffu);
          const float* P = Ptab + (int)(info >> 16) * CS;
          const int s0 = c * Tr::PER16;
          if (PREC == TUCKER_PREC_BF16) {
            const float4 p0 = *reinterpret_cast<const float4*>(P + s0);
            const float4 p1 = *reinterpret_cast<const float4*>(P + s0 + 4);
            const float4 q0 = *reinterpret_cast<const float4*>(aN + t * CS + s0);
            const float4 q1 = *reinterpret_cast<const float4*>(aN + t * CS + s0 + 4);
            out.x = pack_bf16(p0.x * q0.x, p0.y * q0.y);
            out.y = pack_bf16(p0.z * q0.z, p0.w * q0.w);
            out.z = pack_bf16(p1.x * q1.x, p1.y * q1.y);
            out.w = pack_bf16(p1.z * q1.z, p1.w * q1.w);
          } else {
            const float4 p0 = *reinterpret_cast<const float4*>(P + s0);
            const float4 q0 = *reinterpret_cast<const float4*>(aN + t * CS + s0);
            out.x = to_tf32(p0.x * q0.x);
            out.y = to_tf32(p0.y * q0.y);
            out.z = to_tf32(p0.z * q0.z);
            out.w = to_tf32(p0.w * q0.w);
          }
        }
        unsigned char* dst = (isB ? sB : sA) + r * TC_ROWB + ((c ^ (r & 7)) << 4);
        *reinterpret_cast<uint4*>(dst) = out;
      }
      fence_proxy_async();          // generic-proxy writes -> visible to the tensor core
      mbar_arrive(&bar_tempty[ts]);
      mbar_arrive(&bar_ofull[os]);
      asm volatile("bar.sync 1, %0;" ::"r"(TC_BUILD_WARPS * 32) : "memory");   // Ptab reuse
    }
  }

  // ---------------- epilogue: warps 0..7 (two per TMEM lane quadrant)
  __syncthreads();
  float* outp = a.partial + ((size_t)split * a.ntiles + (blockIdx.x % a.ntiles)) * (TC_M * TC_N);
  if (warp < TC_BUILD_WARPS) {
    bool ok = true;
    if (nchunks > 0) ok = mbar_wait(&bar_done, 0, a.status, &abort_flag);
    ok = __all_sync(0xffffffffu, ok);
    tc_fence_after();
    const int quad = warp & 3, half = warp >> 2;         // lanes 32*quad.., columns half*128..
    const int row = quad * 32 + lane;
    for (int cb = 0; cb < TC_N / 2; cb += 16) {
      const int col = half * (TC_N / 2) + cb;
      uint32_t v[16];
      if (nchunks > 0 && ok) {
        const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)col;
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
      float4* dst = reinterpret_cast<float4*>(outp + (size_t)row * TC_N + col);
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
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N)
                 : "memory");
  }
}

// G[r][c] = G[c][r] = sum over splits of the partial tiles (upper instances only)
__global__ void k_tc_reduce(const float* partial, int nsplit, int ntiles, int Ti, int d, double* G) {
  int rem = blockIdx.y, tj = 0;
  while (true) {
    const int cnt = min(2 * tj + 2, Ti);
    if (rem < cnt) break;
    rem -= cnt;
    ++tj;
  }
  const int ti = rem;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < TC_M * TC_N; e += gridDim.x * blockDim.x) {
    const int r = ti * TC_M + e / TC_N, c = tj * TC_N + e % TC_N;
    if (r >= d || c >= d || r > c) continue;
    double v = 0.0;
    for (int sp = 0; sp < nsplit; ++sp)
      v += (double)partial[((size_t)sp * ntiles + blockIdx.y) * (TC_M * TC_N) + e];
    G[(size_t)r * d + c] = v;
    G[(size_t)c * d + r] = v;
  }
}

// ------------------------------------------------------------------ host side
static int tiles_of(int d, int* Ti, int* Tj) {
  *Ti = (d + TC_M - 1) / TC_M;
  *Tj = (d + TC_N - 1) / TC_N;
  int n = 0;
  for (int j = 0; j < *Tj; ++j) n += std::min(2 * j + 2, *Ti);
  return n;
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

static size_t tc_smem_bytes(int sumR, int RN, int CS) {
  const size_t ops = (size_t)TC_STAGES * (TC_M + TC_N) * TC_ROWB;
  const size_t tab = (size_t)TC_TSTAGES * sumR * CS * 4;
  const size_t P = (size_t)(TC_N / RN + 2 + TC_M / RN + 2) * CS * 4;
  const size_t dec = (size_t)(TC_N / RN + 2 + TC_M / RN + 2) * TUCKER_MAX_ORDER * 4 + (TC_M + TC_N) * 4;
  return ops + tab + P + dec + 1024;
}

size_t gram_tc_workspace(tucker_handle* h, int prec, int d, int sumR, int64_t cap) {
  int Ti, Tj;
  const int ntiles = tiles_of(d, &Ti, &Tj);
  const int CS = chunk_samples(prec);
  const int64_t nch = (cap + CS - 1) / CS;
  const int ns = pick_splits(ntiles, nch, h->num_sms);
  // pack (sum R_n entries per sample) + partial tiles
  return (size_t)nch * CS * sumR * 4 + 4096 + (size_t)ns * ntiles * TC_M * TC_N * 4 + 4096;
}

tucker_status launch_gram_tc(tucker_handle* h, const RowSet& s, int prec, int64_t cap, char* ws,
                             size_t ws_bytes, double* G) {
  int Ti, Tj;
  const int ntiles = tiles_of(s.d, &Ti, &Tj);
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
  a.RN = s.R[s.N - 1];
  a.Ti = Ti; a.Tj = Tj; a.ntiles = ntiles; a.nsplit = ns;
  a.n_rows = p.n_rows = s.n_rows;
  a.status = h->d_status;
  const size_t pack_bytes = (size_t)nch * sumR * CS * 4;
  const size_t part_bytes = (size_t)ns * ntiles * TC_M * TC_N * 4;
  if (pack_bytes + part_bytes + 512 > ws_bytes) return fail(h, TUCKER_EINTERNAL, "tc workspace too small");
  float* pack = reinterpret_cast<float*>(ws);
  float* partial = reinterpret_cast<float*>(ws + ((pack_bytes + 255) & ~size_t(255)));
  p.is64 = s.is64;
  p.w = s.w;
  p.CS = CS;
  p.cap_chunks = nch;
  p.pack = pack;
  a.pack = pack;
  a.partial = partial;
  // >= 120 KB keeps one CTA per SM (the kernel allocates 256 TMEM columns)
  const size_t smem = std::max<size_t>(tc_smem_bytes(sumR, a.RN, CS), 120 * 1024);
  if (smem > 227 * 1024)
    return fail(h, TUCKER_ENOTSUP, "tensor-core Gram needs %zu bytes of shared memory "
                "(sum R_n = %d, R_N = %d)", smem, sumR, a.RN);
  int pg = (int)std::min<int64_t>((nch * sumR * CS + 255) / 256, (int64_t)h->num_sms * 16);
  if (pg < 1) pg = 1;
  TK_COUNT(h);
  k_tc_pack<<<pg, 256, 0, h->stream>>>(p);
  TK_LAUNCH(h);
  auto kern = prec == TUCKER_PREC_BF16 ? k_syrk_tc<TUCKER_PREC_BF16> : k_syrk_tc<TUCKER_PREC_TF32>;
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TK_COUNT(h);
  kern<<<ntiles * ns, TC_THREADS, smem, h->stream>>>(a);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_tc_reduce<<<dim3(32, ntiles), 256, 0, h->stream>>>(partial, ns, ntiles, Ti, s.d, G);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
