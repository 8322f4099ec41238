// Internal definitions shared by the CUDA translation units of libtucker.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include "tucker.h"

namespace tk {

// ----------------------------------------------------------------- handle

// Device-side status word: kernels record the first error code seen.
enum DeviceErr : int {
  DEV_OK = 0,
  DEV_NOTSPD = TUCKER_ENOTSPD,
  DEV_RANK = TUCKER_ERANK,
  DEV_DRAWLIMIT = TUCKER_EDRAWLIMIT,
  DEV_HASHFULL = TUCKER_EHASHFULL,
  DEV_INTERNAL = TUCKER_EINTERNAL,
};

struct HashTable {
  const uint64_t* src_keys = nullptr;  // COO keys the table was built from
  int64_t nnz = 0;
  uint64_t* slot_key = nullptr;        // 2^log2 slots; empty = ~0
  uint32_t* slot_idx = nullptr;        // index into the COO arrays
  int log2 = 0;
  size_t bytes = 0;
};

struct CholCache {
  double* L = nullptr;    // d x d lower factor (row-major), FP64
  double* regdiag = nullptr;  // d: lambda * (1 or D_j)
  double* Linv = nullptr;     // inverses of the 64 x 64 diagonal blocks of L
  double* LT = nullptr;       // L transposed (upper triangle), d x d
  double* tmp = nullptr;      // d doubles of solve scratch
  double* part = nullptr;     // per-CTA partial norms of a refinement correction
  float* L32 = nullptr;       // FP32 factor of the mixed solver (d x d)
  float* LT32 = nullptr;      // its transpose
  float* Linv32 = nullptr;    // its inverted 64 x 64 diagonal blocks
  float* X32 = nullptr;       // explicit L32^-1, row-major (small d only)
  float* XC32 = nullptr;      // the same, column-major
  int inv32 = 0;          // X32 / XC32 are ready
  int mixed = 0;          // the cached factor is the FP32 one (L then holds M itself)
  int prep64 = 0;         // LT / Linv of the FP64 factor are ready
  int prep32 = 0;         // L32 / LT32 / Linv32 are ready (the FP32 factor, or the FP64 one rounded)
  int kpcg = 0;           // the solves are Kronecker-preconditioned CG on L32 = M~ (no factor)
  double* kv[TUCKER_MAX_ORDER] = {};  // KRON_PCG: eigenvectors V_n of A^(n)T A^(n) (R_n x R_n)
  double* ke[TUCKER_MAX_ORDER] = {};  // KRON_PCG: their eigenvalues (R_n)
  float* sg = nullptr;    // KRON_PCG: 2 d floats of product exchange
  double* kres = nullptr; // KRON_PCG: (iterations, final relative residual) per solve
  int kres_n = 0;         // solves recorded in kres during this call
  double ktol = 1e-4;     // relative residual each CG solve stops at
  int kron_ready = 0;     // kv / ke hold the eigendecompositions of the current factors
  int kN = 0;             // order and ranks of kv / ke
  int kR[TUCKER_MAX_ORDER] = {};
  int d = 0;
  size_t cap = 0;         // bytes allocated behind L
  uint64_t id = 0;        // solve id of the cached factor (0 = none)
};

}  // namespace tk

struct tucker_handle {
  cudaStream_t stream = nullptr;
  int device = 0;
  int num_sms = 0;
  int sync_mode = 1;
  char* ws = nullptr;           // workspace (bump-allocated per call)
  size_t ws_cap = 0;
  int* d_status = nullptr;      // device status word
  int* h_status = nullptr;      // pinned host copy
  double* h_kev = nullptr;      // pinned: the factor eigenvalues the refinement's first check reads
  double* keep = nullptr;       // kAuxDoubles of device scratch that outlives the workspace
  tk::HashTable hash;
  tk::CholCache chol;
  uint64_t next_solve_id = 1;
  int64_t launches = 0;         // kernels launched by this handle (all calls)
  int solver = 0;               // tucker_solver: FP64 Cholesky (0), mixed (1), Kronecker CG (2)
  int64_t factor_m = 0;         // draws of each sketched factor update of an ALS sweep (0: exact)
  int timing = 0;               // record per-kernel events (ev[8..11]) during this call
  int chol_cluster[2] = {0, 0}; // CTAs of the one-cluster FP32 Cholesky of order chol_cluster_key
  int chol_cluster_key = -1;    // (without, with the explicit inverse; 0: does not fit)
  cudaEvent_t ev[16];
  cudaStream_t aux = nullptr;   // second stream: work that runs beside the factorisation
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  char err[512];
};

namespace tk {

constexpr int kAuxDoubles = 8192 + 64;   // d <= 8192 plus a few scalars

// Record a host-side error message on the handle and return the status.
tucker_status fail(tucker_handle* h, tucker_status s, const char* fmt, ...);

// Check a CUDA runtime result; on failure record it and return ECUDA.
#define TK_CUDA(h, call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return ::tk::fail((h), TUCKER_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                          \
  } while (0)

#define TK_LAUNCH(h)                                                                  \
  do {                                                                                \
    cudaError_t e_ = cudaGetLastError();                                              \
    if (e_ != cudaSuccess)                                                            \
      return ::tk::fail((h), TUCKER_ECUDA, "kernel launch: %s (%s:%d)",               \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                  \
  } while (0)

// Count one kernel launch on the handle (reported through tucker_stats).
#define TK_COUNT(h) (++(h)->launches)

// Launch on h->stream with programmatic dependent launch allowed: the grid may
// be scheduled while the previous kernel on the stream drains, which hides the
// launch latency between short dependent kernels.  Every kernel launched this
// way calls pdl_wait() first, before any access to global memory, so it sees
// all of the previous kernel's writes and overwrites nothing that kernel reads.
// Used where the previous operation on the stream is one of this library's
// kernels (an event record may sit in between), or where the host has just
// synchronised the stream; never right behind an event wait on another stream
// or behind a memset or copy whose data the kernel reads.
template <class... KArgs, class... Args>
inline cudaError_t launch_dep(tucker_handle* h, void (*k)(KArgs...), dim3 grid, dim3 block,
                              size_t smem, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ++h->launches;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// Wait for the previous kernel on the stream (and its memory writes); a no-op
// when the kernel was not launched with programmatic dependent launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

#define TK_TRY(expr)                                                                  \
  do {                                                                                \
    tucker_status s_ = (expr);                                                        \
    if (s_ != TUCKER_OK) return s_;                                                   \
  } while (0)

// Make sure the workspace holds `bytes`; reallocates (after a stream sync).
tucker_status ws_reserve(tucker_handle* h, size_t bytes);

// Synchronise and turn a device status into a tucker_status (clears it).
tucker_status device_status(tucker_handle* h);

// After launching work: in synchronous mode wait and report device errors.
tucker_status finish(tucker_handle* h);

// Bump allocator over the workspace.  Run once with base == nullptr to size.
struct Arena {
  char* base;
  size_t off = 0;
  explicit Arena(char* b) : base(b) {}
  template <class T>
  T* get(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += n * sizeof(T) + 16;
    return p;
  }
};

inline int ceil_div(int64_t a, int64_t b) { return int((a + b - 1) / b); }

// --------------------------------------------------------- device helpers

__device__ __forceinline__ void set_status(int* st, int code) {
  atomicCAS(st, 0, code);
}

__device__ __forceinline__ double load_as_double(const void* p, int64_t i, int is64) {
  return is64 ? static_cast<const double*>(p)[i] : double(static_cast<const float*>(p)[i]);
}

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 4 x 64-bit counter,
// 2 x 64-bit key, ten rounds with Weyl key bumps between rounds.
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
    uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U64x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// First index i in C[0..n) with C[i] > target (C non-decreasing, C[n-1] > target).
__device__ __forceinline__ int upper_bound_u64(const uint64_t* C, int n, uint64_t target) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (C[mid] > target) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// ------------------------------------------ mbarrier and bulk-copy (TMA) PTX
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
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide exclusive scan of one int64 per thread (blockDim.x <= 1024,
// multiple of 32).  `smem` holds >= 32 int64.  Returns the exclusive prefix;
// *total receives the block sum.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* smem,
                                                         int64_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int64_t s = lane < nw ? smem[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) smem[lane] = s;
  }
  __syncthreads();
  int64_t base = wid ? smem[wid - 1] : 0;
  *total = smem[nw - 1];
  __syncthreads();
  return base + x - v;
}

// Open-addressing hash table of observed keys (linear probing, Fibonacci hash).
__device__ __forceinline__ bool hash_contains(const uint64_t* slot_key, int log2, int max_probes,
                                              uint64_t key, int* status) {
  const uint64_t mask = (uint64_t(1) << log2) - 1;
  uint64_t s = (key * 0x9E3779B97F4A7C15ull) >> (64 - log2);
  for (int p = 0; p < max_probes; ++p) {
    uint64_t k = slot_key[s];
    if (k == key) return true;
    if (k == ~uint64_t(0)) return false;
    s = (s + 1) & mask;
  }
  set_status(status, DEV_HASHFULL);
  return false;
}

// Value of key in the COO (looked up through the hash table); 0 if absent.
__device__ __forceinline__ double hash_value(const uint64_t* slot_key, const uint32_t* slot_idx, int log2,
                             int max_probes, const void* vals, int is64, uint64_t key) {
  const uint64_t mask = (uint64_t(1) << log2) - 1;
  uint64_t s = (key * 0x9E3779B97F4A7C15ull) >> (64 - log2);
  for (int p = 0; p < max_probes; ++p) {
    uint64_t k = slot_key[s];
    if (k == key) return load_as_double(vals, slot_idx[s], is64);
    if (k == ~uint64_t(0)) return 0.0;
    s = (s + 1) & mask;
  }
  return 0.0;
}

// --------------------------------------------------- cross-file launchers

// Division by a small positive integer q as a multiply-high and a shift
// (Granlund and Montgomery, PLDI 1994): for x < 2^16, x / q = (umulhi(x, mul) + x) >> shift
// with shift = ceil(log2 q) and mul = floor(2^32 (2^shift - q) / q) + 1.
struct FastDiv {
  uint32_t q, mul, shift;
};

static inline FastDiv make_fastdiv(uint32_t q) {
  FastDiv f;
  f.q = q;
  uint32_t sh = 0;
  while ((1u << sh) < q) ++sh;
  f.shift = sh;
  f.mul = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << sh) - q)) / q + 1);
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t x, const FastDiv& f) {
  return (__umulhi(x, f.mul) + x) >> f.shift;
}

struct FactorSet {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  int R[TUCKER_MAX_ORDER];
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  int d;
  uint64_t total;   // prod I_n
};

// Scratch of the level walks (walk.cu): the buffer and the sample capacity it was sized for.
struct WalkBuf {
  double* p = nullptr;
  int64_t cap = 0;
  int64_t I2 = 0;                     // I_2: runs of equal (i_1, i_2) along the sorted sample
};

struct RowSet {                       // the deduplicated sample as device arrays
  int N;
  int R[TUCKER_MAX_ORDER];
  int stride[TUCKER_MAX_ORDER];       // prod_{m > n} R_m
  const void* A[TUCKER_MAX_ORDER];
  int is64;
  int d;
  const uint32_t* idx[TUCKER_MAX_ORDER];
  const double* w;
  const int* n_rows;                  // device: number of real rows (prefix of the sample)
};

RowSet make_rowset(const FactorSet& F, uint32_t* const* idx, const double* w, const int* n_rows);

// The lambda-ridge sampler's tables and outputs (ridge.cu).
struct RidgeSampArgs {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  int K[TUCKER_MAX_ORDER];
  int dK;
  const double* usq[TUCKER_MAX_ORDER];     // K_n x I_n
  const double* c;                         // dK
  uint64_t* ccdf;                          // dK: component CDF
  uint64_t* colcdf[TUCKER_MAX_ORDER];      // K_n x I_n: column CDFs
  double* rc;                              // dK: q^c_t / Q^c
  double* rrow[TUCKER_MAX_ORDER];          // I_n x K_n: q^(n,t)_i / Q^(n,t), row-major over i
  uint64_t seed, sweep;
  int64_t m;
  uint64_t* keys_out;                      // m
  int64_t* T_out;                          // nullable: receives T = m
  const uint64_t* keys_u;                  // n_unique sorted keys
  const int* n_unique;
  double* prob;                            // n_unique
  int* status;
};

struct RidgeState {
  RidgeSampArgs a;
};


// leverage.cu
tucker_status launch_leverage(tucker_handle* h, const FactorSet& F, double* const* lev,
                              uint64_t* const* cdf, int* d_rank, double* const* evecs,
                              double* const* evals, double* const* gram_out);
// generic small helpers (exact.cu)
tucker_status launch_gram(tucker_handle* h, const FactorSet& F, double* const* gram);

// sort.cu
tucker_status sort_dedupe(tucker_handle* h, const uint64_t* keys_in, int64_t n, int key_bits,
                          uint64_t* keys_u, uint32_t* counts_u, int* d_n_unique,
                          char* scratch, size_t scratch_bytes);
size_t sort_dedupe_scratch(int64_t n);

// device scan of int64 counts (single CTA; n <= 1<<20).
void launch_scan_i64(tucker_handle* h, const int64_t* in, int64_t* out_excl, int64_t n,
                     int64_t* total);

}  // namespace tk
