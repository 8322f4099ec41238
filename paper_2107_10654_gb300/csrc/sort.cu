// Dedupe of sampled rows: LSD radix sort of the 64-bit keys (8-bit digits,
// only as many passes as the key range needs) followed by a run-length encode
// into (key_u, count_u).  Sampling is with replacement (Alg. 1 loop), so equal
// rows merge into one row of weight c_u / (T p_u).
//
// Each sort pass: per-tile digit histogram -> per-digit exclusive scan over
// the tiles (one CTA per digit) -> stable scatter.  A tile is 4096 keys, 512
// per warp in 16 rounds of 32; inside a round, lanes holding the same digit
// find each other with match_any, so a key's rank is the digit's tile base,
// plus the counts of earlier warps, plus the counts of earlier rounds of its
// warp, plus the equal digits in lower lanes -- input order, hence stable.
#include <cooperative_groups.h>

#include "common.cuh"

namespace tk {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;

// ---------------------------------------------------------- int64 scan (1 CTA)
__global__ void __launch_bounds__(1024) k_scan_i64(const int64_t* in, int64_t* out, int64_t n,
                                                   int64_t* total) {
  pdl_wait();
  __shared__ int64_t tmp[32];
  int64_t carry = 0;
  for (int64_t base = 0; base < n; base += 4 * (int64_t)blockDim.x) {
    int64_t i0 = base + 4 * (int64_t)threadIdx.x;
    int64_t v[4], s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) { v[j] = (i0 + j < n) ? in[i0 + j] : 0; s += v[j]; }
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, tmp, &tot);
    int64_t run = carry + ex;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (i0 + j < n) out[i0 + j] = run;
      run += v[j];
    }
    carry += tot;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

void launch_scan_i64(tucker_handle* h, const int64_t* in, int64_t* out_excl, int64_t n,
                     int64_t* total) {
  // a launch error stays in cudaGetLastError for the caller's check
  (void)launch_dep(h, k_scan_i64, 1, 1024, 0, in, out_excl, n, total);
}

// ------------------------------------------------------------------ radix sort
constexpr int RX = 256;                         // 8-bit digits
constexpr int RX_THREADS = 256;
constexpr int RX_WARPS = RX_THREADS / 32;
constexpr int RX_ROUNDS = 16;
constexpr int RX_TILE = RX_THREADS * RX_ROUNDS;  // 4096 keys

__global__ void __launch_bounds__(RX_THREADS) k_rx_hist(const uint64_t* keys, int64_t n, int shift,
                                                        int* hist, int ntiles) {
  __shared__ int cnt[RX];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * RX_TILE;
#pragma unroll 4
  for (int j = 0; j < RX_ROUNDS; ++j) {
    const int64_t i = base + j * RX_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(int)((keys[i] >> shift) & (RX - 1))], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// rowoff[d][t] = sum_{t' < t} hist[d][t'], tot[d] = sum_t hist[d][t]  (one CTA per digit)
__global__ void __launch_bounds__(1024) k_rx_colscan(const int* hist, int ntiles, int* rowoff,
                                                     int* tot) {
  __shared__ int64_t tmp[32];
  const int* row = hist + (int64_t)blockIdx.x * ntiles;
  int* orow = rowoff + (int64_t)blockIdx.x * ntiles;
  int64_t carry = 0;
  for (int b = 0; b < ntiles; b += 4 * (int)blockDim.x) {
    const int i0 = b + 4 * threadIdx.x;
    int v[4];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) { v[j] = i0 + j < ntiles ? row[i0 + j] : 0; s += v[j]; }
    int64_t all;
    int64_t ex = carry + block_exclusive_scan(s, tmp, &all);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (i0 + j < ntiles) orow[i0 + j] = (int)ex;
      ex += v[j];
    }
    carry += all;
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = (int)carry;
}

__global__ void __launch_bounds__(RX_THREADS) k_rx_scatter(const uint64_t* in, uint64_t* out,
                                                           int64_t n, int shift, const int* rowoff,
                                                           const int* tot, int ntiles) {
  __shared__ int64_t tmp[32];
  __shared__ int wcnt[RX_WARPS][RX];
  __shared__ int wofs[RX_WARPS][RX];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t base = (int64_t)blockIdx.x * RX_TILE + (int64_t)w * (RX_ROUNDS * 32);
  uint64_t k[RX_ROUNDS];
  int dg[RX_ROUNDS];
#pragma unroll
  for (int r = 0; r < RX_ROUNDS; ++r) {
    const int64_t i = base + r * 32 + lane;
    k[r] = i < n ? in[i] : 0;
    dg[r] = i < n ? (int)((k[r] >> shift) & (RX - 1)) : -1;
  }
  for (int d = lane; d < RX; d += 32) wcnt[w][d] = 0;
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int r = 0; r < RX_ROUNDS; ++r) {              // per-warp digit counts
    const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
    if (dg[r] >= 0 && (peers & lt) == 0) wcnt[w][dg[r]] += __popc(peers);
    __syncwarp();
  }
  // digit bases: all tiles' totals of smaller digits, plus this tile's offset
  int64_t all;
  const int64_t dbase = block_exclusive_scan((int64_t)tot[threadIdx.x], tmp, &all) +
                        rowoff[(int64_t)threadIdx.x * ntiles + blockIdx.x];
  {
    int64_t run = dbase;
    for (int ww = 0; ww < RX_WARPS; ++ww) {
      wofs[ww][threadIdx.x] = (int)run;
      run += wcnt[ww][threadIdx.x];
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RX_ROUNDS; ++r) {
    const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
    int pos = 0;
    if (dg[r] >= 0) pos = wofs[w][dg[r]] + __popc(peers & lt);
    __syncwarp();
    if (dg[r] >= 0) {
      out[pos] = k[r];
      if ((peers & lt) == 0) wofs[w][dg[r]] += __popc(peers);
    }
    __syncwarp();
  }
}

// ------------------------------------------------- small samples: one cluster
// For n <= CL_MAX keys the whole sort + dedupe runs in one launch of a cluster
// of CL_CTAS CTAs (CL_CTAS_WIDE, where the device schedules it, up to
// CL_MAX_WIDE keys).  The keys stay in the CTAs' shared memory between passes
// (CTA c holds sorted positions [c CL_CHUNK, (c + 1) CL_CHUNK)): a pass reads
// its 8192 keys (32 warps x 8 rounds x 32 lanes) from its own shared memory,
// ranks them stably as above (per-warp digit counts, rank within a round from
// the lanes holding the same digit), finding those lanes with one ballot per
// digit bit instead of match_any, and stores each key straight into the shared
// memory of the CTA that owns its new position.
// Digits are up to 10 bits (as many passes as the key range needs, all of
// equal width), per-CTA digit totals are exchanged through distributed shared
// memory, and cluster barriers separate the passes.
// Lanes holding the same digit as this lane (invalid lanes carry digit -1):
// the AND of one ballot per digit bit.  Every lane executes every ballot
// (dbits is uniform), so the full mask is always valid.
__device__ __forceinline__ unsigned digit_peers(int dg, int dbits) {
  const unsigned inv = __ballot_sync(0xffffffffu, dg < 0);
  unsigned m = ~inv;
  for (int b = 0; b < dbits; ++b) {
    const int bit = (dg >> b) & 1;
    const unsigned bb = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bb : ~bb;
  }
  return dg < 0 ? inv : m;
}

constexpr int CL_CTAS = 8;                                  // portable cluster size
constexpr int CL_CTAS_WIDE = 16;                            // opt-in size, where schedulable
constexpr int CL_THREADS = 1024;
constexpr int CL_WARPS = CL_THREADS / 32;
constexpr int CL_ROUNDS = 8;
constexpr int CL_CHUNK = CL_THREADS * CL_ROUNDS;            // 8192 keys per CTA
constexpr int64_t CL_MAX = (int64_t)CL_CTAS * CL_CHUNK;     // 65536
constexpr int64_t CL_MAX_WIDE = (int64_t)CL_CTAS_WIDE * CL_CHUNK;   // 131072
constexpr int CL_MAX_DBITS = 10;

static int cl_digit_bits(int key_bits) {
  const int passes = key_bits > 0 ? (key_bits + CL_MAX_DBITS - 1) / CL_MAX_DBITS : 1;
  const int b = (key_bits + passes - 1) / passes;
  return b > 0 ? b : 1;
}

// ints of the per-warp digit table, which afterwards holds the CTA's head positions
static __host__ __device__ int cl_wofs_ints(int dbits) {
  const int t = CL_WARPS << dbits;
  return t > CL_CHUNK ? t : CL_CHUNK;
}

static size_t cl_smem_bytes(int dbits) {
  const size_t rx = size_t(1) << dbits;
  return (size_t)CL_CHUNK * 8 + (size_t)cl_wofs_ints(dbits) * 4 + rx * 4;
}

template <int CTAS>
__global__ void __launch_bounds__(CL_THREADS)
    k_sort_dedupe_cluster(const uint64_t* keys_in, int n, int key_bits, int dbits,
                          uint64_t* keys_u, uint32_t* counts_u, int* d_n_unique) {
  pdl_wait();
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char csm[];
  const int RXB = 1 << dbits;
  uint64_t* kbuf = reinterpret_cast<uint64_t*>(csm);           // this CTA's keys
  int* wofs = reinterpret_cast<int*>(kbuf + CL_CHUNK);         // [CL_WARPS][RXB] counts, offsets
  int* ctot = wofs + cl_wofs_ints(dbits);                      // [RXB] this CTA's digit totals
  __shared__ int64_t tmp[32];
  __shared__ int cta_heads[2];                                // heads, first head position
  const int c = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const int lbase = w * (CL_ROUNDS * 32);
  const int64_t cbase = (int64_t)c * CL_CHUNK;
  uint64_t k[CL_ROUNDS];
  bool valid[CL_ROUNDS];
#pragma unroll
  for (int r = 0; r < CL_ROUNDS; ++r) {
    const int64_t i = cbase + lbase + r * 32 + lane;
    valid[r] = i < n;
    k[r] = valid[r] ? keys_in[i] : 0;
  }
  const uint64_t dmask = (uint64_t)RXB - 1;
  for (int shift = 0; shift < key_bits; shift += dbits) {
    if (shift > 0) {
#pragma unroll
      for (int r = 0; r < CL_ROUNDS; ++r) k[r] = kbuf[lbase + r * 32 + lane];
    }
    int dg[CL_ROUNDS];
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; ++r) dg[r] = valid[r] ? (int)((k[r] >> shift) & dmask) : -1;
    for (int e = threadIdx.x; e < CL_WARPS * RXB; e += CL_THREADS) wofs[e] = 0;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; ++r) {
      const unsigned peers = digit_peers(dg[r], dbits);
      if (dg[r] >= 0 && (peers & lt) == 0) wofs[w * RXB + dg[r]] += __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    for (int t = threadIdx.x; t < RXB; t += CL_THREADS) {     // per-warp exclusive offsets
      int run = 0;
      for (int ww = 0; ww < CL_WARPS; ++ww) {
        const int v = wofs[ww * RXB + t];
        wofs[ww * RXB + t] = run;
        run += v;
      }
      ctot[t] = run;
    }
    cluster.sync();                           // every CTA's totals final; every key loaded
    int64_t all_d = 0, before = 0;
    if (threadIdx.x < RXB) {
      int v[CTAS];
#pragma unroll
      for (int cc = 0; cc < CTAS; ++cc) v[cc] = *cluster.map_shared_rank(&ctot[threadIdx.x], cc);
#pragma unroll
      for (int cc = 0; cc < CTAS; ++cc) {
        all_d += v[cc];
        if (cc < c) before += v[cc];
      }
    }
    int64_t total;
    const int64_t dbase = block_exclusive_scan(threadIdx.x < RXB ? all_d : 0, tmp, &total);
    if (threadIdx.x < RXB)
      for (int ww = 0; ww < CL_WARPS; ++ww) wofs[ww * RXB + threadIdx.x] += (int)(dbase + before);
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; ++r) {
      const unsigned peers = digit_peers(dg[r], dbits);
      int pos = 0;
      if (dg[r] >= 0) pos = wofs[w * RXB + dg[r]] + __popc(peers & lt);
      __syncwarp();
      if (dg[r] >= 0) {
        *cluster.map_shared_rank(kbuf + (pos & (CL_CHUNK - 1)), pos / CL_CHUNK) = k[r];
        if ((peers & lt) == 0) wofs[w * RXB + dg[r]] += __popc(peers);
      }
      __syncwarp();
    }
    cluster.sync();                           // every key in its new place; ctot reads done
  }
  if (key_bits <= 0) {                        // one possible key: the input order is sorted
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; ++r) kbuf[lbase + r * 32 + lane] = k[r];
    cluster.sync();
  }
  // run-length encode: thread t owns sorted positions [cbase + 8 t, +8)
  const int l0 = threadIdx.x * CL_ROUNDS;
  uint64_t prevk = 0;
  if (l0 > 0) prevk = kbuf[l0 - 1];
  else if (c > 0) prevk = *cluster.map_shared_rank(kbuf + (CL_CHUNK - 1), c - 1);
  bool head[CL_ROUNDS];
  uint64_t kr[CL_ROUNDS];
  int nh = 0;
#pragma unroll
  for (int r = 0; r < CL_ROUNDS; ++r) {
    const int64_t i = cbase + l0 + r;
    kr[r] = kbuf[l0 + r];
    head[r] = i < n && (i == 0 || kr[r] != (r ? kr[r - 1] : prevk));
    nh += head[r];
  }
  int64_t cnt;
  const int ul = (int)block_exclusive_scan(nh, tmp, &cnt);     // this thread's first local head
  int* hpos = wofs;                                            // local head -> sorted position
  {
    int q = ul;
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; ++r)
      if (head[r]) hpos[q++] = (int)(cbase + l0 + r);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    cta_heads[0] = (int)cnt;
    cta_heads[1] = cnt > 0 ? hpos[0] : n;
  }
  cluster.sync();
  int64_t ubase = 0, utot = 0;
  int next_first = n;                                          // first head after this CTA
  {
    int hv[CTAS], fv[CTAS];
#pragma unroll
    for (int cc = 0; cc < CTAS; ++cc) {
      hv[cc] = *cluster.map_shared_rank(&cta_heads[0], cc);
      fv[cc] = *cluster.map_shared_rank(&cta_heads[1], cc);
    }
#pragma unroll
    for (int cc = CTAS - 1; cc >= 0; --cc) {
      if (cc < c) ubase += hv[cc];
      utot += hv[cc];
      if (cc > c && hv[cc] > 0) next_first = fv[cc];
    }
  }
  {
    int q = ul;
#pragma unroll
    for (int r = 0; r < CL_ROUNDS; ++r)
      if (head[r]) {
        const int e = q + 1 < (int)cnt ? hpos[q + 1] : next_first;
        keys_u[ubase + q] = kr[r];
        counts_u[ubase + q] = (uint32_t)(e - (int)(cbase + l0 + r));
        ++q;
      }
  }
  if (c == 0 && threadIdx.x == 0) *d_n_unique = (int)utot;
  cluster.sync();                             // no CTA leaves while another reads its heads
}

// ------------------------------------------------------------ run-length encode
__global__ void __launch_bounds__(SORT_THREADS) k_rle_heads(const uint64_t* k, int64_t n,
                                                            int64_t* block_counts) {
  __shared__ int64_t tmp[32];
  const int64_t base = (int64_t)blockIdx.x * SORT_TILE + threadIdx.x * SORT_ITEMS;
  int c = 0;
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j) {
    int64_t i = base + j;
    if (i < n && (i == 0 || k[i] != k[i - 1])) ++c;
  }
  int64_t tot;
  block_exclusive_scan(c, tmp, &tot);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SORT_THREADS) k_rle_write(const uint64_t* k, int64_t n,
                                                            const int64_t* block_offs,
                                                            uint64_t* keys_u, int64_t* start) {
  __shared__ int64_t tmp[32];
  const int64_t base = (int64_t)blockIdx.x * SORT_TILE + threadIdx.x * SORT_ITEMS;
  int c = 0;
  bool head[SORT_ITEMS];
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j) {
    int64_t i = base + j;
    head[j] = i < n && (i == 0 || k[i] != k[i - 1]);
    c += head[j];
  }
  int64_t tot;
  int64_t u = block_offs[blockIdx.x] + block_exclusive_scan(c, tmp, &tot);
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j)
    if (head[j]) { keys_u[u] = k[base + j]; start[u] = base + j; ++u; }
}

__global__ void k_rle_counts(const int64_t* start, const int64_t* n_unique64, int64_t n,
                             uint32_t* counts, int* n_unique) {
  const int64_t nu = *n_unique64;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t e = (u + 1 < nu) ? start[u + 1] : n;
    counts[u] = (uint32_t)(e - start[u]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_unique = (int)nu;
}

size_t sort_dedupe_scratch(int64_t n) {
  const int64_t nb = (n + SORT_TILE - 1) / SORT_TILE;
  const int64_t nt = (n + RX_TILE - 1) / RX_TILE;
  return size_t(n) * 8 * 2 + size_t(RX * nt) * 4 * 2 + RX * 4 + 256 + size_t(nb) * 16 +
         size_t(n) * 8 + 4096;
}

static cudaLaunchConfig_t sort_cluster_cfg(cudaLaunchAttribute* at, int ctas, size_t smem,
                                            cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = ctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(ctas);
  cfg.blockDim = dim3(CL_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cfg;
}

// Whether a 16-CTA cluster of the sort kernel with smem bytes each can be
// scheduled (the device's answer, asked once per size).
static bool wide_cluster_ok(size_t smem) {
  static size_t ok = 0, bad = ~size_t(0);
  if (smem <= ok) return true;
  if (smem >= bad) return false;
  const void* kern = (const void*)k_sort_dedupe_cluster<CL_CTAS_WIDE>;
  int n = 0;
  cudaLaunchAttribute at[1];
  cudaLaunchConfig_t cfg = sort_cluster_cfg(at, CL_CTAS_WIDE, smem, nullptr);
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    bad = smem;
    return false;
  }
  ok = smem;
  return true;
}

template <int CTAS>
static tucker_status launch_sort_cluster(tucker_handle* h, const uint64_t* keys_in, int64_t n,
                                         int key_bits, int dbits, size_t smem, uint64_t* keys_u,
                                         uint32_t* counts_u, int* d_n_unique) {
  const void* kern = (const void*)k_sort_dedupe_cluster<CTAS>;
  if (CTAS > 8)
    TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  TK_CUDA(h, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  cudaLaunchAttribute at[2];
  cudaLaunchConfig_t cfg = sort_cluster_cfg(at, CTAS, smem, h->stream);
  // programmatic dependent launch behind the sampler (the kernel waits first)
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.numAttrs = 2;
  TK_COUNT(h);
  TK_CUDA(h, cudaLaunchKernelEx(&cfg, k_sort_dedupe_cluster<CTAS>, keys_in, (int)n, key_bits,
                                dbits, keys_u, counts_u, d_n_unique));
  return TUCKER_OK;
}

// Sort keys_in[0..n) (keys < 2^key_bits) and deduplicate into keys_u/counts_u;
// *d_n_unique (device) receives the number of distinct keys.
tucker_status sort_dedupe(tucker_handle* h, const uint64_t* keys_in, int64_t n, int key_bits,
                          uint64_t* keys_u, uint32_t* counts_u, int* d_n_unique,
                          char* scratch, size_t scratch_bytes) {
  if (scratch_bytes < sort_dedupe_scratch(n))
    return fail(h, TUCKER_EINTERNAL, "sort scratch too small");
  const int nb = ceil_div(n, SORT_TILE);
  const int nt = ceil_div(n, RX_TILE);
  const int dbits = cl_digit_bits(key_bits);
  const size_t csmem = cl_smem_bytes(dbits);
  if (n <= CL_MAX) return launch_sort_cluster<CL_CTAS>(h, keys_in, n, key_bits, dbits, csmem,
                                                       keys_u, counts_u, d_n_unique);
  if (n <= CL_MAX_WIDE && wide_cluster_ok(csmem))
    return launch_sort_cluster<CL_CTAS_WIDE>(h, keys_in, n, key_bits, dbits, csmem, keys_u,
                                             counts_u, d_n_unique);
  Arena ar(scratch);
  uint64_t* b0 = ar.get<uint64_t>(n);
  uint64_t* b1 = ar.get<uint64_t>(n);
  int* hist = ar.get<int>((size_t)RX * nt);
  int* rowoff = ar.get<int>((size_t)RX * nt);
  int* tot = ar.get<int>(RX);
  int64_t* bc = ar.get<int64_t>(nb);
  int64_t* bo = ar.get<int64_t>(nb + 1);
  int64_t* start = ar.get<int64_t>(n);
  int64_t* nu = bo + nb;
  const uint64_t* cur = keys_in;
  uint64_t* nxt = b0;
  for (int shift = 0; shift < key_bits; shift += 8) {
    TK_COUNT(h);
    k_rx_hist<<<nt, RX_THREADS, 0, h->stream>>>(cur, n, shift, hist, nt);
    TK_LAUNCH(h);
    TK_COUNT(h);
    k_rx_colscan<<<RX, 1024, 0, h->stream>>>(hist, nt, rowoff, tot);
    TK_LAUNCH(h);
    TK_COUNT(h);
    k_rx_scatter<<<nt, RX_THREADS, 0, h->stream>>>(cur, nxt, n, shift, rowoff, tot, nt);
    TK_LAUNCH(h);
    cur = nxt;
    nxt = nxt == b0 ? b1 : b0;
  }
  TK_COUNT(h);
  k_rle_heads<<<nb, SORT_THREADS, 0, h->stream>>>(cur, n, bc);
  launch_scan_i64(h, bc, bo, nb, nu);
  TK_COUNT(h);
  k_rle_write<<<nb, SORT_THREADS, 0, h->stream>>>(cur, n, bo, keys_u, start);
  TK_COUNT(h);
  k_rle_counts<<<ceil_div(n, 256), 256, 0, h->stream>>>(start, nu, n, counts_u, d_n_unique);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
