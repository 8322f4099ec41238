// Dedupe of sampled rows: LSD radix sort of the 64-bit keys (4-bit digits,
// only as many passes as the key range needs) followed by a run-length encode
// into (key_u, count_u).  Sampling is with replacement (Alg. 1 loop), so equal
// rows merge into one row of weight c_u / (T p_u).
//
// Each sort pass: per-tile digit histogram -> exclusive scan over
// (digit, tile) -> stable scatter.  A tile is 256 threads x 8 consecutive keys;
// the rank of a key inside its tile is its digit's tile offset plus the number
// of equal digits in earlier threads (block scan over digit-major counters)
// plus the equal digits earlier in the same thread, which keeps the sort stable.
#include "common.cuh"

namespace tk {

constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int RADIX = 16;

// ---------------------------------------------------------- int64 scan (1 CTA)
__global__ void __launch_bounds__(1024) k_scan_i64(const int64_t* in, int64_t* out, int64_t n,
                                                   int64_t* total) {
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
  TK_COUNT(h);
  k_scan_i64<<<1, 1024, 0, h->stream>>>(in, out_excl, n, total);
}

// ------------------------------------------------------------------ radix sort
__global__ void __launch_bounds__(SORT_THREADS) k_radix_hist(const uint64_t* keys, int64_t n,
                                                             int shift, int64_t* hist,
                                                             int nblocks) {
  __shared__ unsigned cnt[RADIX];
  if (threadIdx.x < RADIX) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * SORT_TILE + threadIdx.x * SORT_ITEMS;
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j)
    if (base + j < n) atomicAdd(&cnt[(keys[base + j] >> shift) & (RADIX - 1)], 1u);
  __syncthreads();
  if (threadIdx.x < RADIX) hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(SORT_THREADS) k_radix_scatter(const uint64_t* in, uint64_t* out,
                                                                int64_t n, int shift,
                                                                const int64_t* offs,
                                                                int nblocks) {
  __shared__ int64_t cnt[RADIX * SORT_THREADS];     // digit-major [digit][thread]
  __shared__ int64_t tmp[32];
  __shared__ int64_t tile_start[RADIX];
  const int t = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * SORT_TILE + t * SORT_ITEMS;
  uint64_t k[SORT_ITEMS];
  int dg[SORT_ITEMS];
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j) {
    k[j] = (base + j < n) ? in[base + j] : ~uint64_t(0);
    dg[j] = (int)((k[j] >> shift) & (RADIX - 1));
  }
#pragma unroll
  for (int d = 0; d < RADIX; ++d) {
    int c = 0;
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) c += (dg[j] == d);
    cnt[d * SORT_THREADS + t] = c;
  }
  __syncthreads();
  // exclusive scan of the flat digit-major array; thread t owns 16 consecutive entries
  int64_t loc[RADIX], s = 0;
#pragma unroll
  for (int j = 0; j < RADIX; ++j) { loc[j] = cnt[t * RADIX + j]; s += loc[j]; }
  int64_t tot;
  int64_t ex = block_exclusive_scan(s, tmp, &tot);
#pragma unroll
  for (int j = 0; j < RADIX; ++j) { cnt[t * RADIX + j] = ex; ex += loc[j]; }
  __syncthreads();
  if (t < RADIX) tile_start[t] = cnt[t * SORT_THREADS];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < SORT_ITEMS; ++j) {
    if (base + j >= n) break;
    int before = 0;
#pragma unroll
    for (int jj = 0; jj < j; ++jj) before += (dg[jj] == dg[j]);
    int64_t r = cnt[dg[j] * SORT_THREADS + t] + before - tile_start[dg[j]];
    out[offs[(int64_t)dg[j] * nblocks + blockIdx.x] + r] = k[j];
  }
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
  int64_t nb = (n + SORT_TILE - 1) / SORT_TILE;
  return size_t(n) * 8 * 2 + size_t(RADIX * nb) * 8 * 2 + size_t(nb) * 16 + size_t(n) * 8 + 4096;
}

// Sort keys_in[0..n) (keys < 2^key_bits) and deduplicate into keys_u/counts_u;
// *d_n_unique (device) receives the number of distinct keys.
tucker_status sort_dedupe(tucker_handle* h, const uint64_t* keys_in, int64_t n, int key_bits,
                          uint64_t* keys_u, uint32_t* counts_u, int* d_n_unique,
                          char* scratch, size_t scratch_bytes) {
  if (scratch_bytes < sort_dedupe_scratch(n))
    return fail(h, TUCKER_EINTERNAL, "sort scratch too small");
  const int nb = ceil_div(n, SORT_TILE);
  Arena ar(scratch);
  uint64_t* b0 = ar.get<uint64_t>(n);
  uint64_t* b1 = ar.get<uint64_t>(n);
  int64_t* hist = ar.get<int64_t>((size_t)RADIX * nb);
  int64_t* offs = ar.get<int64_t>((size_t)RADIX * nb);
  int64_t* bc = ar.get<int64_t>(nb);
  int64_t* bo = ar.get<int64_t>(nb + 1);
  int64_t* start = ar.get<int64_t>(n);
  int64_t* nu = bo + nb;
  TK_CUDA(h, cudaMemcpyAsync(b0, keys_in, n * 8, cudaMemcpyDeviceToDevice, h->stream));
  const uint64_t* cur = b0;
  uint64_t* nxt = b1;
  for (int shift = 0; shift < key_bits; shift += 4) {
    TK_COUNT(h);
    k_radix_hist<<<nb, SORT_THREADS, 0, h->stream>>>(cur, n, shift, hist, nb);
    launch_scan_i64(h, hist, offs, (int64_t)RADIX * nb, nullptr);
    TK_COUNT(h);
    k_radix_scatter<<<nb, SORT_THREADS, 0, h->stream>>>(cur, nxt, n, shift, offs, nb);
    TK_LAUNCH(h);
    const uint64_t* t = cur;
    cur = nxt;
    nxt = const_cast<uint64_t*>(t);
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
