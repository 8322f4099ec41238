// Product-distribution sampling of rows of K (Alg. 3 line 3; Lemma 4.1 at
// lambda = 0; the N inverse-CDF searches of the proof of Thm 4.2) and the
// observed-entry hash table used for missing data (Sec. 4.2).
//
// Draw t: Philox4x64-10(counter = (t, s, 0, 0), key = (seed, sweep)); mode n
// takes word n%4 of stream s = n/4 as u and selects
//     i_n = min{i : C_n[i] > floor(u * Q_n / 2^64)}          (integer only)
// so every draw is bit-identical to the CPU oracle given the same C_n.  In
// augmented mode (Alg. 1 with d'_eff = 0) the top bit of word 0 of stream 2
// selects a regulariser row j = floor(u' * d / 2^64), u' = word 1 of stream 2.
// The key of a draw is the row-major linear row index of K (prod(I) + j for
// regulariser rows).
#include "common.cuh"

namespace tk {

struct SampleArgs {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  const uint64_t* cdf[TUCKER_MAX_ORDER];
  uint64_t seed;
  uint64_t sweep;
  int reg;
  int d;
  uint64_t total;
  int64_t t0, count;
  uint64_t* keys_out;          // [count] keys of draws t0 .. t0+count-1
  // missing mode (slot_key != nullptr)
  const uint64_t* slot_key;
  int log2;
  int max_probes;
  uint8_t* accept;             // [count]
  int64_t* block_counts;       // [gridDim.x]
  int* status;
  int cdf_in_smem;
  // cutpoint guide tables (Chen & Asau, 1974): for the 2^kbits buckets of the
  // 64-bit uniform u, guide[b] = min{i : C[i] > floor(b Q / 2^kbits)}, the
  // first candidate for every u of bucket b; a forward scan finishes the search
  const uint32_t* guide;              // nullable; modes concatenated
  int64_t gofs[TUCKER_MAX_ORDER];
  int kbits[TUCKER_MAX_ORDER];
  int items;                          // consecutive draws per thread (<= SAMPLE_ITEMS)
  int64_t* T_out;                     // nullable: receives T_val (dense mode: T = m)
  int64_t T_val;
};

__global__ void k_guide(SampleArgs a, uint32_t* guide) {
  for (int n = 0; n < a.N; ++n) {
    const int64_t K = int64_t(1) << a.kbits[n];
    const uint64_t* C = a.cdf[n];
    const int In = (int)a.I[n];
    const uint64_t Q = C[In - 1];
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < K;
         b += (int64_t)gridDim.x * blockDim.x) {
      const uint64_t lb = a.kbits[n] ? __umul64hi((uint64_t)b << (64 - a.kbits[n]), Q) : 0;
      guide[a.gofs[n] + b] = (uint32_t)upper_bound_u64(C, In, lb);
    }
  }
}

constexpr int SAMPLE_THREADS = 256;
constexpr int SAMPLE_ITEMS = 4;            // draws per thread (consecutive)

__device__ __forceinline__ uint64_t draw_key(const SampleArgs& a, const uint64_t* const* C,
                                             const uint32_t* const* Gd, uint64_t t) {
  uint64_t key = 0;
  U64x4 w = philox4x64_10(t, 0, 0, 0, a.seed, a.sweep);
  for (int n = 0; n < a.N; ++n) {
    if (n == 4) w = philox4x64_10(t, 1, 0, 0, a.seed, a.sweep);
    const int In = (int)a.I[n];
    const uint64_t Q = C[n][In - 1];
    const uint64_t u = w.v[n & 3];
    const uint64_t target = __umul64hi(u, Q);
    int i;
    if (Gd) {                                   // min{i : C[i] > target} from the bucket's cutpoint
      i = a.kbits[n] ? (int)Gd[n][u >> (64 - a.kbits[n])] : 0;
      while (C[n][i] <= target) ++i;
    } else {
      i = upper_bound_u64(C[n], In, target);
    }
    key = key * (uint64_t)In + (uint64_t)i;
  }
  if (a.reg == TUCKER_REG_AUGMENTED) {
    U64x4 c = philox4x64_10(t, 2, 0, 0, a.seed, a.sweep);
    if (c.v[0] >> 63) key = a.total + __umul64hi(c.v[1], (uint64_t)a.d);
  }
  return key;
}

__global__ void __launch_bounds__(SAMPLE_THREADS) k_sample(SampleArgs a) {
  pdl_wait();
  extern __shared__ uint64_t scdf[];
  __shared__ int64_t scan_tmp[32];
  const uint64_t* C[TUCKER_MAX_ORDER];
  const uint32_t* Gd[TUCKER_MAX_ORDER];
  bool guided = false;
  if (a.cdf_in_smem) {
    int64_t off = 0;
    for (int n = 0; n < a.N; ++n) {
      for (int64_t i = threadIdx.x; i < a.I[n]; i += blockDim.x) scdf[off + i] = a.cdf[n][i];
      C[n] = scdf + off;
      off += a.I[n];
    }
    if (a.guide) {
      uint32_t* sg = reinterpret_cast<uint32_t*>(scdf + off);
      int64_t tot = 0;
      for (int n = 0; n < a.N; ++n) tot += int64_t(1) << a.kbits[n];
      for (int64_t i = threadIdx.x; i < tot; i += blockDim.x) sg[i] = a.guide[i];
      for (int n = 0; n < a.N; ++n) Gd[n] = sg + a.gofs[n];
      guided = true;
    }
    __syncthreads();
  } else {
    for (int n = 0; n < a.N; ++n) C[n] = a.cdf[n];
  }
  if (a.T_out && blockIdx.x == 0 && threadIdx.x == 0) *a.T_out = a.T_val;
  const int64_t base = (int64_t)blockIdx.x * SAMPLE_THREADS * a.items +
                       (int64_t)threadIdx.x * a.items;
  int nacc = 0;
#pragma unroll
  for (int j = 0; j < SAMPLE_ITEMS; ++j) {
    int64_t e = base + j;
    if (j >= a.items || e >= a.count) break;
    uint64_t key = draw_key(a, C, guided ? Gd : nullptr, (uint64_t)(a.t0 + e));
    a.keys_out[e] = key;
    if (a.slot_key) {
      bool ok = key >= a.total || hash_contains(a.slot_key, a.log2, a.max_probes, key, a.status);
      a.accept[e] = ok;
      nacc += ok;
    }
  }
  if (a.slot_key) {
    int64_t tot;
    block_exclusive_scan(nacc, scan_tmp, &tot);
    if (threadIdx.x == 0) a.block_counts[blockIdx.x] = tot;
  }
}

// Order-preserving compaction of accepted draws: out[acc_base + rank] = key
// while rank < m; the draw that becomes the m-th accepted one records T.
struct CompactArgs {
  const uint64_t* keys;
  const uint8_t* accept;
  const int64_t* block_offsets;   // exclusive scan of block counts
  int64_t count;
  int64_t t0;
  int64_t m;
  int64_t* acc_total;             // device: accepted so far (before this round)
  uint64_t* out;
  int64_t* T_out;
};

__global__ void __launch_bounds__(SAMPLE_THREADS) k_compact(CompactArgs a) {
  __shared__ int64_t scan_tmp[32];
  const int64_t base = (int64_t)blockIdx.x * SAMPLE_THREADS * SAMPLE_ITEMS +
                       (int64_t)threadIdx.x * SAMPLE_ITEMS;
  int flags[SAMPLE_ITEMS];
  int nacc = 0;
#pragma unroll
  for (int j = 0; j < SAMPLE_ITEMS; ++j) {
    int64_t e = base + j;
    flags[j] = (e < a.count) ? a.accept[e] : 0;
    nacc += flags[j];
  }
  int64_t tot;
  int64_t ex = block_exclusive_scan(nacc, scan_tmp, &tot);
  int64_t rank = *a.acc_total + a.block_offsets[blockIdx.x] + ex;
#pragma unroll
  for (int j = 0; j < SAMPLE_ITEMS; ++j) {
    if (!flags[j]) continue;
    if (rank < a.m) a.out[rank] = a.keys[base + j];
    if (rank == a.m - 1) *a.T_out = a.t0 + base + j + 1;
    ++rank;
  }
}

__global__ void k_add_total(int64_t* acc_total, const int64_t* round_total) {
  *acc_total += *round_total;
}

// --------------------------------------------------------------- hash table

__global__ void k_hash_clear(uint64_t* slot_key, uint64_t nslots) {
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < nslots;
       s += (uint64_t)gridDim.x * blockDim.x)
    slot_key[s] = ~uint64_t(0);
}

__global__ void k_hash_build(const uint64_t* keys, int64_t nnz, uint64_t* slot_key,
                             uint32_t* slot_idx, int log2, int max_probes, int* status) {
  const uint64_t mask = (uint64_t(1) << log2) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nnz;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = keys[i];
    uint64_t s = (key * 0x9E3779B97F4A7C15ull) >> (64 - log2);
    int p = 0;
    for (; p < max_probes; ++p) {
      unsigned long long prev = atomicCAS((unsigned long long*)&slot_key[s],
                                          ~0ull, (unsigned long long)key);
      if (prev == ~0ull || prev == key) { slot_idx[s] = (uint32_t)i; break; }
      s = (s + 1) & mask;
    }
    if (p == max_probes) set_status(status, DEV_HASHFULL);
  }
}

// ------------------------------------------------------------------ host side

tucker_status hash_ensure(tucker_handle* h, const tucker_tensor* X, int* probes_out) {
  const int max_probes = 4096;
  *probes_out = max_probes;
  HashTable& ht = h->hash;
  if (ht.src_keys == X->keys && ht.nnz == X->nnz && ht.slot_key) return TUCKER_OK;
  int log2 = 4;
  while ((uint64_t(1) << log2) < uint64_t(X->nnz) * 2 + 16) ++log2;   // load <= 0.5
  if (X->nnz >= (int64_t(1) << 32) - 1)
    return fail(h, TUCKER_EINVAL, "nnz must be < 2^32 - 1");
  uint64_t nslots = uint64_t(1) << log2;
  size_t bytes = nslots * (sizeof(uint64_t) + sizeof(uint32_t));
  if (ht.bytes < bytes) {
    if (ht.slot_key) {
      TK_CUDA(h, cudaStreamSynchronize(h->stream));
      cudaFree(ht.slot_key);
      ht.slot_key = nullptr;
      ht.bytes = 0;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(h, TUCKER_ENOMEM, "hash table of %zu bytes", bytes);
    }
    ht.slot_key = static_cast<uint64_t*>(p);
    ht.bytes = bytes;
  }
  ht.slot_idx = reinterpret_cast<uint32_t*>(ht.slot_key + nslots);
  ht.log2 = log2;
  int grid = h->num_sms * 8;
  TK_COUNT(h);
  k_hash_clear<<<grid, 256, 0, h->stream>>>(ht.slot_key, nslots);
  TK_LAUNCH(h);
  TK_COUNT(h);
  k_hash_build<<<grid, 256, 0, h->stream>>>(X->keys, X->nnz, ht.slot_key, ht.slot_idx, log2,
                                            max_probes, h->d_status);
  TK_LAUNCH(h);
  ht.src_keys = X->keys;
  ht.nnz = X->nnz;
  return TUCKER_OK;
}

static int guide_bits(int64_t I) {
  int kb = 0;
  while (kb < 12 && (int64_t(1) << kb) < I) ++kb;
  return kb;
}

// Bytes sample_keys may take from the caller's arena beyond the caller's own
// buffers: the guide tables and, with observed entries, the per-round buffers.
size_t sample_keys_scratch(const FactorSet& F, bool observed) {
  size_t g = 0;
  for (int n = 0; n < F.N; ++n) g += (size_t(1) << guide_bits(F.I[n])) * 4;
  return g + 512 + (observed ? (size_t)((1 << 26) * 9 + (8 << 20)) : 0);
}

static int cdf_smem_bytes(const SampleArgs& a) {
  int64_t tot = 0;
  for (int n = 0; n < a.N; ++n) tot += a.I[n];
  return tot * 8 <= 160 * 1024 ? (int)(tot * 8) : -1;
}

// Draw keys for the sketch.  Dense: keys_out[0..m).  Missing: rounds of draws
// until m are accepted (host loop, one sync per round).  *T_host receives T;
// d_T (device int64) too.
tucker_status sample_keys(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                          int64_t m, uint64_t seed, uint64_t sweep, int reg,
                          const tucker_tensor* observed, int64_t max_draws,
                          uint64_t* keys_out, int64_t* d_T, int64_t* T_host, Arena& ar) {
  SampleArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  for (int n = 0; n < F.N; ++n) { a.I[n] = F.I[n]; a.cdf[n] = cdf[n]; }
  a.seed = seed;
  a.sweep = sweep;
  a.reg = reg;
  a.d = F.d;
  a.total = F.total;
  a.status = h->d_status;
  int smem = cdf_smem_bytes(a);
  a.cdf_in_smem = smem >= 0;
  if (smem < 0) smem = 0;
  const int64_t expect_draws = observed ? 4 * m : m;
  if (a.cdf_in_smem && expect_draws >= (int64_t(1) << 20)) {
    // guide tables: 2^ceil(log2 I_n) buckets per mode (at most 2^12), if they fit too;
    // only for large draw counts (their build is one more launch)
    int64_t gtot = 0;
    for (int n = 0; n < F.N; ++n) {
      const int kb = guide_bits(F.I[n]);
      a.kbits[n] = kb;
      a.gofs[n] = gtot;
      gtot += int64_t(1) << kb;
    }
    if (smem + gtot * 4 <= 200 * 1024) {
      uint32_t* gbuf = ar.get<uint32_t>(gtot);
      TK_COUNT(h);
      k_guide<<<ceil_div(gtot, 256) < h->num_sms ? ceil_div(gtot, 256) : h->num_sms, 256, 0,
                h->stream>>>(a, gbuf);
      TK_LAUNCH(h);
      a.guide = gbuf;
      smem += (int)(gtot * 4);
    }
  }
  TK_CUDA(h, cudaFuncSetAttribute(k_sample, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int per_block = SAMPLE_THREADS * SAMPLE_ITEMS;
  a.items = SAMPLE_ITEMS;
  if (!observed) {
    // one draw per thread until there are enough draws to fill every SM four times
    a.items = m >= (int64_t)h->num_sms * SAMPLE_THREADS * SAMPLE_ITEMS ? SAMPLE_ITEMS : 1;
    a.t0 = 0;
    a.count = m;
    a.keys_out = keys_out;
    a.T_out = d_T;                          // T = m, written by the kernel
    a.T_val = m;
    TK_CUDA(h, launch_dep(h, k_sample, ceil_div(m, (int64_t)SAMPLE_THREADS * a.items),
                          SAMPLE_THREADS, smem, a));
    *T_host = m;
    return TUCKER_OK;
  }
  int probes = 0;
  TK_TRY(hash_ensure(h, observed, &probes));
  // round size: ~1.5x the expected draws for the observed fraction, >= 2^16
  double frac = double(observed->nnz) / double(F.total);
  if (reg == TUCKER_REG_AUGMENTED) frac = 0.5 + 0.5 * frac;
  int64_t round = (int64_t)(1.5 * double(m) / (frac > 1e-6 ? frac : 1e-6)) + 65536;
  if (round > (int64_t(1) << 26)) round = int64_t(1) << 26;
  const int64_t limit = max_draws > 0 ? max_draws : 64 * m;
  const int nblk = ceil_div(round, per_block);
  uint64_t* tmp_keys = ar.get<uint64_t>(round);
  uint8_t* acc = ar.get<uint8_t>(round);
  int64_t* bc = ar.get<int64_t>(nblk);
  int64_t* bo = ar.get<int64_t>(nblk);
  int64_t* rt = ar.get<int64_t>(2);      // [0] round total, [1] accepted so far
  TK_CUDA(h, cudaMemsetAsync(rt, 0, 2 * sizeof(int64_t), h->stream));
  TK_CUDA(h, cudaMemsetAsync(d_T, 0, sizeof(int64_t), h->stream));
  a.slot_key = h->hash.slot_key;
  a.log2 = h->hash.log2;
  a.max_probes = probes;
  a.keys_out = tmp_keys;
  a.accept = acc;
  a.block_counts = bc;
  int64_t t0 = 0;
  for (;;) {
    int64_t cnt = round;
    if (t0 + cnt > limit) cnt = limit - t0;
    if (cnt <= 0) return fail(h, TUCKER_EDRAWLIMIT, "missing-entry sampling: %lld draws used "
                              "before %lld accepted", (long long)t0, (long long)m);
    a.t0 = t0;
    a.count = cnt;
    int g = ceil_div(cnt, per_block);
    TK_COUNT(h);
    k_sample<<<g, SAMPLE_THREADS, smem, h->stream>>>(a);
    TK_LAUNCH(h);
    launch_scan_i64(h, bc, bo, g, rt);
    TK_LAUNCH(h);
    CompactArgs c;
    c.keys = tmp_keys; c.accept = acc; c.block_offsets = bo; c.count = cnt; c.t0 = t0;
    c.m = m; c.acc_total = rt + 1; c.out = keys_out; c.T_out = d_T;
    TK_COUNT(h);
    k_compact<<<g, SAMPLE_THREADS, 0, h->stream>>>(c);
    TK_LAUNCH(h);
    TK_COUNT(h);
    k_add_total<<<1, 1, 0, h->stream>>>(rt + 1, rt);
    TK_LAUNCH(h);
    int64_t acc_host = 0;
    int st = 0;
    TK_CUDA(h, cudaMemcpyAsync(&acc_host, rt + 1, sizeof(int64_t), cudaMemcpyDeviceToHost,
                               h->stream));
    TK_CUDA(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                               h->stream));
    TK_CUDA(h, cudaStreamSynchronize(h->stream));
    if (st) return device_status(h);
    t0 += cnt;
    if (acc_host >= m) break;
  }
  TK_CUDA(h, cudaMemcpyAsync(T_host, d_T, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
  TK_CUDA(h, cudaStreamSynchronize(h->stream));
  return TUCKER_OK;
}

}  // namespace tk
