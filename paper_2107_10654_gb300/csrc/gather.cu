// Gather of the sampled entries of vec(X) and the per-row weights (a fused
// pass over the deduplicated sample).
//
// For distinct row u with key k_u and multiplicity c_u:
//   real row (k_u < prod I): i_n from the row-major key; x_u = X[k_u] (dense)
//       or the observed value looked up in the hash table (missing data);
//       p_u = prod_n q_{i_n}/Q_n, evaluated as p = q_1/Q_1, p = p*(q_n/Q_n),
//       then p = 0.5 p in augmented mode (Lemma 4.1 at lambda = 0; Sec. 3
//       augmented distribution);
//   regulariser row j = k_u - prod I (augmented mode): x_u = 0 (b-bar = [b; 0]
//       of Eq. problem_def), p_u = 0.5/d, and D_j = w_u;
//   w_u = c_u / (T p_u)   (squared row scale 1/(Pr(j) s) of Alg. 1, summed
//       over the c_u copies).
// p_u uses the same IEEE operations in the same order as the CPU oracle, so it
// is bit-identical to it.  When per-mode tables are supplied (ftab[i] = q_i/Q_n
// and rtab[i] = 1/ftab[i], one division per factor row instead of several FP64
// divisions per sampled row -- GB300's FP64 rate is 1/64 of FP32), p_u is the
// product of table entries (still bit-identical) and w_u = c_u (1/T) prod_n rtab,
// which differs from c_u / (T p_u) by a few units in the last place.
#include "common.cuh"

namespace tk {

struct IdxPtrs { uint32_t* p[TUCKER_MAX_ORDER]; };

struct GatherArgs {
  int N;
  int64_t I[TUCKER_MAX_ORDER];
  const uint64_t* cdf[TUCKER_MAX_ORDER];
  int reg;
  int d;
  uint64_t total;
  const uint64_t* keys_u;
  const uint32_t* counts;
  const int* n_unique;
  const int64_t* T;
  const void* dense;
  int is64;
  const uint64_t* slot_key;
  const uint32_t* slot_idx;
  int log2, max_probes;
  const void* vals;
  uint32_t* idx[TUCKER_MAX_ORDER];   // [n_unique] per mode (j for regulariser rows in idx[0])
  double* w;
  double* x;
  double* p;
  float* sw32;                        // nullable: sqrt(w) in FP32
  int* n_real;
  double* D;                          // [d], zeroed by the caller
  const double* p_in;                 // nullable: probabilities of a frozen sample
  const double* ftab;                 // nullable: per-mode q_i / Q_n, modes concatenated
  const double* rtab;                 // 1 / ftab
  int64_t toff[TUCKER_MAX_ORDER];     // first entry of mode n in the tables
  int small;                          // prod I_n < 2^32: 32-bit key decode
};

// ftab[off_n + i] = q_i / Q_n, rtab = 1 / ftab, for every factor row of every mode.
__global__ void k_prob_tables(GatherArgs a) {
  for (int n = 0; n < a.N; ++n) {
    const uint64_t* C = a.cdf[n];
    const double Q = (double)C[a.I[n] - 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.I[n];
         i += (int64_t)gridDim.x * blockDim.x) {
      const uint64_t q = C[i] - (i ? C[i - 1] : 0);
      const double f = (double)q / Q;
      const_cast<double*>(a.ftab)[a.toff[n] + i] = f;
      const_cast<double*>(a.rtab)[a.toff[n] + i] = 1.0 / f;
    }
  }
}

__global__ void k_gather_weights(GatherArgs a) {
  const int nu = *a.n_unique;
  const double T = (double)*a.T;
  const double invT = a.rtab ? 1.0 / T : 0.0;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nu; u += gridDim.x * blockDim.x) {
    const uint64_t key = a.keys_u[u];
    double p, x, rinv = 0.0;                     // rinv = 1 / p from the tables
    if (key < a.total) {
      uint32_t ii[TUCKER_MAX_ORDER];
      if (a.small) {
        uint32_t rem = (uint32_t)key;
        for (int n = a.N - 1; n >= 0; --n) {
          const uint32_t In = (uint32_t)a.I[n];
          ii[n] = rem % In;
          rem /= In;
        }
      } else {
        uint64_t rem = key;
        for (int n = a.N - 1; n >= 0; --n) {
          ii[n] = (uint32_t)(rem % (uint64_t)a.I[n]);
          rem /= (uint64_t)a.I[n];
        }
      }
      p = 0.0;
      for (int n = 0; n < a.N; ++n) {
        a.idx[n][u] = ii[n];
        if (a.p_in) continue;
        double f;
        if (a.ftab) {
          f = a.ftab[a.toff[n] + ii[n]];
          const double r = a.rtab[a.toff[n] + ii[n]];
          rinv = n ? rinv * r : r;
        } else {
          const uint64_t* C = a.cdf[n];
          const uint64_t q = C[ii[n]] - (ii[n] ? C[ii[n] - 1] : 0);
          f = (double)q / (double)C[a.I[n] - 1];
        }
        p = n ? p * f : f;
      }
      if (a.p_in) p = a.p_in[u];
      else if (a.reg == TUCKER_REG_AUGMENTED) { p = 0.5 * p; rinv = 2.0 * rinv; }
      if (a.dense) x = load_as_double(a.dense, (int64_t)key, a.is64);
      else if (a.slot_key)
        x = hash_value(a.slot_key, a.slot_idx, a.log2, a.max_probes, a.vals, a.is64, key);
      else x = 0.0;
      if (u == nu - 1) *a.n_real = nu;
    } else {
      const uint32_t j = (uint32_t)(key - a.total);
      p = a.p_in ? a.p_in[u] : 0.5 / (double)a.d;
      x = 0.0;
      for (int n = 0; n < a.N; ++n) a.idx[n][u] = 0;
      a.idx[0][u] = j;
      if (u == 0 || a.keys_u[u - 1] < a.total) *a.n_real = u;
    }
    const bool fast = a.ftab && !a.p_in && key < a.total;
    const double w = fast ? (double)a.counts[u] * (invT * rinv) : (double)a.counts[u] / (T * p);
    a.w[u] = w;
    a.x[u] = x;
    a.p[u] = p;
    if (a.sw32) a.sw32[u] = sqrtf((float)w);
    if (key >= a.total) a.D[key - a.total] = w;
  }
}

// The per-mode probability tables of the gather (they need only the CDFs, so a
// caller may build them beside the sampling and pass tables_ready to the gather).
tucker_status launch_prob_tables(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                                 double* ptab) {
  GatherArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  int64_t sumI = 0;
  for (int n = 0; n < F.N; ++n) {
    a.I[n] = F.I[n];
    a.cdf[n] = cdf[n];
    a.toff[n] = sumI;
    sumI += F.I[n];
  }
  a.ftab = ptab;
  a.rtab = ptab + sumI;
  int tg = ceil_div(F.I[0] > 1024 ? F.I[0] : 1024, 256);
  if (tg > h->num_sms * 4) tg = h->num_sms * 4;
  TK_COUNT(h);
  k_prob_tables<<<tg, 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

tucker_status launch_gather(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                            int reg, const uint64_t* keys_u, const uint32_t* counts,
                            const int* d_nu, const int64_t* d_T, const tucker_tensor* X,
                            int64_t cap, uint32_t* const* idx, double* w, double* x, double* p,
                            float* sw32, int* d_nreal, double* D, const double* p_in,
                            double* ptab, bool tables_ready) {
  GatherArgs a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  for (int n = 0; n < F.N; ++n) { a.I[n] = F.I[n]; a.cdf[n] = cdf[n]; a.idx[n] = idx[n]; }
  a.reg = reg;
  a.d = F.d;
  a.total = F.total;
  a.keys_u = keys_u;
  a.counts = counts;
  a.n_unique = d_nu;
  a.T = d_T;
  a.is64 = X->dtype == TUCKER_F64;
  a.dense = X->dense;
  a.p_in = p_in;
  if (!X->dense && X->keys) {
    a.slot_key = h->hash.slot_key;
    a.slot_idx = h->hash.slot_idx;
    a.log2 = h->hash.log2;
    a.max_probes = 4096;
    a.vals = X->vals;
  }
  a.w = w; a.x = x; a.p = p; a.sw32 = sw32; a.n_real = d_nreal; a.D = D;
  a.small = F.total <= 0xffffffffull;
  TK_CUDA(h, cudaMemsetAsync(D, 0, sizeof(double) * F.d, h->stream));
  if (ptab && !p_in) {
    int64_t sumI = 0;
    for (int n = 0; n < F.N; ++n) { a.toff[n] = sumI; sumI += F.I[n]; }
    a.ftab = ptab;
    a.rtab = ptab + sumI;
    if (!tables_ready) TK_TRY(launch_prob_tables(h, F, cdf, ptab));
  }
  int grid = ceil_div(cap, 256);
  if (grid > h->num_sms * 16) grid = h->num_sms * 16;
  if (grid < 1) grid = 1;
  TK_COUNT(h);
  k_gather_weights<<<grid, 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// Rows of K for every observed entry (exact missing-data update): decode the
// keys into per-mode indices and widen the values to FP64.
__global__ void k_decode_rows(int N, FactorSet F, const uint64_t* keys, int64_t n,
                              uint32_t* const* idxp, IdxPtrs idx, const void* vals, double* x) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    uint64_t rem = keys[u];
    for (int k = N - 1; k >= 0; --k) {
      idx.p[k][u] = (uint32_t)(rem % (uint64_t)F.I[k]);
      rem /= (uint64_t)F.I[k];
    }
    x[u] = load_as_double(vals, u, F.is64);
  }
}

tucker_status launch_decode_rows(tucker_handle* h, const FactorSet& F, const uint64_t* keys,
                                 int64_t n, uint32_t* const* idx, const void* vals, double* x) {
  IdxPtrs ip;
  for (int k = 0; k < F.N; ++k) ip.p[k] = idx[k];
  int grid = ceil_div(n, 256);
  if (grid > h->num_sms * 16) grid = h->num_sms * 16;
  TK_COUNT(h);
  k_decode_rows<<<grid, 256, 0, h->stream>>>(F.N, F, keys, n, nullptr, ip, vals, x);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

// FP64 copies of FP32 factors (the FP64 products with the sampled rows then
// load doubles instead of converting every entry on the FP64 pipe).
struct ToF64Args {
  int N;
  int64_t len[TUCKER_MAX_ORDER];
  const float* src[TUCKER_MAX_ORDER];
  double* dst[TUCKER_MAX_ORDER];
};

__global__ void k_to_f64(ToF64Args a) {
  const int n = blockIdx.y;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.len[n];
       i += (int64_t)gridDim.x * blockDim.x)
    a.dst[n][i] = (double)a.src[n][i];
}

tucker_status launch_to_f64(tucker_handle* h, const FactorSet& F, double* const* out) {
  ToF64Args a;
  memset(&a, 0, sizeof(a));
  a.N = F.N;
  int64_t mx = 1;
  for (int n = 0; n < F.N; ++n) {
    a.len[n] = F.I[n] * F.R[n];
    a.src[n] = static_cast<const float*>(F.A[n]);
    a.dst[n] = out[n];
    if (a.len[n] > mx) mx = a.len[n];
  }
  int gx = ceil_div(mx, 256);
  if (gx > 64) gx = 64;
  TK_COUNT(h);
  k_to_f64<<<dim3(gx, F.N), 256, 0, h->stream>>>(a);
  TK_LAUNCH(h);
  return TUCKER_OK;
}

}  // namespace tk
