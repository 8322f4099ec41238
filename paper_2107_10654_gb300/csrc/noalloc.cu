// Allocation-free variant of tucker_sample_rows.
//
// Who needs it: code that must not allocate device memory while it runs,
// for example a caller inside a memory pool it does not own, a process that
// has reserved (or capped) all device memory for itself ahead of time, or a
// real-time loop where a cudaMalloc could stall or fail at an awkward
// moment.  Such callers cannot create a tucker_handle, because the handle
// allocates its workspace on demand.
//
// This entry point runs the same kernels as tucker_sample_rows (fixed-point
// CDFs, Philox draws, radix sort, run-length dedupe, probabilities) but takes
// all of its scratch from one statically sized device array below.  The
// array is part of the library image: every GPU that loads libtucker holds
// these TUCKER_NOALLOC_SCRATCH_BYTES until the process exits.
#include <mutex>

#include "common.cuh"

namespace tk {

tucker_status launch_cdf_from_lev(tucker_handle* h, int N, const int64_t* I,
                                  const double* const* lev, uint64_t* const* cdf,
                                  bool dep = false);
size_t sample_keys_scratch(const FactorSet& F, bool observed);
tucker_status sample_keys(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                          int64_t m, uint64_t seed, uint64_t sweep, int reg,
                          const tucker_tensor* observed, int64_t max_draws,
                          uint64_t* keys_out, int64_t* d_T, int64_t* T_host, Arena& ar);
tucker_status launch_gather(tucker_handle* h, const FactorSet& F, const uint64_t* const* cdf,
                            int reg, const uint64_t* keys_u, const uint32_t* counts,
                            const int* d_nu, const int64_t* d_T, const tucker_tensor* X,
                            int64_t cap, uint32_t* const* idx, double* w, double* x, double* p,
                            float* sw32, int* d_nreal, double* D, const double* p_in,
                            double* ptab, bool tables_ready = false);

// The shared scratch.  Host code must not pass this symbol to a kernel: in
// host code it is only a stand-in, so its device address is looked up with
// cudaGetSymbolAddress once per device (see noalloc_device below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[TUCKER_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;

// Per device: the array's device address and the two attributes the call
// needs, cached after the first successful lookup only (a lookup that failed,
// e.g. behind a pending error of earlier work, is tried again next call).
struct NoallocDevice {
  std::mutex mu;
  bool ready = false;
  void* scratch = nullptr;
  int cc = 0;          // compute capability, major * 10 + minor
  int sms = 0;
};
static NoallocDevice g_dev[kMaxDevices];

// Look up (once per device, with that device current) the device address of
// the scratch array, the compute capability and the SM count.
static cudaError_t noalloc_device(int device, NoallocDevice** out) {
  NoallocDevice& nd = g_dev[device];
  std::lock_guard<std::mutex> lock(nd.mu);
  if (!nd.ready) {
    int major = 0, minor = 0, sms = 0;
    void* p = nullptr;
    cudaError_t e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    if (e == cudaSuccess)
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return e != cudaSuccess ? e : cudaErrorInvalidSymbol;
    }
    nd.scratch = p;
    nd.cc = major * 10 + minor;
    nd.sms = sms;
    nd.ready = true;
  }
  *out = &nd;
  return cudaSuccess;
}

static tucker_status noalloc_fail(char* err, size_t len, tucker_status s, const char* msg) {
  if (err && len) snprintf(err, len, "%s", msg);
  return s;
}

}  // namespace tk

using namespace tk;

extern "C" tucker_status tucker_sample_rows_noalloc(void* cuda_stream, int N, const int64_t* I,
                                                    const int* R, const double* const* lev,
                                                    int64_t m, uint64_t seed, uint32_t sweep,
                                                    tucker_reg reg, tucker_samples* out,
                                                    char* err_host, size_t err_len) {
  if (err_host && err_len) err_host[0] = 0;
  if (!lev || !out || !out->keys || !out->counts || !out->prob || !I || !R)
    return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "null scores, dims, ranks or outputs");
  if (N < 1 || N > TUCKER_MAX_ORDER)
    return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "order out of range");
  if (m < 1 || m >= (int64_t(1) << 31))
    return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "m out of range");
  if (out->capacity < m)
    return noalloc_fail(err_host, err_len, TUCKER_ECAPACITY, "output capacity < m");
  if (reg != TUCKER_REG_EXACT && reg != TUCKER_REG_AUGMENTED)
    return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "bad reg mode");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(err_host, err_len, TUCKER_ECUDA, "no current CUDA device");
  }
  NoallocDevice* nd = nullptr;
  if (noalloc_device(device, &nd) != cudaSuccess)
    return noalloc_fail(err_host, err_len, TUCKER_ECUDA,
                        "device attributes or the scratch array's address could not be read");
  if (nd->cc != 103) return noalloc_fail(err_host, err_len, TUCKER_ENOTSUP, "needs an sm_103 GPU");
  void* scratch = nd->scratch;

  // A handle that lives on the stack and points into the static scratch:
  // no workspace growth, no pinned host buffer, no events are created.
  tucker_handle h;
  h.err[0] = 0;
  h.stream = static_cast<cudaStream_t>(cuda_stream);
  h.device = device;
  h.num_sms = nd->sms;
  int host_status = 0;
  h.h_status = &host_status;
  h.d_status = static_cast<int*>(scratch);               // first 256 bytes
  h.ws = static_cast<char*>(scratch) + 256;
  h.ws_cap = TUCKER_NOALLOC_SCRATCH_BYTES - 256;

  FactorSet F;
  memset(&F, 0, sizeof(F));
  F.N = N;
  int64_t d = 1;
  uint64_t total = 1;
  double tot = 1.0;
  for (int n = 0; n < N; ++n) {
    if (I[n] < 1 || I[n] > (int64_t(1) << 31) || R[n] < 1 || R[n] > TUCKER_MAX_RANK || !lev[n])
      return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "bad dims, ranks or scores");
    F.I[n] = I[n];
    F.R[n] = R[n];
    d *= R[n];
    tot *= double(I[n]);
    total *= (uint64_t)I[n];
  }
  if (d > 8192) return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "prod(R_n) exceeds 8192");
  // linear row keys must not wrap: the same bound as tucker_sample_rows
  if (tot >= 4.0e18) return noalloc_fail(err_host, err_len, TUCKER_EINVAL, "prod(I_n) too large");
  F.d = (int)d;
  F.total = total;

  // Same buffer plan as tucker_sample_rows, checked against the fixed size.
  uint64_t* cdf[TUCKER_MAX_ORDER];
  uint32_t* idx[TUCKER_MAX_ORDER];
  auto carve = [&](Arena& ar, uint64_t** raw, int64_t** dT, char** ss, int** nu, int** nreal,
                   double** w, double** x, double** D) {
    for (int n = 0; n < N; ++n) cdf[n] = ar.get<uint64_t>(F.I[n]);
    *raw = ar.get<uint64_t>(m);
    *dT = ar.get<int64_t>(1);
    *ss = ar.get<char>(sort_dedupe_scratch(m));
    *nu = ar.get<int>(1);
    *nreal = ar.get<int>(1);
    for (int n = 0; n < N; ++n) idx[n] = ar.get<uint32_t>(m);
    *w = ar.get<double>(m);
    *x = ar.get<double>(m);
    *D = ar.get<double>(F.d);
  };
  uint64_t* raw;
  int64_t* dT;
  char* ss;
  int *nu, *nreal;
  double *w, *x, *D;
  Arena sz(nullptr);
  carve(sz, &raw, &dT, &ss, &nu, &nreal, &w, &x, &D);
  if (sz.off + sample_keys_scratch(F, false) > h.ws_cap) {
    char msg[200];
    snprintf(msg, sizeof(msg), "m = %lld needs %zu scratch bytes; the fixed array holds %zu "
             "(TUCKER_NOALLOC_SCRATCH_BYTES)", (long long)m, sz.off + sample_keys_scratch(F, false),
             h.ws_cap);
    return noalloc_fail(err_host, err_len, TUCKER_ECAPACITY, msg);
  }
  Arena ar(h.ws);
  carve(ar, &raw, &dT, &ss, &nu, &nreal, &w, &x, &D);

  // The status word is the only scratch that must start at zero; every other
  // buffer is fully written before it is read.
  if (cudaMemsetAsync(h.d_status, 0, sizeof(int), h.stream) != cudaSuccess) {
    cudaGetLastError();
    return noalloc_fail(err_host, err_len, TUCKER_ECUDA, "cudaMemsetAsync failed");
  }
  tucker_status st = launch_cdf_from_lev(&h, N, I, lev, cdf);
  int64_t T = 0;
  if (st == TUCKER_OK)
    st = sample_keys(&h, F, cdf, m, seed, sweep, reg, nullptr, 0, raw, dT, &T, ar);
  if (st == TUCKER_OK) {
    uint64_t range = F.total + (reg == TUCKER_REG_AUGMENTED ? (uint64_t)F.d : 0);
    int bits = 1;
    while (bits < 64 && (range - 1) >> bits) ++bits;
    st = sort_dedupe(&h, raw, m, bits, out->keys, out->counts, nu, ss, sort_dedupe_scratch(m));
  }
  if (st == TUCKER_OK) {
    tucker_tensor none;
    memset(&none, 0, sizeof(none));
    none.order = N;
    none.dtype = TUCKER_F64;
    st = launch_gather(&h, F, cdf, reg, out->keys, out->counts, nu, dT, &none, m, idx, w, x,
                       out->prob, nullptr, nreal, D, nullptr, nullptr);
  }
  int nuh = 0;
  if (st == TUCKER_OK) {
    if (cudaMemcpyAsync(&nuh, nu, sizeof(int), cudaMemcpyDeviceToHost, h.stream) != cudaSuccess) {
      cudaGetLastError();
      st = TUCKER_ECUDA;
    }
  }
  if (st == TUCKER_OK) st = device_status(&h);
  if (st != TUCKER_OK) {
    if (err_host && err_len) snprintf(err_host, err_len, "%s", h.err[0] ? h.err : "device error");
    return st;
  }
  out->n_unique = nuh;
  out->n_draws = T;
  return TUCKER_OK;
}
