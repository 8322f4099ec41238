// Tensor-core (tcgen05) Gram of the implicit Kronecker rows: placeholder
// until the sm_103a kernel lands; reports the precisions as unsupported.
#include "common.cuh"

namespace tk {

int gram_tc_supported(int prec, int d) { (void)prec; (void)d; return 0; }

size_t gram_tc_workspace(tucker_handle* h, int prec, int d, int64_t cap) {
  (void)h; (void)prec; (void)d; (void)cap;
  return 0;
}

tucker_status launch_gram_tc(tucker_handle* h, const RowSet& s, int prec, int64_t cap, char* ws,
                             size_t ws_bytes, double* G) {
  (void)s; (void)prec; (void)cap; (void)ws; (void)ws_bytes; (void)G;
  return fail(h, TUCKER_ENOTSUP, "tensor-core Gram not available");
}

}  // namespace tk
