// Number-theoretic-transform engine (placeholder until the transform lands).
#include "ks_internal.cuh"

namespace ks {

size_t ntt_workspace_bytes(int log_n, int nprod) {
  (void)log_n;
  (void)nprod;
  return 0;
}

cudaError_t launch_ntt_products(const Product *prods, int nprod, int log_n, int d, void *scratch,
                                cudaStream_t s) {
  (void)prods; (void)nprod; (void)log_n; (void)d; (void)scratch; (void)s;
  return cudaErrorNotSupported;
}

}  // namespace ks
