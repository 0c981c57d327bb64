// Tensor-core face-products (placeholder until the tcgen05 kernels land).
#include "common.cuh"
#include "internal.cuh"

namespace wp {
size_t tc_facewise_workspace(int64_t, int64_t, int64_t, int64_t, int) { return 0; }
int tc_facewise(const float*, const float*, float*, int64_t, int64_t, int64_t, int64_t, bool, bool,
                int, void*, size_t, cudaStream_t) {
  return WP_ERR_UNSUPPORTED;
}
}  // namespace wp
