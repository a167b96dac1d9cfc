// Tensor-core tall update (placeholder until the tcgen05 kernel lands).
#include "common.cuh"
#include "internal.h"

namespace rbgs {
size_t tc_gsplit_floats(int64_t K) { return (size_t)(K + 64) * 64 * 2; }
rbgs_status tc_split_g(int64_t, int64_t, const double*, int64_t, float*, const int*, cudaStream_t) {
  return RBGS_EINVAL;
}
rbgs_status tall_update_tc(int64_t, int64_t, int64_t, const float*, int64_t, const float*, int64_t, const float*,
                           float*, int64_t, const int*, cudaStream_t) {
  return RBGS_EINVAL;
}
}  // namespace rbgs
