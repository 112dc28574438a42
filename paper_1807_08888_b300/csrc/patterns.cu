#include "nuri_internal.cuh"
namespace nuri {
void topk_patterns(nuri_graph*, int32_t, int32_t, uint32_t, cudaStream_t, nuri_result**) {
  NURI_FAIL(NURI_ERR_INVALID, "pattern queries are not available in this build");
}
}  // namespace nuri
