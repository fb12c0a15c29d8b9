// Split-IMEX internal step (not built yet: entry points report unsupported).
#include "slim_split.h"

namespace slim {
size_t split_aux2d_len(const DevMesh& m) { return (size_t)16 * m.n_tri; }
slim_status split_rhs2d(slim_state*, double, double*, cudaStream_t) {
  set_error("split scheme not available");
  return SLIM_ERR_UNSUPPORTED;
}
slim_status split_step(slim_state*, double, double, cudaStream_t) {
  set_error("split scheme not available");
  return SLIM_ERR_UNSUPPORTED;
}
int split_kernel_count(const slim_state*) { return 0; }
}  // namespace slim
