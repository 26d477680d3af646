// Tensor-core (tcgen05) grade product for the mixed path: placeholder until implemented.
#include "mtp_internal.h"

namespace mtp {
bool grade_tc_available(const mtp_model*) { return false; }
void run_grade_tc(mtp_model*, int64_t, const float*, const float*, int64_t, double*, int32_t*, cudaStream_t) {
  throw Fail{MTP_ERR_UNSUPPORTED, "tensor-core grade not built"};
}
}  // namespace mtp
