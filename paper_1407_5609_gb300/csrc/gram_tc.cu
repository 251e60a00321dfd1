// Dense all-pairs stage on tcgen05 tensor cores (placeholder until the kernel lands).
#include "common.cuh"

namespace cppgb {

bool gram_tc_available() { return false; }

int launch_gram_tc(const void*, int, int64_t, int64_t, int64_t, int64_t, const float*, DenseScalars*, Candidate*,
                   int64_t, cudaStream_t) {
  return set_error(CPPGB_ERR_ARG, "tensor-core filter modes are not available in this build");
}

}  // namespace cppgb
