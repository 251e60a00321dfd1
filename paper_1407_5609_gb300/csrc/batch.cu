// Batched closest pair + FRNN over many instances (placeholder until the persistent kernel lands).
#include "common.cuh"

extern "C" {
size_t cpp_batch_workspace_size(const cpp_instance*, int64_t) { return 256; }
int cpp_batch(const cpp_instance*, int64_t, cpp_pair_result*, int64_t*, int32_t*, int64_t, void*, size_t, void*) {
  return cppgb::set_error(CPPGB_ERR_ARG, "cpp_batch is not available in this build");
}
}
