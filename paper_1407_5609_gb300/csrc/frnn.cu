// Fixed-radius near neighbours (placeholder until the grid kernels land).
#include "common.cuh"

extern "C" {
size_t frnn_query_workspace_size(int64_t, int) { return 256; }
int frnn_query(const float*, int64_t, int, int64_t, double, int64_t*, int32_t*, int64_t, int64_t*, void*, size_t,
               void*) {
  return cppgb::set_error(CPPGB_ERR_ARG, "frnn_query is not available in this build");
}
size_t cpp_batch_workspace_size(const cpp_instance*, int64_t) { return 256; }
int cpp_batch(const cpp_instance*, int64_t, cpp_pair_result*, int64_t*, int32_t*, int64_t, void*, size_t, void*) {
  return cppgb::set_error(CPPGB_ERR_ARG, "cpp_batch is not available in this build");
}
}
