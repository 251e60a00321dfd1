// ALU peak microbenchmarks (diagnostics; no counterpart in the paper): the two CUDA-core rates the
// roofline of the FP32 dense path and of the two-locus POPC scan are measured against.
//
//   FFMA  every thread runs FF_CHAINS independent fused multiply-add chains (2 flop each); the
//         chains are independent, so the FMA pipe, not the dependence latency, sets the rate.
//   POPC  every thread runs PC_CHAINS independent chains a = popc(a ^ k) + a: one POPC and one
//         integer add per step; the add runs on the full-rate integer pipe, the POPC on the
//         quarter-rate one, so the POPC pipe sets the rate.
// Both run on a full persistent grid (8 blocks of 256 threads per SM) and are timed with CUDA events;
// the results are written out so that no work can be dropped.
#include "common.cuh"

namespace cppgb {
namespace {

constexpr int PK_NT = 256, PK_BLOCKS_PER_SM = 8;
constexpr int FF_CHAINS = 8, PC_CHAINS = 8;

__global__ void __launch_bounds__(PK_NT) ffma_peak_kernel(float* __restrict__ out, int iters, float a, float b) {
  float x[FF_CHAINS];
#pragma unroll
  for (int c = 0; c < FF_CHAINS; ++c) x[c] = (float)(threadIdx.x + c);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < FF_CHAINS; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < FF_CHAINS; ++c) s += x[c];
  out[blockIdx.x * PK_NT + threadIdx.x] = s;
}

__global__ void __launch_bounds__(PK_NT) popc_peak_kernel(unsigned* __restrict__ out, int iters, unsigned k) {
  unsigned x[PC_CHAINS];
#pragma unroll
  for (int c = 0; c < PC_CHAINS; ++c) x[c] = threadIdx.x * 0x9e3779b9u + (unsigned)c;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < PC_CHAINS; ++c) x[c] = (unsigned)__popc(x[c] ^ (k + (unsigned)u)) + x[c];
  }
  unsigned s = 0u;
#pragma unroll
  for (int c = 0; c < PC_CHAINS; ++c) s ^= x[c];
  out[blockIdx.x * PK_NT + threadIdx.x] = s;
}

}  // namespace
}  // namespace cppgb

using namespace cppgb;

extern "C" {

int cpp_measure_alu_peaks(double* ffma_tflops, double* popc_tops) {
  if (!ffma_tflops || !popc_tops) return set_error(CPPGB_ERR_ARG, "output pointers are NULL");
  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * PK_BLOCKS_PER_SM;
  void* buf = nullptr;
  CPPGB_CUDA_TRY(cudaMalloc(&buf, sizeof(float) * (size_t)blocks * PK_NT));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](auto launch, int reps) -> double {
    launch();  // warm-up
    cudaEventRecord(e0, 0);
    for (int r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, 0);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return (double)ms / reps;
  };
  const int iters = 2048;
  const double ops = (double)blocks * PK_NT * iters * 16;
  const double ms_f = timed([&] { ffma_peak_kernel<<<blocks, PK_NT>>>((float*)buf, iters, 0.999999f, 1e-7f); }, 5);
  const double ms_p = timed([&] { popc_peak_kernel<<<blocks, PK_NT>>>((unsigned*)buf, iters, 0x5bd1e995u); }, 5);
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(buf);
  if (err != cudaSuccess) return set_error(CPPGB_ERR_CUDA, "peak kernels failed: %s", cudaGetErrorString(err));
  *ffma_tflops = ops * FF_CHAINS * 2.0 / (ms_f * 1e-3) / 1e12;
  *popc_tops = ops * PC_CHAINS / (ms_p * 1e-3) / 1e12;
  return CPPGB_OK;
}

}  // extern "C"
