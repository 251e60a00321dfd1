// Device-wide exclusive prefix sums (counts -> offsets), used to lay out CSR rows and cell lists.
//
// Three phases per level: each 1024-thread block scans 4096 elements and writes its total; the
// block totals are scanned (recursively, one more level per factor of 4096); the scanned totals
// are added back.  out[n] receives the grand total.
#include "common.cuh"

namespace cppgb {
namespace {

constexpr int SCAN_NT = 1024, SCAN_PER = 4, SCAN_TILE = SCAN_NT * SCAN_PER;

template <class In>
__global__ void __launch_bounds__(SCAN_NT) scan_tile_kernel(const In* __restrict__ in, int64_t n,
                                                            int64_t* __restrict__ out, int64_t* __restrict__ sums) {
  __shared__ int64_t warp_tot[SCAN_NT / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int64_t v[SCAN_PER];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t k = base + (int64_t)tid * SCAN_PER + q;
    v[q] = k < n ? (int64_t)in[k] : 0;
    s += v[q];
  }
  // inclusive scan of the per-thread sums within the warp, then across warps
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
  }
  __syncthreads();
  int64_t run = x - s + (w > 0 ? warp_tot[w - 1] : 0);  // exclusive prefix of this thread
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t k = base + (int64_t)tid * SCAN_PER + q;
    if (k < n) out[k] = run;
    run += v[q];
  }
  if (tid == SCAN_NT - 1) sums[blockIdx.x] = run;
}

__global__ void add_block_offsets_kernel(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] += offs[k / SCAN_TILE];
}

__global__ void write_total_kernel(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ tot) {
  out[n] = *tot;
}

// Reduce-then-scan for up to SCAN_NT tiles: the tile totals, then every tile adds the totals of the
// tiles before it (at most SCAN_NT values, one per thread) and scans itself.  Two launches.
template <class In>
__global__ void __launch_bounds__(SCAN_NT) tile_sum_kernel(const In* __restrict__ in, int64_t n,
                                                           int64_t* __restrict__ sums) {
  __shared__ int64_t red[SCAN_NT / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t k = base + (int64_t)q * SCAN_NT + tid;
    s += k < n ? (int64_t)in[k] : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (w == 0) {
    int64_t t = red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sums[blockIdx.x] = t;
  }
}

template <class In>
__global__ void __launch_bounds__(SCAN_NT) scan_tile_prefixed_kernel(const In* __restrict__ in, int64_t n,
                                                                     int64_t* __restrict__ out,
                                                                     const int64_t* __restrict__ sums) {
  __shared__ int64_t warp_tot[SCAN_NT / 32];
  __shared__ int64_t pre_red[SCAN_NT / 32];
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  // totals of the tiles before this one
  int64_t pv = (sums && tid < (int)blockIdx.x) ? sums[tid] : 0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) pv += __shfl_down_sync(0xffffffffu, pv, o);
  if (lane == 0) pre_red[w] = pv;
  int64_t v[SCAN_PER];
  int64_t s = 0;
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t k = base + (int64_t)tid * SCAN_PER + q;
    v[q] = k < n ? (int64_t)in[k] : 0;
    s += v[q];
  }
  int64_t x = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = warp_tot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;
    int64_t p = pre_red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p += __shfl_down_sync(0xffffffffu, p, o);
    if (lane == 0) pre_red[0] = p;
  }
  __syncthreads();
  int64_t run = pre_red[0] + x - s + (w > 0 ? warp_tot[w - 1] : 0);
#pragma unroll
  for (int q = 0; q < SCAN_PER; ++q) {
    const int64_t k = base + (int64_t)tid * SCAN_PER + q;
    if (k < n) out[k] = run;
    run += v[q];
  }
  if (blockIdx.x == gridDim.x - 1 && tid == SCAN_NT - 1) out[n] = run;
}

template <class In>
int scan_level(const In* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t st) {
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb <= SCAN_NT) {
    if (nb > 1) {
      tile_sum_kernel<In><<<(unsigned)nb, SCAN_NT, 0, st>>>(in, n, tmp);
      CPPGB_LAUNCH_CHECK();
    }
    scan_tile_prefixed_kernel<In><<<(unsigned)nb, SCAN_NT, 0, st>>>(in, n, out, nb > 1 ? tmp : nullptr);
    CPPGB_LAUNCH_CHECK();
    return CPPGB_OK;
  }
  int64_t* sums = tmp;            // nb block totals
  int64_t* sums_scan = tmp + nb;  // their exclusive scan (+ total at [nb])
  scan_tile_kernel<In><<<(unsigned)nb, SCAN_NT, 0, st>>>(in, n, out, sums);
  CPPGB_LAUNCH_CHECK();
  if (nb == 1) {
    write_total_kernel<<<1, 1, 0, st>>>(out, n, sums);
    CPPGB_LAUNCH_CHECK();
    return CPPGB_OK;
  }
  int rc = scan_level<int64_t>(sums, nb, sums_scan, tmp + 2 * nb + 1, st);
  if (rc) return rc;
  add_block_offsets_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, sums_scan);
  CPPGB_LAUNCH_CHECK();
  write_total_kernel<<<1, 1, 0, st>>>(out, n, sums_scan + nb);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

}  // namespace

size_t scan_temp_elems(int64_t n) {
  size_t t = 0;
  while (n > 1) {
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    t += (size_t)(2 * nb + 1);
    n = nb;
  }
  return t + 4;
}

int launch_exclusive_scan_i32(const int32_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t st) {
  if (n <= 0) {
    CPPGB_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return CPPGB_OK;
  }
  return scan_level<int32_t>(in, n, out, tmp, st);
}

int launch_exclusive_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t st) {
  if (n <= 0) {
    CPPGB_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return CPPGB_OK;
  }
  return scan_level<int64_t>(in, n, out, tmp, st);
}

}  // namespace cppgb
