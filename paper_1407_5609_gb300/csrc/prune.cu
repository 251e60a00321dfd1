// Reference pruning of the dense stage's tiles: the reference-point bound behind Algorithms MK and
// MPR (Sec. 3.1-3.3), applied to whole tiles instead of single pairs.
//
// For reference points r_k and any two points, the triangle inequality gives
//   d(x_i, x_j) >= | d(r_k, x_i) - d(r_k, x_j) |.
// Each row i gets, for each of PRUNE_REFS reference rows, an interval [lo, hi] that contains the
// exact distance d(r_k, x_i) (computed in FP32 from the stored rows, widened by the rounding bound
// and the rows' residuals eps).  A 128-row block's interval is the hull of its rows' intervals; for
// a tile (row block I, column block J) the gap between I's and J's intervals, maximised over the
// references, is a lower bound on every pair's distance in the tile.  Tiles whose bound exceeds
// sqrt(U0) -- U0 an exact upper bound on the best d^2 -- cannot hold the answer or a tie with it
// and are left out of the dense stage.
//
// U0 follows Algorithm MK's initial best-so-far: the rows are sorted by their distance to the first
// reference and each row is paired with the next few rows of that order (pairs allowed by the
// exclusion); each such pair's distance, computed from the stored rows with a rigorous error bound,
// gives an upper bound on its exact d^2, and U0 is the least of them.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace cppgb {
namespace {

template <class T>
__device__ __forceinline__ float to_f32(T v);
template <>
__device__ __forceinline__ float to_f32<__half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// One warp per row (grid-stride): dot products with the reference rows (staged in shared memory as
// FP32), D~ = |x~_i|^2 + |x~_r|^2 - 2 x~_i.x~_r, v = sqrt(max(D~, 0)), and the interval
//   [v - delta, v + delta],  delta = sqrt(kappa_ref m) + 2u v + eps_i + eps_r,
// m = max |x~|^2: |D~ - |x~_i - x~_r|^2| <= kappa_ref m, |sqrt(a) - sqrt(b)| <= sqrt(|a - b|), one
// rounding of the square root, and the residuals of both rows.
template <class T>
__global__ void __launch_bounds__(256) ref_interval_kernel(const T* __restrict__ X, int64_t n, int64_t n_pad,
                                                           int64_t Kp, const float* __restrict__ norms,
                                                           const float* __restrict__ eps, PruneRefs refs,
                                                           float kappa_ref, const DenseScalars* sc,
                                                           float* __restrict__ lo, float* __restrict__ hi) {
  extern __shared__ float rs[];  // [PRUNE_REFS][Kp]
  for (int64_t e = threadIdx.x; e < (int64_t)PRUNE_REFS * Kp; e += blockDim.x) {
    const int q = (int)(e / Kp);
    rs[e] = to_f32(X[refs.row[q] * Kp + (e - q * Kp)]);
  }
  __syncthreads();
  const float m = __uint_as_float(sc->n2_bits);
  const float root_e = sqrtf(kappa_ref * m) * (1.f + 0x1p-20f);
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); i < n; i += (int64_t)gridDim.x * wpb) {
    float acc[PRUNE_REFS];
#pragma unroll
    for (int q = 0; q < PRUNE_REFS; ++q) acc[q] = 0.f;
    const T* x = X + i * Kp;
    for (int64_t k = lane; k < Kp; k += 32) {
      const float xv = to_f32(x[k]);
#pragma unroll
      for (int q = 0; q < PRUNE_REFS; ++q) acc[q] = fmaf(xv, rs[q * Kp + k], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < PRUNE_REFS; ++q)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane < PRUNE_REFS) {
      float dot = acc[0];
#pragma unroll
      for (int q = 1; q < PRUNE_REFS; ++q) dot = lane == q ? acc[q] : dot;
      const int64_t r = refs.row[lane];
      const float D = (norms[i] + norms[r]) - 2.f * dot;
      const float v = sqrtf(fmaxf(D, 0.f));
      const float delta = ((root_e + 2.f * 0x1p-24f * v) + (eps[i] + eps[r])) * (1.f + 0x1p-20f) + 1e-30f;
      lo[(int64_t)lane * n_pad + i] = __fsub_rd(v, delta);
      hi[(int64_t)lane * n_pad + i] = __fadd_ru(v, delta);
    }
  }
}

// Hull of the rows' intervals per 128-row block and reference (rows < n only; an empty block gets
// the empty interval [+inf, -inf], which excludes every tile it takes part in -- it holds no pair).
// With `perm`, block b holds the rows perm[128 b ..] (sorted positions).
__global__ void block_interval_kernel(const float* __restrict__ lo, const float* __restrict__ hi, int64_t n,
                                      int64_t n_pad, int64_t nbi, const int32_t* __restrict__ perm,
                                      float* __restrict__ blo, float* __restrict__ bhi) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)PRUNE_REFS * nbi) return;
  const int64_t q = e / nbi, b = e % nbi;
  float a = __int_as_float(0x7f800000), z = __int_as_float(0xff800000);
  for (int64_t p = b * 128; p < b * 128 + 128 && p < n; ++p) {
    const int64_t i = perm ? (int64_t)perm[p] : p;
    a = fminf(a, lo[q * n_pad + i]);
    z = fmaxf(z, hi[q * n_pad + i]);
  }
  blo[e] = a;
  bhi[e] = z;
}

// Xs[p] = X[perm[p]] (16-byte words), norms_s[p] = norms[perm[p]]; zero rows past n.
__global__ void permute_rows_kernel(const uint4* __restrict__ X, int64_t n, int64_t n_pad, int64_t words,
                                    const float* __restrict__ norms, const int32_t* __restrict__ perm,
                                    uint4* __restrict__ Xs, float* __restrict__ norms_s) {
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t p = (int64_t)blockIdx.x * wpb + (threadIdx.x >> 5); p < n_pad; p += (int64_t)gridDim.x * wpb) {
    const int64_t src = p < n ? (int64_t)perm[p] : -1;
    for (int64_t w = lane; w < words; w += 32)
      Xs[p * words + w] = src >= 0 ? X[src * words + w] : make_uint4(0u, 0u, 0u, 0u);
    if (lane == 0) norms_s[p] = src >= 0 ? norms[src] : 0.f;
  }
}

// Counting sort of the rows by their distance to reference 0 (65536 buckets over [0, vmax]); the
// order inside a bucket is whatever the atomics give, which only changes which pairs seed U0.
__device__ __forceinline__ int sort_key(float lo0, float hi0, float vmax) {
  const float v = 0.5f * (fmaxf(lo0, 0.f) + hi0);
  const float t = v / vmax * 65536.f;
  return t >= 65535.f ? 65535 : (t > 0.f ? (int)t : 0);
}

__global__ void sort_hist_kernel(const float* __restrict__ lo, const float* __restrict__ hi, int64_t n,
                                 const DenseScalars* sc, int32_t* __restrict__ hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float vmax = 2.f * sqrtf(__uint_as_float(sc->n2_bits)) + 1.f;
  atomicAdd(&hist[sort_key(lo[i], hi[i], vmax)], 1);
}

__global__ void sort_scatter_kernel(const float* __restrict__ lo, const float* __restrict__ hi, int64_t n,
                                    const DenseScalars* sc, const int64_t* __restrict__ start,
                                    int32_t* __restrict__ cursor, int32_t* __restrict__ perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float vmax = 2.f * sqrtf(__uint_as_float(sc->n2_bits)) + 1.f;
  const int k = sort_key(lo[i], hi[i], vmax);
  perm[start[k] + atomicAdd(&cursor[k], 1)] = (int32_t)i;
}

// Seed pairs: one warp per (sorted position p, offset s), s = 1 .. PRUNE_SEEDS; pairs with
// j - i >= excl.  D~ = |x~_i|^2 + |x~_j|^2 - 2 x~_i.x~_j in FP32 (exact 16-bit products, 32-lane
// sums) is within kappa_ref m of |x~_i - x~_j|^2, so with the rows' residuals
//   d(x_i, x_j) <= sqrt(D~ + kappa_ref m) + eps_i + eps_j,
// whose square (rounded up) lowers the running bound U.
template <class T>
__global__ void __launch_bounds__(256) seed_pairs_kernel(const T* __restrict__ X, int64_t Kp,
                                                         const float* __restrict__ norms, const float* __restrict__ eps,
                                                         const int32_t* __restrict__ perm, int64_t n, int64_t excl,
                                                         float kappa_ref, DenseScalars* sc) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t p = w / PRUNE_SEEDS, s = w % PRUNE_SEEDS + 1;
  if (p + s >= n) return;
  const int32_t a = perm[p], b = perm[p + s];
  const int64_t i = a < b ? a : b, j = a < b ? b : a;
  if (j - i < excl) return;  // warp-uniform
  const T* x = X + i * Kp;
  const T* y = X + j * Kp;
  float dot = 0.f;
  for (int64_t k = lane; k < Kp; k += 32) dot = fmaf(to_f32(x[k]), to_f32(y[k]), dot);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  if (lane == 0) {
    const float m = __uint_as_float(sc->n2_bits);
    const float D = (norms[i] + norms[j]) - 2.f * dot;
    const float r = sqrtf(fmaxf(D + kappa_ref * m, 0.f)) * (1.f + 0x1p-20f) + (eps[i] + eps[j]);
    atomic_min_nonneg(&sc->U_bits, r * r * (1.f + 0x1p-19f) + 1e-30f);
  }
}

float kappa_ref_for(int64_t Kp) {
  // dot: 32-lane sums of exact products, (Kp/32 + 5) u each; norms: (Kp/32 + 6) u each; 2 roundings
  // of magnitudes <= 4 m (the epilogue of D~)
  const double u = 0x1p-24, K = (double)Kp;
  return (float)((2.0 * (K / 32.0 + 5.0) * 1.01 * u + 2.0 * (K / 32.0 + 6.0) * 1.01 * u + 8.0 * u) * 1.01);
}

}  // namespace

int launch_prune_intervals(const void* X, int mode, int64_t n, int64_t n_pad, int64_t Kp, const float* norms,
                           const float* eps, const DenseScalars* sc, float* lo, float* hi, float* blo, float* bhi,
                           cudaStream_t st) {
  PruneRefs refs;
  for (int q = 0; q < PRUNE_REFS; ++q) refs.row[q] = (int64_t)(((double)q + 0.5) * (double)n / PRUNE_REFS);
  const float kappa_ref = kappa_ref_for(Kp);
  const size_t smem = (size_t)PRUNE_REFS * (size_t)Kp * sizeof(float);
  if (smem > 200 * 1024) return set_error(CPPGB_ERR_ARG, "pruning supports d <= 5120");
  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)(4 * sms);
  if (mode == CPPGB_MODE_FILTER_BF16) {
    CPPGB_CUDA_TRY(cudaFuncSetAttribute(ref_interval_kernel<__nv_bfloat16>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ref_interval_kernel<__nv_bfloat16><<<grid, 256, smem, st>>>((const __nv_bfloat16*)X, n, n_pad, Kp, norms, eps, refs,
                                                               kappa_ref, sc, lo, hi);
  } else {
    CPPGB_CUDA_TRY(cudaFuncSetAttribute(ref_interval_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
    ref_interval_kernel<__half><<<grid, 256, smem, st>>>((const __half*)X, n, n_pad, Kp, norms, eps, refs, kappa_ref,
                                                        sc, lo, hi);
  }
  CPPGB_LAUNCH_CHECK();
  const int64_t nbi = n_pad / 128;
  block_interval_kernel<<<(unsigned)((PRUNE_REFS * nbi + 255) / 256), 256, 0, st>>>(lo, hi, n, n_pad, nbi, nullptr,
                                                                                   blo, bhi);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_prune_permute(const void* X, int64_t n, int64_t n_pad, int64_t Kp, const float* norms,
                         const int32_t* perm, const float* lo, const float* hi, void* Xs, float* norms_s, float* blo,
                         float* bhi, cudaStream_t st) {
  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  permute_rows_kernel<<<(unsigned)(8 * sms), 256, 0, st>>>((const uint4*)X, n, n_pad, Kp * 2 / 16, norms, perm,
                                                           (uint4*)Xs, norms_s);
  CPPGB_LAUNCH_CHECK();
  const int64_t nbi = n_pad / 128;
  block_interval_kernel<<<(unsigned)((PRUNE_REFS * nbi + 255) / 256), 256, 0, st>>>(lo, hi, n, n_pad, nbi, perm, blo,
                                                                                   bhi);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_prune_seeds(const void* X, int mode, int64_t Kp, const float* norms, const float* eps, const float* lo,
                       const float* hi, int64_t n, int64_t excl, DenseScalars* sc, int32_t* hist, int32_t* cursor,
                       int64_t* start, int64_t* tmp, int32_t* perm, cudaStream_t st) {
  if (n < 2) return CPPGB_OK;
  CPPGB_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int32_t) * 65536, st));
  CPPGB_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int32_t) * 65536, st));
  const unsigned nb = (unsigned)((n + 255) / 256);
  sort_hist_kernel<<<nb, 256, 0, st>>>(lo, hi, n, sc, hist);
  CPPGB_LAUNCH_CHECK();
  int rc = launch_exclusive_scan_i32(hist, 65536, start, tmp, st);
  if (rc) return rc;
  sort_scatter_kernel<<<nb, 256, 0, st>>>(lo, hi, n, sc, start, cursor, perm);
  CPPGB_LAUNCH_CHECK();
  const int64_t warps = n * PRUNE_SEEDS;
  const unsigned sb = (unsigned)((warps + 7) / 8);
  const float kappa_ref = kappa_ref_for(Kp);
  if (mode == CPPGB_MODE_FILTER_BF16)
    seed_pairs_kernel<__nv_bfloat16><<<sb, 256, 0, st>>>((const __nv_bfloat16*)X, Kp, norms, eps, perm, n, excl,
                                                          kappa_ref, sc);
  else
    seed_pairs_kernel<__half><<<sb, 256, 0, st>>>((const __half*)X, Kp, norms, eps, perm, n, excl, kappa_ref, sc);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

}  // namespace cppgb
