// Row preparation for the dense all-pairs stage.
//
// Each row x_i of the search (a point of the CPP, or a z-normalised l-mer of the motif search) is
// stored as x~_i in the dense stage's element type (FP32, FP16 or BF16), padded with zeros to Kp
// columns and n_pad rows.  Alongside it go |x~_i|^2 (FP32) and eps_i, an upper bound on the
// Euclidean distance |x_i - x~_i| between the exact row and the stored one.  By the triangle
// inequality every pair then satisfies | |x_i - x_j| - |x~_i - x~_j| | <= eps_i + eps_j, which is
// what makes the low-precision filter exact after the FP64 recheck.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace cppgb {
namespace {

constexpr float kU32 = 0x1p-24f;  // unit roundoff of FP32

template <class T>
__device__ __forceinline__ T to_elem(float v);
template <>
__device__ __forceinline__ float to_elem<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half to_elem<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

__device__ __forceinline__ float from_elem(float v) { return v; }
__device__ __forceinline__ float from_elem(__half v) { return __half2float(v); }
__device__ __forceinline__ float from_elem(__nv_bfloat16 v) { return __bfloat162float(v); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-block maxima of eps and |x~|^2, then one atomic per block.
__device__ __forceinline__ void block_max_to(float eps, float n2, DenseScalars* sc) {
  __shared__ float s_eps[32], s_n2[32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  eps = warp_max(eps);
  n2 = warp_max(n2);
  if (lane == 0) { s_eps[w] = eps; s_n2[w] = n2; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    float e = lane < nw ? s_eps[lane] : 0.f, q = lane < nw ? s_n2[lane] : 0.f;
    e = warp_max(e);
    q = warp_max(q);
    if (lane == 0) {
      atomic_max_nonneg(&sc->eps_bits, e);
      atomic_max_nonneg(&sc->n2_bits, q);
    }
  }
}

// One warp per row.  Points: x_ik read as FP64 or FP32, stored rounded to T.
template <class T, class Src>
__global__ void __launch_bounds__(256) prep_points_kernel(const Src* __restrict__ pts, int64_t n, int64_t d,
                                                         int64_t ld, T* __restrict__ X, int64_t n_pad,
                                                         int64_t Kp, float* __restrict__ norms,
                                                         float* __restrict__ eps_out, DenseScalars* sc) {
  int lane = threadIdx.x & 31;
  int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float n2 = 0.f, dd = 0.f, xx = 0.f;
  bool bad = false;
  if (row < n_pad) {
    T* out = X + row * Kp;
    for (int64_t k = lane; k < Kp; k += 32) {
      float q = 0.f;
      if (row < n && k < d) {
        Src x = pts[row * ld + k];
        bad |= !isfinite((double)x) ;
        float r = (float)x;  // rounding of an FP64 input to FP32: error <= 2^-24 |x| (added below)
        T t = to_elem<T>(r);
        q = from_elem(t);
        bad |= !isfinite(q);
        float dl = r - q;  // exact in FP32
        dd = fmaf(dl, dl, dd);
        xx = fmaf(r, r, xx);
        out[k] = t;
      } else {
        out[k] = to_elem<T>(0.f);
      }
      n2 = fmaf(q, q, n2);
    }
  }
  n2 = warp_sum(n2);
  dd = warp_sum(dd);
  xx = warp_sum(xx);
  bad = __any_sync(0xffffffffu, bad);
  float e = 0.f;
  if (row < n) {
    // |x - x~| <= |x - fl32(x)| + |fl32(x) - x~|; the first is <= 2^-24 |x| for FP64 input,
    // plus a subnormal allowance; sums are padded by 2^-10 for their own FP32 error.
    float r32 = sizeof(Src) == 8 ? kU32 * sqrtf(xx) * 1.001f + sqrtf((float)d) * 0x1p-149f : 0.f;
    e = (sqrtf(dd) * (1.f + 0x1p-10f) + r32);
    if (lane == 0) {
      norms[row] = n2;
      eps_out[row] = e;
      if (bad) atomicOr(&sc->status, 1u);
    }
  } else if (row < n_pad && lane == 0) {
    norms[row] = 0.f;
    eps_out[row] = 0.f;
  }
  block_max_to(e, n2 * (1.f + 0x1p-12f), sc);
}

// One warp per l-mer T_i = a_i .. a_{i+l-1} (Sec. 2).  z-normalisation in FP32:
//   c_k = a_{i+k} - a_i (shift by the first sample: exact in real arithmetic for z, and keeps the
//   values small), mu = mean(c) (Kahan per lane + tree), v = sum (c_k - mu)^2, sigma = sqrt(v / l),
//   z_k = (c_k - mu) / sigma.
// Error of the FP32 z-row against the exact one (derivation in the design notes):
//   |z - z*| <= sqrt(l) * u * (22 M / sigma + 11),  M = max_k |c_k|,  taken x2 for safety.
template <class T>
__global__ void __launch_bounds__(256) prep_lmers_kernel(const float* __restrict__ a, int64_t n, int64_t l,
                                                        T* __restrict__ X, int64_t n_pad, int64_t Kp,
                                                        float* __restrict__ norms, float* __restrict__ eps_out,
                                                        DenseScalars* sc) {
  int lane = threadIdx.x & 31;
  int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  float e = 0.f, n2 = 0.f;
  if (row < n) {
    const float* w = a + row;
    float base = w[0];
    // mean of the shifted window
    float s = 0.f, comp = 0.f, M = 0.f;
    bool bad = false;
    for (int64_t k = lane; k < l; k += 32) {
      float x = w[k];
      bad |= !isfinite(x);
      float c = x - base;
      M = fmaxf(M, fabsf(c));
      float y = c - comp;
      float t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    s = warp_sum(s);
    M = warp_max(M);
    bad = __any_sync(0xffffffffu, bad);
    float mu = s / (float)l;
    float v = 0.f, vc = 0.f;
    for (int64_t k = lane; k < l; k += 32) {
      float c = (w[k] - base) - mu;
      float y = fmaf(c, c, -vc);
      float t = v + y;
      vc = (t - v) - y;
      v = t;
    }
    v = warp_sum(v);
    float sd = sqrtf(v / (float)l);
    bool degenerate = bad || !(sd > 0.f) || !isfinite(sd);
    float dd = 0.f;
    T* out = X + row * Kp;
    for (int64_t k = lane; k < Kp; k += 32) {
      float q = 0.f;
      if (k < l && !degenerate) {
        float z = __fdiv_rn((w[k] - base) - mu, sd);
        T t = to_elem<T>(z);
        q = from_elem(t);
        float dl = z - q;  // exact in FP32
        dd = fmaf(dl, dl, dd);
        out[k] = t;
      } else {
        out[k] = to_elem<T>(0.f);
      }
      n2 = fmaf(q, q, n2);
    }
    n2 = warp_sum(n2);
    dd = warp_sum(dd);
    float sl = sqrtf((float)l);
    float e_prep = 2.f * sl * kU32 * (22.f * (M / sd) + 11.f);
    e = degenerate ? 0.f : sqrtf(dd) * (1.f + 0x1p-10f) + e_prep;
    if (lane == 0) {
      norms[row] = n2;
      eps_out[row] = e;
      if (bad) atomicOr(&sc->status, 1u);
      else if (degenerate) atomicOr(&sc->status, 2u);
    }
  } else if (row < n_pad) {
    T* out = X + row * Kp;
    for (int64_t k = lane; k < Kp; k += 32) out[k] = to_elem<T>(0.f);
    if (lane == 0) { norms[row] = 0.f; eps_out[row] = 0.f; }
  }
  block_max_to(e, n2 * (1.f + 0x1p-12f), sc);
}

template <class T>
int prep_points_t(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, void* X, int64_t n_pad,
                  int64_t Kp, float* norms, float* eps, DenseScalars* sc, cudaStream_t st) {
  int64_t blocks = (n_pad + 7) / 8;
  if (blocks == 0) return CPPGB_OK;
  if (dtype == CPPGB_F64)
    prep_points_kernel<T, double><<<(unsigned)blocks, 256, 0, st>>>((const double*)pts, n, d, ld, (T*)X, n_pad,
                                                                     Kp, norms, eps, sc);
  else
    prep_points_kernel<T, float><<<(unsigned)blocks, 256, 0, st>>>((const float*)pts, n, d, ld, (T*)X, n_pad,
                                                                    Kp, norms, eps, sc);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

template <class T>
int prep_lmers_t(const float* series, int64_t n, int64_t l, void* X, int64_t n_pad, int64_t Kp, float* norms,
                 float* eps, DenseScalars* sc, cudaStream_t st) {
  int64_t blocks = (n_pad + 7) / 8;
  if (blocks == 0) return CPPGB_OK;
  prep_lmers_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(series, n, l, (T*)X, n_pad, Kp, norms, eps, sc);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

}  // namespace

int launch_prep_points(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, void* X,
                       int64_t n_pad, int64_t Kp, float* norms, float* eps, DenseScalars* sc, cudaStream_t st) {
  switch (mode) {
    case CPPGB_MODE_PLAIN_FP32: return prep_points_t<float>(pts, dtype, n, d, ld, X, n_pad, Kp, norms, eps, sc, st);
    case CPPGB_MODE_FILTER_FP16: return prep_points_t<__half>(pts, dtype, n, d, ld, X, n_pad, Kp, norms, eps, sc, st);
    case CPPGB_MODE_FILTER_BF16:
      return prep_points_t<__nv_bfloat16>(pts, dtype, n, d, ld, X, n_pad, Kp, norms, eps, sc, st);
  }
  return set_error(CPPGB_ERR_ARG, "unknown mode %d", mode);
}

int launch_prep_lmers(const float* series, int64_t n, int64_t l, int mode, void* X, int64_t n_pad, int64_t Kp,
                      float* norms, float* eps, DenseScalars* sc, cudaStream_t st) {
  switch (mode) {
    case CPPGB_MODE_PLAIN_FP32: return prep_lmers_t<float>(series, n, l, X, n_pad, Kp, norms, eps, sc, st);
    case CPPGB_MODE_FILTER_FP16: return prep_lmers_t<__half>(series, n, l, X, n_pad, Kp, norms, eps, sc, st);
    case CPPGB_MODE_FILTER_BF16:
      return prep_lmers_t<__nv_bfloat16>(series, n, l, X, n_pad, Kp, norms, eps, sc, st);
  }
  return set_error(CPPGB_ERR_ARG, "unknown mode %d", mode);
}

}  // namespace cppgb
