// FP64 recheck of the dense stage's surviving candidates.
//
// A candidate survives when its filtered value D~ is <= theta(U_final), i.e. when the lower bound
// on its true squared distance does not exceed the final upper bound U on the best one.  Each
// survivor's squared distance is then recomputed from the caller's original data in FP64 with the
// definition of Sec. 2, sum_k (x_ik - x_jk)^2, summed in coordinate order with explicitly rounded
// operations (no fused multiply-add), and the lexicographic minimum of (d^2, i, j) is taken.
// For l-mers, each window is z-normalised first with its own mean and population standard
// deviation, again with two sequential passes in index order.
#include "common.cuh"

namespace cppgb {
namespace {

__device__ __forceinline__ double sq_rn(double t) { return __dmul_rn(t, t); }

template <class Src>
__device__ double exact_d2_points(const Src* __restrict__ pts, int64_t d, int64_t ld, int64_t i, int64_t j) {
  const Src* x = pts + i * ld;
  const Src* y = pts + j * ld;
  double s = 0.0;
  for (int64_t k = 0; k < d; ++k) s = __dadd_rn(s, sq_rn(__dsub_rn((double)x[k], (double)y[k])));
  return s;
}

// mean and population standard deviation of one window, two sequential passes
__device__ void window_stats(const float* __restrict__ w, int64_t l, double* mu, double* sd) {
  double s = 0.0;
  for (int64_t k = 0; k < l; ++k) s = __dadd_rn(s, (double)w[k]);
  double m = __ddiv_rn(s, (double)l);
  double v = 0.0;
  for (int64_t k = 0; k < l; ++k) v = __dadd_rn(v, sq_rn(__dsub_rn((double)w[k], m)));
  *mu = m;
  *sd = __dsqrt_rn(__ddiv_rn(v, (double)l));
}

__device__ double exact_d2_lmers(const float* __restrict__ a, int64_t l, int64_t i, int64_t j) {
  double mi, si, mj, sj;
  window_stats(a + i, l, &mi, &si);
  window_stats(a + j, l, &mj, &sj);
  const float* wi = a + i;
  const float* wj = a + j;
  double s = 0.0;
  for (int64_t k = 0; k < l; ++k) {
    double zi = __ddiv_rn(__dsub_rn((double)wi[k], mi), si);
    double zj = __ddiv_rn(__dsub_rn((double)wj[k], mj), sj);
    s = __dadd_rn(s, sq_rn(__dsub_rn(zi, zj)));
  }
  return s;
}

__device__ __forceinline__ int64_t live_count(const DenseScalars* sc, int64_t cap) {
  int64_t c = (int64_t)sc->n_cand;
  return c < cap ? c : cap;
}

// Pass A: survivors get their FP64 d^2; the global minimum of the d^2 bit patterns is kept.
template <class Getter>
__device__ void recheck_body(Getter get, DenseScalars* sc, const Candidate* __restrict__ cand,
                             int64_t cap, double* __restrict__ d2buf) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= live_count(sc, cap)) return;
  const float th = theta_of(__uint_as_float(sc->U_bits), sc->bp);
  Candidate cd = cand[c];
  if (!(cd.d2f <= th) || !(cd.d2f < __int_as_float(0x7f800000))) {
    d2buf[c] = -1.0;
    return;
  }
  double s = get(cd.i, cd.j);
  d2buf[c] = s;
  atomicMin(&sc->best_bits, (unsigned long long)__double_as_longlong(s));
  atomicAdd(&sc->n_rech, 1ull);
  atomic_max_nonneg(&sc->ferr_bits, (float)fabs(__dsub_rn(s, (double)cd.d2f)));
}

template <class Src>
__global__ void recheck_points_kernel(const Src* __restrict__ pts, int64_t d, int64_t ld, DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                      double* __restrict__ d2buf) {
  recheck_body([&](int64_t i, int64_t j) { return exact_d2_points(pts, d, ld, i, j); }, sc, cand, cap, d2buf);
}

__global__ void recheck_lmers_kernel(const float* __restrict__ a, int64_t l, DenseScalars* sc,
                                     const Candidate* __restrict__ cand, int64_t cap, double* __restrict__ d2buf) {
  recheck_body([&](int64_t i, int64_t j) { return exact_d2_lmers(a, l, i, j); }, sc, cand, cap, d2buf);
}

// Pass B: among the survivors at the minimal d^2, the lexicographically smallest (i, j).
__global__ void argmin_pair_kernel(DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                   const double* __restrict__ d2buf) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= live_count(sc, cap)) return;
  double s = d2buf[c];
  if (s < 0.0) return;
  if ((unsigned long long)__double_as_longlong(s) == sc->best_bits) {
    Candidate cd = cand[c];
    atomicMin(&sc->best_ij, ((unsigned long long)(uint32_t)cd.i << 32) | (uint32_t)cd.j);
  }
}

__global__ void init_scalars_kernel(DenseScalars* sc) {
  DenseScalars z;
  z.bp.eps_pair = 0.f;
  z.bp.e_acc = 0.f;
  z.U_bits = 0x7f800000u;  // +inf
  z.eps_bits = 0u;
  z.n2_bits = 0u;
  z.status = 0u;
  z.n_cand = 0ull;
  z.n_rech = 0ull;
  z.best_bits = 0x7ff0000000000000ull;  // +inf
  z.best_ij = ~0ull;
  z.ferr_bits = 0u;
  z.pad[0] = 0u;
  *sc = z;
}

__global__ void bounds_kernel(DenseScalars* sc, float kappa) {
  const float eps = __uint_as_float(sc->eps_bits), n2 = __uint_as_float(sc->n2_bits);
  sc->bp.eps_pair = 2.f * eps * (1.f + 0x1p-20f);
  sc->bp.e_acc = kappa * n2 * (1.f + 0x1p-20f);
}

}  // namespace

int launch_init_scalars(DenseScalars* sc, cudaStream_t st) {
  init_scalars_kernel<<<1, 1, 0, st>>>(sc);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_bounds(DenseScalars* sc, float kappa, cudaStream_t st) {
  bounds_kernel<<<1, 1, 0, st>>>(sc, kappa);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

static int finish(DenseScalars* sc, const Candidate* cand, int64_t cap, double* d2buf, int64_t blocks,
                  cudaStream_t st) {
  argmin_pair_kernel<<<(unsigned)blocks, 128, 0, st>>>(sc, cand, cap, d2buf);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_recheck_points(const void* pts, int dtype, int64_t d, int64_t ld, DenseScalars* sc,
                          const Candidate* cand, int64_t cap, double* d2buf, int64_t n_live, cudaStream_t st) {
  const int64_t blocks = (n_live + 127) / 128;
  if (blocks == 0) return CPPGB_OK;
  if (dtype == CPPGB_F64)
    recheck_points_kernel<double><<<(unsigned)blocks, 128, 0, st>>>((const double*)pts, d, ld, sc, cand, cap, d2buf);
  else
    recheck_points_kernel<float><<<(unsigned)blocks, 128, 0, st>>>((const float*)pts, d, ld, sc, cand, cap, d2buf);
  CPPGB_LAUNCH_CHECK();
  return finish(sc, cand, cap, d2buf, blocks, st);
}

int launch_recheck_lmers(const float* series, int64_t l, DenseScalars* sc, const Candidate* cand,
                         int64_t cap, double* d2buf, int64_t n_live, cudaStream_t st) {
  const int64_t blocks = (n_live + 127) / 128;
  if (blocks == 0) return CPPGB_OK;
  recheck_lmers_kernel<<<(unsigned)blocks, 128, 0, st>>>(series, l, sc, cand, cap, d2buf);
  CPPGB_LAUNCH_CHECK();
  return finish(sc, cand, cap, d2buf, blocks, st);
}

}  // namespace cppgb
