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

__device__ __forceinline__ int64_t live_count(const DenseScalars* sc, int64_t cap) {
  int64_t c = (int64_t)sc->n_cand;
  return c < cap ? c : cap;
}

// Pass A: survivors get their FP64 d^2; the global minimum of the d^2 bit patterns is kept.
template <class Getter>
__device__ void recheck_body(Getter get, DenseScalars* sc, const Candidate* __restrict__ cand,
                             int64_t cap, double* __restrict__ d2buf) {
  const int64_t live = live_count(sc, cap);
  const float th = theta_of(__uint_as_float(sc->U_bits), sc->bp);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < live; c += (int64_t)gridDim.x * blockDim.x) {
    const Candidate cd = cand[c];
    if (!(cd.d2f <= th) || !(cd.d2f < __int_as_float(0x7f800000))) {
      d2buf[c] = -1.0;
      continue;
    }
    const double s = get(cd.i, cd.j);
    d2buf[c] = s;
    atomicMin(&sc->best_bits, (unsigned long long)__double_as_longlong(s));
    atomicAdd(&sc->n_rech, 1ull);
    atomic_max_nonneg(&sc->ferr_bits, (float)fabs(__dsub_rn(s, (double)cd.d2f)));
  }
}

template <class Src>
__global__ void recheck_points_kernel(const Src* __restrict__ pts, int64_t d, int64_t ld, DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                      double* __restrict__ d2buf) {
  recheck_body([&](int64_t i, int64_t j) { return exact_d2_points(pts, d, ld, i, j); }, sc, cand, cap, d2buf);
}

// l-mers, in two kernels.  The screen lists the candidates whose D~ can still reach the final bound
// (most emitted candidates were written before the bound settled: the survivors are a few per
// thousand, and they cluster, since one tile emits many).  Then one warp takes each survivor.
// Each window w is z-normalised with its mean m = (sum_k w_k) / l and population standard deviation
// sd = sqrt((sum_k (w_k - m)^2) / l), z_k = (w_k - m) / sd, and d^2 = sum_k (z_ik - z_jk)^2, every
// operation rounded (no contraction) and every sum in index order.  The sums keep that order -- one
// lane adds each -- while their terms (the converted values, the deviations, the divisions of the
// z-values) are computed by all lanes at once into shared memory, RCH at a time.
constexpr int RW = 4, RCH = 512, RGRID = 152 * 16;

__global__ void screen_lmers_kernel(DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                    double* __restrict__ d2buf, int32_t* __restrict__ surv) {
  const int64_t live = live_count(sc, cap);
  const float th = theta_of(__uint_as_float(sc->U_bits), sc->bp);
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < live; c += (int64_t)gridDim.x * blockDim.x) {
    const float d2f = cand[c].d2f;
    if (d2f <= th && d2f < __int_as_float(0x7f800000)) surv[atomicAdd(&sc->n_surv, 1u)] = (int32_t)c;
    else d2buf[c] = -1.0;
  }
}

// sum_k t_k in index order, the terms written by `term` (all lanes) into buf[q], RCH at a time;
// lane q (q < nsums) keeps sum q
template <class Term>
__device__ __forceinline__ double ordered_sum(int64_t l, int lane, int nsums, double (&buf)[2][RCH], Term term) {
  double v = 0.0;
  for (int64_t k0 = 0; k0 < l; k0 += RCH) {
    const int cnt = (int)(l - k0 < RCH ? l - k0 : RCH);
#pragma unroll 4
    for (int k = lane; k < cnt; k += 32) term(k0 + k, k);
    __syncwarp();
    if (lane < nsums)
      for (int k = 0; k < cnt; ++k) v = __dadd_rn(v, buf[lane][k]);
    __syncwarp();
  }
  return v;
}

__global__ void __launch_bounds__(32 * RW) recheck_lmers_kernel(const float* __restrict__ a, int64_t l,
                                                                DenseScalars* sc, const Candidate* __restrict__ cand,
                                                                const int32_t* __restrict__ surv,
                                                                double* __restrict__ d2buf) {
  __shared__ double sbuf[RW][2][RCH];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double (&buf)[2][RCH] = sbuf[w];
  const int64_t ns = (int64_t)sc->n_surv;
  const double dl = (double)l;
  for (int64_t k = (int64_t)blockIdx.x * RW + w; k < ns; k += (int64_t)gridDim.x * RW) {
    const int32_t c = surv[k];
    const Candidate cd = cand[c];
    const float* wi = a + cd.i;
    const float* wj = a + cd.j;
    // means (lane 0: window i, lane 1: window j)
    const double sm = ordered_sum(l, lane, 2, buf, [&](int64_t g, int k2) {
      buf[0][k2] = (double)wi[g];
      buf[1][k2] = (double)wj[g];
    });
    const double m = lane < 2 ? __ddiv_rn(sm, dl) : 0.0;
    const double mi = __shfl_sync(0xffffffffu, m, 0), mj = __shfl_sync(0xffffffffu, m, 1);
    // population variances
    const double sv = ordered_sum(l, lane, 2, buf, [&](int64_t g, int k2) {
      buf[0][k2] = sq_rn(__dsub_rn((double)wi[g], mi));
      buf[1][k2] = sq_rn(__dsub_rn((double)wj[g], mj));
    });
    const double sd = lane < 2 ? __dsqrt_rn(__ddiv_rn(sv, dl)) : 1.0;
    const double si = __shfl_sync(0xffffffffu, sd, 0), sj = __shfl_sync(0xffffffffu, sd, 1);
    // the distance (lane 0)
    const double s = ordered_sum(l, lane, 1, buf, [&](int64_t g, int k2) {
      const double zi = __ddiv_rn(__dsub_rn((double)wi[g], mi), si);
      const double zj = __ddiv_rn(__dsub_rn((double)wj[g], mj), sj);
      buf[0][k2] = sq_rn(__dsub_rn(zi, zj));
    });
    if (lane == 0) {
      d2buf[c] = s;
      atomicMin(&sc->best_bits, (unsigned long long)__double_as_longlong(s));
      atomicAdd(&sc->n_rech, 1ull);
      atomic_max_nonneg(&sc->ferr_bits, (float)fabs(__dsub_rn(s, (double)cd.d2f)));
    }
  }
}

// Pass B: among the survivors at the minimal d^2, the lexicographically smallest (i, j).
__global__ void argmin_pair_kernel(DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                   const double* __restrict__ d2buf) {
  const int64_t live = live_count(sc, cap);
  const unsigned long long best = sc->best_bits;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < live; c += (int64_t)gridDim.x * blockDim.x) {
    const double s = d2buf[c];
    if (s < 0.0) continue;
    if ((unsigned long long)__double_as_longlong(s) == best) {
      const Candidate cd = cand[c];
      atomicMin(&sc->best_ij, ((unsigned long long)(uint32_t)cd.i << 32) | (uint32_t)cd.j);
    }
  }
}

__global__ void pass2_gate_kernel(DenseScalars* sc, int64_t cap) {
  const bool redo = sc->status == 0u && (int64_t)sc->n_cand > cap;
  sc->redo = redo ? 1u : 0u;
  if (redo) sc->n_cand = 0ull;  // the bound U is final now; the second pass emits against it
}

__global__ void dense_result_kernel(const DenseScalars* sc, int64_t cap, const int64_t* tcount, int64_t tiles_total,
                                    cpp_pair_result* res) {
  cpp_pair_result r;
  const unsigned int st = sc->status;
  r.status = (st & 3u) ? CPPGB_ERR_NUMERIC : (st & 4u) ? CPPGB_ERR_TIMEOUT
             : (int64_t)sc->n_cand > cap ? CPPGB_ERR_CAPACITY : CPPGB_OK;
  const double best = __longlong_as_double((long long)sc->best_bits);
  if (r.status != CPPGB_OK || sc->best_ij == ~0ull || !(best < __longlong_as_double(0x7ff0000000000000ll))) {
    r.i = r.j = -1;
    r.dist = r.dist2 = __longlong_as_double(0x7ff0000000000000ll);
  } else {
    r.i = (int64_t)(sc->best_ij >> 32);
    r.j = (int64_t)(sc->best_ij & 0xffffffffu);
    r.dist2 = best;
    r.dist = __dsqrt_rn(best);
  }
  r.filter_err = (double)__uint_as_float(sc->ferr_bits);
  r.filter_bound = (double)__uint_as_float(sc->U_bits);
  r.n_emitted = (int64_t)sc->n_cand;
  r.n_rechecked = (int64_t)sc->n_rech;
  r.filter_e_acc = (double)sc->bp.e_acc;
  r.filter_eps = (double)sc->bp.eps_pair;
  r.tiles_kept = tcount ? *tcount : -1;
  r.tiles_total = tcount ? tiles_total : -1;
  r.reserved = 0;
  *res = r;
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
  z.n_surv = 0u;
  z.redo = 0u;
  z.pad = 0u;
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

constexpr unsigned RB = 128, RBLOCKS = 152 * 8;  // grid-stride candidate kernels

static unsigned cand_blocks(int64_t cap) {
  const int64_t b = (cap + RB - 1) / RB;
  return (unsigned)(b < RBLOCKS ? (b > 0 ? b : 1) : RBLOCKS);
}

int launch_recheck_points(const void* pts, int dtype, int64_t d, int64_t ld, DenseScalars* sc,
                          const Candidate* cand, int64_t cap, double* d2buf, cudaStream_t st) {
  const unsigned blocks = cand_blocks(cap);
  if (dtype == CPPGB_F64)
    recheck_points_kernel<double><<<blocks, RB, 0, st>>>((const double*)pts, d, ld, sc, cand, cap, d2buf);
  else
    recheck_points_kernel<float><<<blocks, RB, 0, st>>>((const float*)pts, d, ld, sc, cand, cap, d2buf);
  CPPGB_LAUNCH_CHECK();
  argmin_pair_kernel<<<blocks, RB, 0, st>>>(sc, cand, cap, d2buf);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_recheck_lmers(const float* series, int64_t l, DenseScalars* sc, int32_t* surv, const Candidate* cand,
                         int64_t cap, double* d2buf, cudaStream_t st) {
  const unsigned blocks = cand_blocks(cap);
  screen_lmers_kernel<<<blocks, RB, 0, st>>>(sc, cand, cap, d2buf, surv);
  CPPGB_LAUNCH_CHECK();
  recheck_lmers_kernel<<<RGRID, 32 * RW, 0, st>>>(series, l, sc, cand, surv, d2buf);
  CPPGB_LAUNCH_CHECK();
  argmin_pair_kernel<<<blocks, RB, 0, st>>>(sc, cand, cap, d2buf);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_pass2_gate(DenseScalars* sc, int64_t cap, cudaStream_t st) {
  pass2_gate_kernel<<<1, 1, 0, st>>>(sc, cap);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_dense_result(const DenseScalars* sc, int64_t cap, const int64_t* tcount, int64_t tiles_total,
                        cpp_pair_result* res, cudaStream_t st) {
  dense_result_kernel<<<1, 1, 0, st>>>(sc, cap, tcount, tiles_total, res);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

}  // namespace cppgb
