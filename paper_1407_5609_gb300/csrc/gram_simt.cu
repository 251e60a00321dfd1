// Dense all-pairs stage on FP32 CUDA cores (the plain comparison path).
//
// Every pair (i, j), i < j, j - i >= excl, of the n rows of X is evaluated in the Gram form
//   D~_ij = |x~_i|^2 + |x~_j|^2 - 2 x~_i . x~_j
// over 128 x 128 tiles of the upper triangle (FFMA, 8 x 8 accumulators per thread).  The tile
// epilogue is fused: the tile minimum tightens a global upper bound U on the best true d^2, and
// every pair whose lower bound could still be <= U is emitted as a candidate for the FP64
// recheck.  The brute force over all pairs is the O(n^2 l) algorithm stated in Sec. 3.
#include "common.cuh"
#include "tile_simt.cuh"

namespace cppgb {
namespace {

constexpr int BM = 128, BK = 16, NT = 256;

// RADIUS = false: closest-pair epilogue (tile minimum, bound update, emission against the bound).
// RADIUS = true:  fixed-radius epilogue (Sec. 3.5): emit every pair whose lower bound on d is <= R,
//                 i.e. D~ <= theta(R^2); no bound update.
// (the accumulation bound used with these tiles is derived on the host: sequential FFMA over Kp)
template <bool RADIUS>
__global__ void __launch_bounds__(NT, 2)
    gram_simt_kernel(const float* __restrict__ X, int64_t n, int64_t Kp, int64_t excl, int64_t delta,
                     const float* __restrict__ norms, DenseScalars* sc,
                     Candidate* __restrict__ cand, int64_t cap, float rr, int64_t shard, int64_t nshards,
                     const unsigned int* __restrict__ gate) {
  __shared__ __align__(16) TileSmem sm;
  __shared__ float red[NT / 32];
  if (gate && *gate == 0u) return;  // a second pass that is not needed

  int64_t bi, bj;
  tri_decode((int64_t)blockIdx.x * nshards + shard, delta, &bi, &bj);
  const int64_t row0 = bi * BM, col0 = bj * BM;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  float acc[8][8];
  simt_tile_mainloop(X, Kp, row0, col0, sm, acc);

  // ---- fused epilogue: D~, tile minimum, bound update, candidate emission
  int64_t gi[8], gj[8];
  float nx[8], ny[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    gi[r] = row0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
    gj[r] = col0 + (r < 4 ? tx * 4 + r : 64 + tx * 4 + r - 4);
    nx[r] = norms[gi[r]];
    ny[r] = norms[gj[r]];
  }
  float tmin = __int_as_float(0x7f800000);
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      bool ok = gi[r] < n && gj[c] < n && gj[c] - gi[r] >= excl;
      float D = fmaf(-2.f, acc[r][c], nx[r] + ny[c]);
      D = ok ? D : __int_as_float(0x7f800000);
      acc[r][c] = D;
      tmin = fminf(tmin, D);
    }
  float th, ub = 0.f;
  const BoundParams bp = sc->bp;
  if (RADIUS) {
    th = theta_of(rr, bp);
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    if ((tid & 31) == 0) red[tid >> 5] = tmin;
    __syncthreads();
    tmin = red[0];
#pragma unroll
    for (int w = 1; w < NT / 32; ++w) tmin = fminf(tmin, red[w]);
    if (tmin == __int_as_float(0x7f800000)) return;  // no valid pair in this tile

    ub = upper_d2(tmin, bp);
    const float Ug = __uint_as_float(*reinterpret_cast<volatile unsigned int*>(&sc->U_bits));
    th = theta_of(fminf(Ug, ub), bp);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (acc[r][c] <= th) {
        unsigned long long k = atomicAdd(&sc->n_cand, 1ull);
        if ((int64_t)k < cap) {
          Candidate cd;
          cd.i = (int32_t)gi[r];
          cd.j = (int32_t)gj[c];
          cd.d2f = acc[r][c];
          cd.pad = 0.f;
          cand[k] = cd;
        }
      }
    }
  if (!RADIUS && tid == 0) atomic_min_nonneg(&sc->U_bits, ub);
}

}  // namespace

template <bool RADIUS>
static int launch_simt(const float* X, int64_t n, int64_t Kp, int64_t excl, const float* norms, DenseScalars* sc,
                       Candidate* cand, int64_t cap, float rr, cudaStream_t st, int64_t shard, int64_t nshards,
                       const unsigned int* gate) {
  if (Kp % BK) return set_error(CPPGB_ERR_ARG, "internal: Kp %% 16 != 0");
  const int64_t nb = (n + BM - 1) / BM;
  // smallest block offset whose tiles hold a pair with j - i >= excl
  int64_t delta = excl <= BM - 1 ? 0 : (excl - (BM - 1) + BM - 1) / BM;
  const int64_t m = nb - delta;
  const int64_t all = tri_count(m);
  const int64_t tiles = all > shard ? (all - shard + nshards - 1) / nshards : 0;  // this shard's tiles
  if (tiles <= 0) return CPPGB_OK;
  if (tiles > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "too many tiles (%lld)", (long long)tiles);
  gram_simt_kernel<RADIUS><<<(unsigned)tiles, NT, 0, st>>>(X, n, Kp, excl, delta, norms, sc, cand, cap, rr,
                                                                   shard, nshards, gate);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_gram_simt(const float* X, int64_t n, int64_t Kp, int64_t excl, const float* norms, DenseScalars* sc,
                     Candidate* cand, int64_t cap, cudaStream_t st, int64_t shard, int64_t nshards,
                     const unsigned int* gate) {
  return launch_simt<false>(X, n, Kp, excl, norms, sc, cand, cap, 0.f, st, shard, nshards, gate);
}

int launch_gram_simt_radius(const float* X, int64_t n, int64_t Kp, const float* norms, DenseScalars* sc,
                            Candidate* cand, int64_t cap, float rr, cudaStream_t st) {
  return launch_simt<true>(X, n, Kp, 1, norms, sc, cand, cap, rr, st, 0, 1, nullptr);
}

}  // namespace cppgb
