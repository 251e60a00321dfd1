// Dense all-pairs stage on the 5th-generation tensor cores (tcgen05), FP16 or BF16 operands.
//
// Same contract as the FP32 stage (gram_simt.cu): every pair (i, j), i < j, j - i >= excl, of the
// rows of X gets D~_ij = |x~_i|^2 + |x~_j|^2 - 2 x~_i . x~_j, the tile minima tighten the global
// upper bound U, and pairs whose lower bound can still reach U are emitted for the FP64 recheck.
// This is the brute-force O(n^2 l) evaluation of Sec. 3 with the Gram products on tensor cores.
//
// Kernel organisation (one persistent CTA per SM, 6 warps):
//   warp 0      TMA producer: 128x64 (A) and 256x64 (B) 16-bit tiles, 128-byte swizzle, into a
//               4-stage shared-memory ring guarded by full/empty mbarriers
//   warp 1      allocates 512 TMEM columns; one lane issues tcgen05.mma (M=128, N=256, K=16) into
//               one of two 256-column FP32 accumulators, commits to the ring and to the epilogue
//   warps 2-5   epilogue: tcgen05.ld of the accumulator rows, D~ = nx + (ny - 2 S), running minima,
//               threshold test per 32-column chunk, rare candidate emission, bound publication
// Tiles are 128 rows x 256 columns of the upper triangle, walked in bands of 16 column blocks (the
// band's B panels stay in L2 while the row panels stream once per band).  Every mbarrier wait is
// bounded (about 2 s of %globaltimer): on a timeout the CTA flags CPPGB_ERR_TIMEOUT, drains what it
// issued, frees its TMEM and exits.
#include <cuda.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace cppgb {
namespace {
using namespace tc;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NTHREADS = 192;
constexpr int BAND = 16;  // column blocks per band (4 MB of B panels stay in L2); 8, 32, 64 measured slower
constexpr int MAX_BANDS = 480;
constexpr uint32_t TMEM_COLS = 512;

// Tile schedule: bands of column blocks; inside a band, row-block-major.  off[b] = tiles before
// band b; nfull[b] = leading row blocks whose every column block in the band holds a valid pair.
struct TileSched {
  int64_t n, excl;
  int32_t nbands, nbi, nbj, band;
  int32_t rstep, pad;  // 128-row blocks per schedule row: 1 (one CTA) or 2 (a CTA pair)
  int64_t off[MAX_BANDS + 1];
  int32_t nfull[MAX_BANDS];
};

// first column block bj whose tile (bi, bj) holds a pair with j - i >= excl (j < n); -1 if none
__host__ __device__ __forceinline__ int64_t first_bj(int64_t bi, int64_t n, int64_t excl) {
  const int64_t need = excl + (int64_t)BM * bi;  // smallest admissible j for the tile's first row
  if (n - 1 < need) return -1;
  const int64_t v = need - (BN - 1);
  return v <= 0 ? 0 : (v + BN - 1) / BN;
}
__host__ __device__ __forceinline__ int64_t row_count(int64_t bi, int64_t bj0, int64_t bj1, int64_t n,
                                                      int64_t excl) {
  const int64_t f = first_bj(bi, n, excl);
  if (f < 0) return 0;
  const int64_t lo = f > bj0 ? f : bj0;
  return bj1 > lo ? bj1 - lo : 0;
}

// `band` is the caller's cursor: each role walks its tiles in increasing t, so it only moves forward.
__device__ __forceinline__ void decode_tile(const TileSched& ts, int64_t t, int* band, int64_t* bi, int64_t* bj) {
  int b = *band;
  while (b + 1 < ts.nbands && ts.off[b + 1] <= t) ++b;
  *band = b;
  const int64_t bj0 = (int64_t)b * ts.band;
  const int64_t bj1 = bj0 + ts.band < ts.nbj ? bj0 + ts.band : ts.nbj;
  const int64_t w = bj1 - bj0;
  int64_t r = t - ts.off[b];
  const int64_t full = (int64_t)ts.nfull[b] * w;
  if (r < full) {
    *bi = r / w;
    *bj = bj0 + r % w;
    return;
  }
  r -= full;
  for (int64_t row = ts.nfull[b]; row < ts.nbi; ++row) {
    const int64_t c = row_count(row * ts.rstep, bj0, bj1, ts.n, ts.excl);
    if (r < c) {
      *bi = row;
      *bj = bj1 - c + r;
      return;
    }
    r -= c;
  }
  *bi = 0;
  *bj = 0;  // unreachable for t < total
}

// ------------------------------------------------------------------ shared epilogue
// Per-thread epilogue state: running minimum of D~, snapshot of the global bound, emission threshold.
struct EpiState {
  float tmin, Usnap, th;
};

__device__ __forceinline__ void epi_init(EpiState& es, DenseScalars* sc, const BoundParams& bp) {
  es.tmin = __int_as_float(0x7f800000);
  es.Usnap = __uint_as_float(*reinterpret_cast<volatile unsigned int*>(&sc->U_bits));
  // -inf until this thread has a finite bound, so masked (+inf) entries can never pass it
  es.th = es.Usnap < __int_as_float(0x7f800000) ? theta_of(es.Usnap, bp) : __int_as_float(0xff800000);
}

// One 32-column chunk c of a thread's accumulator row (r = the raw Gram values x~_i . x~_j).
template <bool PERM>
__device__ __forceinline__ void epi_chunk(const uint32_t (&r)[32], int c, int64_t i, float nx, int32_t oi,
                                          bool edge, bool pmask, int32_t xoff, uint32_t xspan, int64_t col0,
                                          int64_t n, int64_t excl, const float* __restrict__ norms,
                                          const BoundParams& bp, DenseScalars* sc, Candidate* __restrict__ cand,
                                          int64_t cap, EpiState& es, const int32_t* __restrict__ perm) {
  const float4* ny4 = reinterpret_cast<const float4*>(norms + col0 + c * 32);
  float dp[32];
  float cmin = __int_as_float(0x7f800000);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float4 v = __ldg(ny4 + q);
    dp[4 * q + 0] = fmaf(-2.f, __uint_as_float(r[4 * q + 0]), v.x);
    dp[4 * q + 1] = fmaf(-2.f, __uint_as_float(r[4 * q + 1]), v.y);
    dp[4 * q + 2] = fmaf(-2.f, __uint_as_float(r[4 * q + 2]), v.z);
    dp[4 * q + 3] = fmaf(-2.f, __uint_as_float(r[4 * q + 3]), v.w);
  }
  if (edge) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int64_t j = col0 + c * 32 + k;
      if (!(i < n && j < n && j - i >= excl)) dp[k] = __int_as_float(0x7f800000);
    }
  }
  if (PERM && pmask) {  // original indices of the chunk's columns (the same for every lane: broadcast loads)
    const int4* pj4 = reinterpret_cast<const int4*>(perm + col0 + c * 32);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int4 o = __ldg(pj4 + q);
      const int32_t oj[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if ((uint32_t)(oi - oj[e] + xoff) < xspan) dp[4 * q + e] = __int_as_float(0x7f800000);
    }
  }
#pragma unroll
  for (int k = 0; k < 32; ++k) cmin = fminf(cmin, dp[k]);
  const float cD = nx + cmin;
  if (cD < es.tmin) {
    es.tmin = cD;
    es.th = theta_of(fminf(es.Usnap, upper_d2(es.tmin, bp)), bp);
  }
  if (cD <= es.th) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const float D = nx + dp[k];
      if (D <= es.th) {
        const unsigned long long slot = atomicAdd(&sc->n_cand, 1ull);
        if ((int64_t)slot < cap) {
          Candidate cd;
          int32_t a = (int32_t)i, b = (int32_t)(col0 + c * 32 + k);
          if (PERM) {
            a = oi;
            b = perm[col0 + c * 32 + k];
          }
          cd.i = a < b ? a : b;
          cd.j = a < b ? b : a;
          cd.d2f = D;
          cd.pad = 0.f;
          cand[slot] = cd;
        }
      }
    }
  }
}

// One thread = one accumulator row (TMEM lane) of a 128 x 256 tile: D~ = nx + (ny - 2 S) for its 256
// columns in 32-column chunks, running minimum, threshold test per chunk, rare candidate emission.
// With `perm` the rows are a permutation of the original ones (row p is original row perm[p]): the
// schedule covers the pairs p < q of positions, a pair is excluded when its original indices are
// closer than excl_orig, and candidates carry original indices (smaller first).
template <bool PERM>
__device__ __forceinline__ void epi_tile(int64_t row0, int64_t col0, uint32_t tbase, int lane, uint32_t quarter,
                                         int64_t n, int64_t excl, const float* __restrict__ norms,
                                         const BoundParams& bp, DenseScalars* sc, Candidate* __restrict__ cand,
                                         int64_t cap, EpiState& es, const int32_t* __restrict__ perm,
                                         int64_t excl_orig) {
  const int64_t i = row0 + quarter * 32 + lane;
  const float nx = norms[i];
  const bool pmask = PERM && excl_orig > 1;
  const int32_t oi = PERM && i < n ? perm[i] : (int32_t)i;
  // |oi - oj| < excl_orig  <=>  (unsigned)(oi - oj + excl_orig - 1) < 2 excl_orig - 1
  const int32_t xoff = (int32_t)excl_orig - 1;
  const uint32_t xspan = 2u * (uint32_t)excl_orig - 1u;
  const bool edge = (row0 + BM - 1 >= n) || (col0 + BN - 1 >= n) || (col0 - (row0 + BM - 1) < excl);
#pragma unroll 1
  for (int c = 0; c < BN / 32; ++c) {
    uint32_t r[32];
    __syncwarp();
    tmem_ld32(tbase + (uint32_t)(c * 32), r);
    epi_chunk<PERM>(r, c, i, nx, oi, edge, pmask, xoff, xspan, col0, n, excl, norms, bp, sc, cand, cap, es, perm);
  }
}

// Publish the warp's bound if it improves the global one, then refresh the snapshot.
__device__ __forceinline__ void epi_publish(int lane, const BoundParams& bp, DenseScalars* sc, EpiState& es) {
  float wmin = es.tmin;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wmin = fminf(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
  float Unew = 0.f;
  if (lane == 0) {
    const float ub = upper_d2(wmin, bp);
    if (ub < es.Usnap) atomic_min_nonneg(&sc->U_bits, ub);
    Unew = __uint_as_float(*reinterpret_cast<volatile unsigned int*>(&sc->U_bits));
  }
  Unew = __shfl_sync(0xffffffffu, Unew, 0);
  if (Unew < es.Usnap) {
    es.Usnap = Unew;
    es.th = theta_of(fminf(es.Usnap, upper_d2(es.tmin, bp)), bp);
  }
}

// ------------------------------------------------------------------ reference pruning of tiles
// A tile (row block bi, column block bj = row blocks 2bj, 2bj + 1) is kept unless, for some
// reference, the gap between the row block's and the column block's distance intervals exceeds
// sqrt(U): then no pair of the tile is within sqrt(U) of the other (triangle inequality).
__global__ void prune_flags_kernel(const __grid_constant__ TileSched ts, int64_t total, int64_t shard,
                                   int64_t nshards, const float* __restrict__ blo, const float* __restrict__ bhi,
                                   int64_t nbi, const DenseScalars* sc, int32_t* __restrict__ flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  int band = 0;
  int64_t lo_b = 0, hi_b = ts.nbands;  // band of tile id g: largest b with off[b] <= g
  const int64_t g = t * nshards + shard;
  while (lo_b + 1 < hi_b) {
    const int64_t mid = (lo_b + hi_b) >> 1;
    if (ts.off[mid] <= g) lo_b = mid;
    else hi_b = mid;
  }
  band = (int)lo_b;
  int64_t bi, bj;
  decode_tile(ts, g, &band, &bi, &bj);
  const float U = __uint_as_float(sc->U_bits);
  const float th = sqrtf(U) * (1.f + 0x1p-20f) + 1e-30f;
  const int64_t c0 = 2 * bj, c1 = 2 * bj + 1 < nbi ? 2 * bj + 1 : 2 * bj;
  float lb = 0.f;
#pragma unroll
  for (int q = 0; q < PRUNE_REFS; ++q) {
    const float ilo = blo[q * nbi + bi], ihi = bhi[q * nbi + bi];
    const float jlo = fminf(blo[q * nbi + c0], blo[q * nbi + c1]), jhi = fmaxf(bhi[q * nbi + c0], bhi[q * nbi + c1]);
    lb = fmaxf(lb, fmaxf(__fsub_rd(jlo, ihi), __fsub_rd(ilo, jhi)));
  }
  flags[t] = (U < __int_as_float(0x7f800000) && lb > th) ? 0 : 1;
}

__global__ void prune_compact_kernel(int64_t total, int64_t shard, int64_t nshards, const int32_t* __restrict__ flags,
                                     const int64_t* __restrict__ pos, int32_t* __restrict__ list) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < total && flags[t]) list[pos[t]] = (int32_t)(t * nshards + shard);
}

// Fault injection for the tests of the bounded waits (cpp_set_fault_injection): when non-zero the TMA
// producer issues no copy, so the MMA issuer's and the epilogue's waits run out and the search
// reports CPPGB_ERR_TIMEOUT.  Nothing is in flight when the CTA exits.  Zero unless a test sets it.
__device__ int g_fault_skip_tma = 0;

struct SmemCtl {
  uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], drain;
  uint32_t tmem_base;
  int abort_flag;
};

// Tile t of this launch: the (bi, bj) pairs of a dump list (DUMP), else tile id t * nshards + shard
// of the band schedule or the entry t of a pruned list.
template <bool DUMP>
__device__ __forceinline__ void tile_of(const TileSched& ts, int64_t t, const int32_t* __restrict__ tlist,
                                        int64_t shard, int64_t nshards, int* band, int64_t* bi, int64_t* bj) {
  if (DUMP) {
    *bi = tlist[2 * t];
    *bj = tlist[2 * t + 1];
    return;
  }
  decode_tile(ts, tlist ? (int64_t)tlist[t] : t * nshards + shard, band, bi, bj);
}

// DUMP (diagnostics, cpp_gram_tile_dump): the tiles are the (bi, bj) pairs of tlist and the
// epilogue writes each tile's raw accumulator S~ = x~_i . x~_j (128 x 256 FP32, row-major) to
// dump[t]; the TMA producer and the MMA issuer are those of the search.
template <bool PERM, bool DUMP>
__global__ void __launch_bounds__(NTHREADS, 1)
    gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TileSched ts, int64_t total_arg,
                   uint32_t ab_fmt, const float* __restrict__ norms, DenseScalars* sc, Candidate* __restrict__ cand,
                   int64_t cap, int64_t kchunks, int64_t shard, int64_t nshards, const int32_t* __restrict__ tlist,
                   const int64_t* __restrict__ tcount, const int32_t* __restrict__ perm, int64_t excl_orig,
                   float* __restrict__ dump, const unsigned int* __restrict__ gate) {
  if (gate && *gate == 0u) return;  // a second pass that is not needed (before any set-up)
  // the tiles: k < total of this shard (t = k * nshards + shard), or the entries of a pruned list
  const int64_t total = tcount ? *tcount : total_arg;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  SmemCtl* ctl = (SmemCtl*)(smem + STAGES * STAGE_BYTES);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&ctl->tfull[a], 1);
      mbar_init(&ctl->tempty[a], 4);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = ctl->tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap) : "memory");
      uint32_t stage = 0, phase = 0;
      int64_t issued = 0;
      int band = 0;
      bool ok = true;
      const bool skip = *reinterpret_cast<volatile int*>(&g_fault_skip_tma) != 0;
      for (int64_t t = blockIdx.x; t < total && ok && !skip; t += gridDim.x) {
        int64_t bi, bj;
        tile_of<DUMP>(ts, t, tlist, shard, nshards, &band, &bi, &bj);
        for (int64_t kc = 0; kc < kchunks; ++kc) {
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1u, abort_flag)) { ok = false; break; }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          mbar_arrive_expect_tx(&ctl->full[stage], STAGE_BYTES);
          tma_load_2d(sa, &tmap, &ctl->full[stage], (int)(kc * BK), (int)(bi * BM));
          tma_load_2d(sa + A_BYTES, &tmap, &ctl->full[stage], (int)(kc * BK), (int)(bj * BN));
          tma_load_2d(sa + A_BYTES + BM * BK * 2, &tmap, &ctl->full[stage], (int)(kc * BK), (int)(bj * BN + BM));
          ++issued;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&sc->status, 4u);
      }
      // drain: every issued copy must have landed before the CTA may exit
      const int64_t last = issued < STAGES ? issued : STAGES;
      for (int64_t q = 1; q <= last; ++q) {
        const int64_t u = issued - q;                // use index of that copy
        const uint32_t s = (uint32_t)(u % STAGES), par = (uint32_t)((u / STAGES) & 1);
        uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&ctl->full[s], par) && globaltimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = make_idesc(ab_fmt, BM, BN);
      uint32_t stage = 0, phase = 0;
      int64_t it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
        const uint32_t acc = (uint32_t)(it & 1), use = (uint32_t)((it >> 1) & 1);
        if (!mbar_wait(&ctl->tempty[acc], use ^ 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dtmem = tmem_base + acc * (uint32_t)BN;
        for (int64_t kc = 0; kc < kchunks; ++kc) {
          if (!mbar_wait(&ctl->full[stage], phase, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
          const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)  // advance 16 elements = 32 bytes inside the swizzle atom
            mma_f16(dtmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc | kk) != 0);
          mma_commit(&ctl->empty[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        mma_commit(&ctl->tfull[acc]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&sc->status, 4u);
      }
      // drain: the commit arrives once every MMA issued so far has completed; TMEM is freed after
      mma_commit(&ctl->drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..5)
    const uint32_t quarter = (uint32_t)(warp & 3);  // TMEM lanes 32*quarter .. +31
    const BoundParams bp = sc->bp;
    EpiState es;
    epi_init(es, sc, bp);
    int64_t it = 0;
    int band = 0;
    for (int64_t t = blockIdx.x; t < total; t += gridDim.x, ++it) {
      int64_t bi, bj;
      tile_of<DUMP>(ts, t, tlist, shard, nshards, &band, &bi, &bj);
      const uint32_t acc = (uint32_t)(it & 1), use = (uint32_t)((it >> 1) & 1);
      const bool got = __all_sync(0xffffffffu, mbar_wait(&ctl->tfull[acc], use, abort_flag));
      if (!got) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(&sc->status, 4u);
        }
        break;
      }
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((quarter * 32u) << 16) + acc * (uint32_t)BN;
      if (DUMP) {
        float4* row = reinterpret_cast<float4*>(dump + ((size_t)t * BM + quarter * 32 + lane) * BN);
#pragma unroll 1
        for (int c = 0; c < BN / 32; ++c) {
          uint32_t r[32];
          __syncwarp();
          tmem_ld32(tbase + (uint32_t)(c * 32), r);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            row[c * 8 + q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                                         __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
        }
      } else {
        epi_tile<PERM>(bi * BM, bj * BN, tbase, lane, quarter, ts.n, ts.excl, norms, bp, sc, cand, cap, es, perm,
                       excl_orig);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->tempty[acc]);
      if (!DUMP) epi_publish(lane, bp, sc, es);
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
    }
    tc_fence_before();
  }

  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ CTA pairs (cta_group::2)
// A cluster of two CTAs on two SMs computes one 256 x 256 tile: CTA r holds the 128 rows of row
// block 2 bi2 + r (A) and rows 128 r .. 128 r + 127 of the column block (its half of B), both in
// 6 stages of 32 KB; the leader (r = 0) issues tcgen05.mma.cta_group::2 with M = 256, N = 256,
// which reads both CTAs' halves, and each CTA's TMEM receives the 128 x 256 accumulator of its own
// rows.  Per pair of SMs a 64-deep K step moves 64 KB from L2 for 256 x 256 x 64 MACs, against
// 96 KB for two single-CTA 128 x 256 tiles: a third less traffic through the L2 -> SM crossbar.
// Barriers: each CTA's copies complete on the leader's full[s] (armed by the leader for both CTAs'
// bytes); the leader's commits arrive on both CTAs' empty[s], tfull[a] and drain; the epilogue
// warps of both CTAs arrive on the leader's tempty[a] (count 8).  Every wait is bounded as in the
// single-CTA kernel, and both CTAs meet in a cluster barrier before freeing TMEM and exiting.
constexpr int P_STAGES = 6;
constexpr int PA_BYTES = BM * BK * 2, PB_BYTES = (BN / 2) * BK * 2, P_STAGE_BYTES = PA_BYTES + PB_BYTES;

struct PairCtl {
  uint64_t full[P_STAGES], empty[P_STAGES], tfull[2], tempty[2], drain;
  uint32_t tmem_base;
  int abort_flag;
};

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(NTHREADS, 1)
    gram_tc_pair_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TileSched ts,
                        int64_t total, uint32_t ab_fmt, const float* __restrict__ norms, DenseScalars* sc,
                        Candidate* __restrict__ cand, int64_t cap, int64_t kchunks, int64_t shard, int64_t nshards,
                        const unsigned int* __restrict__ gate) {
  if (gate && *gate == 0u) return;  // a second pass that is not needed (both CTAs of every cluster)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  PairCtl* ctl = (PairCtl*)(smem + P_STAGES * P_STAGE_BYTES);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int64_t cl = blockIdx.x >> 1, ncl = gridDim.x >> 1;  // this cluster and the number of clusters

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&ctl->tfull[a], 1);
      mbar_init(&ctl->tempty[a], 8);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // one warp of each CTA of the pair allocates the pair's TMEM together
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();  // both CTAs' barriers are initialised before any cross-CTA arrive
  tc_fence_after();
  const uint32_t tmem_base = ctl->tmem_base;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA producer (both CTAs)
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmap) : "memory");
      uint32_t stage = 0, phase = 0;
      int64_t issued = 0;
      int band = 0;
      bool ok = true;
      const bool skip = *reinterpret_cast<volatile int*>(&g_fault_skip_tma) != 0;
      for (int64_t t = cl; t < total && ok && !skip; t += ncl) {
        int64_t bi2, bj;
        decode_tile(ts, t * nshards + shard, &band, &bi2, &bj);
        const int ya = (int)((2 * bi2 + rank) * BM), yb = (int)(bj * BN + rank * (BN / 2));
        for (int64_t kc = 0; kc < kchunks; ++kc) {
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1u, abort_flag)) { ok = false; break; }
          uint8_t* sa = smem + stage * P_STAGE_BYTES;
          const uint32_t full_c = mapa_shared(smem_u32(&ctl->full[stage]), 0u);  // the leader's full[stage]
          if (rank == 0) mbar_arrive_expect_tx(&ctl->full[stage], 2 * P_STAGE_BYTES);
          tma_load_2d_pair(sa, &tmap, full_c, (int)(kc * BK), ya);
          tma_load_2d_pair(sa + PA_BYTES, &tmap, full_c, (int)(kc * BK), yb);
          ++issued;
          if (++stage == P_STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&sc->status, 4u);
      }
      // drain (leader): the last stages' copies of both CTAs land on its full barriers
      if (rank == 0) {
        const int64_t last = issued < P_STAGES ? issued : P_STAGES;
        for (int64_t q = 1; q <= last; ++q) {
          const int64_t u = issued - q;
          const uint32_t s = (uint32_t)(u % P_STAGES), par = (uint32_t)((u / P_STAGES) & 1);
          const uint64_t t0 = globaltimer();
          while (!mbar_try_wait(&ctl->full[s], par) && globaltimer() - t0 < WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---------------------------------------------------------------- pair MMA issuer (leader)
      const uint32_t idesc = make_idesc(ab_fmt, 2 * BM, BN);
      uint32_t stage = 0, phase = 0;
      int64_t it = 0;
      bool ok = true;
      for (int64_t t = cl; t < total && ok; t += ncl, ++it) {
        const uint32_t acc = (uint32_t)(it & 1), use = (uint32_t)((it >> 1) & 1);
        if (!mbar_wait(&ctl->tempty[acc], use ^ 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        const uint32_t dtmem = tmem_base + acc * (uint32_t)BN;
        for (int64_t kc = 0; kc < kchunks; ++kc) {
          if (!mbar_wait(&ctl->full[stage], phase, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * P_STAGE_BYTES);
          const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + PA_BYTES);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_f16_pair(dtmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc | kk) != 0);
          const uint32_t e = smem_u32(&ctl->empty[stage]);
          mma_commit_pair(e);
          mma_commit_pair(mapa_shared(e, 1u));
          if (++stage == P_STAGES) { stage = 0; phase ^= 1u; }
        }
        if (!ok) break;
        const uint32_t f = smem_u32(&ctl->tfull[acc]);
        mma_commit_pair(f);
        mma_commit_pair(mapa_shared(f, 1u));
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&sc->status, 4u);
      }
      // drain: the commits arrive once every pair MMA issued so far has completed
      const uint32_t dr = smem_u32(&ctl->drain);
      mma_commit_pair(dr);
      mma_commit_pair(mapa_shared(dr, 1u));
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < WAIT_NS) {
      }
    } else if (lane == 0) {
      // the peer: its TMEM and shared memory are in use until the leader's last pair MMA completes
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < WAIT_NS) {
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 2..5, both CTAs)
    const uint32_t quarter = (uint32_t)(warp & 3);
    const BoundParams bp = sc->bp;
    EpiState es;
    epi_init(es, sc, bp);
    int64_t it = 0;
    int band = 0;
    for (int64_t t = cl; t < total; t += ncl, ++it) {
      int64_t bi2, bj;
      decode_tile(ts, t * nshards + shard, &band, &bi2, &bj);
      const uint32_t acc = (uint32_t)(it & 1), use = (uint32_t)((it >> 1) & 1);
      const bool got = __all_sync(0xffffffffu, mbar_wait(&ctl->tfull[acc], use, abort_flag));
      if (!got) {
        if (lane == 0) {
          *abort_flag = 1;
          atomicOr(&sc->status, 4u);
        }
        break;
      }
      tc_fence_after();
      const uint32_t tbase = tmem_base + ((quarter * 32u) << 16) + acc * (uint32_t)BN;
      epi_tile<false>((2 * bi2 + (int64_t)rank) * BM, bj * BN, tbase, lane, quarter, ts.n, ts.excl, norms, bp, sc,
                      cand, cap, es, nullptr, 1);
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {  // the leader's tempty[acc]: a local arrive in the leader, a remote one from the peer
        if (rank == 0) mbar_arrive(&ctl->tempty[acc]);
        else mbar_arrive_cluster(mapa_shared(smem_u32(&ctl->tempty[acc]), 0u));
      }
      epi_publish(lane, bp, sc, es);
      if (__any_sync(0xffffffffu, *abort_flag != 0)) break;
    }
    tc_fence_before();
  }

  __syncthreads();
  cluster_sync();  // no cross-CTA arrive or commit is pending past this point
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace

bool gram_tc_available() { return true; }

EncodeTiledFn tensor_map_encoder() {
  // a function-local static is initialised exactly once, even under concurrent first calls
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return nullptr;
  }();
  return fn;
}

int set_fault_gram_tc(int on) {
  CPPGB_CUDA_TRY(cudaMemcpyToSymbol(g_fault_skip_tma, &on, sizeof on));
  return CPPGB_OK;
}

namespace {
// The band schedule of all tiles; returns their number.  rstep = 2: the rows of the schedule are
// pairs of 128-row blocks (a CTA pair's 256 x 256 tile); a pair's columns start where its first
// (lower) row block's do.
int64_t build_sched(int64_t n, int64_t n_pad, int64_t excl, TileSched& ts, int rstep = 1) {
  ts.n = n;
  ts.excl = excl;
  ts.rstep = rstep;
  ts.pad = 0;
  ts.nbi = (int32_t)(n_pad / (BM * rstep));
  ts.nbj = (int32_t)(n_pad / BN);
  int band = tuned_dense_band() > 0 ? tuned_dense_band() : BAND;
  while ((ts.nbj + band - 1) / band > MAX_BANDS) band *= 2;
  ts.band = band;
  ts.nbands = (int32_t)((ts.nbj + band - 1) / band);

  int64_t total = 0;
  for (int b = 0; b < ts.nbands; ++b) {
    const int64_t bj0 = (int64_t)b * band, bj1 = bj0 + band < ts.nbj ? bj0 + band : ts.nbj;
    ts.off[b] = total;
    int32_t nf = 0;
    bool in_full = true;
    for (int64_t bi = 0; bi < ts.nbi; ++bi) {
      const int64_t c = row_count(bi * rstep, bj0, bj1, n, excl);
      if (in_full && c == bj1 - bj0) ++nf;
      else in_full = false;
      total += c;
    }
    ts.nfull[b] = nf;
  }
  ts.off[ts.nbands] = total;
  return total;
}
}  // namespace

int64_t gram_tc_tile_count(int64_t n, int64_t n_pad, int64_t excl, int64_t shard, int64_t nshards) {
  TileSched ts;
  const int64_t all_tiles = build_sched(n, n_pad, excl, ts);
  return all_tiles > shard ? (all_tiles - shard + nshards - 1) / nshards : 0;
}

int launch_gram_tc_prune_list(int64_t n, int64_t n_pad, int64_t excl, const float* blo, const float* bhi,
                              const DenseScalars* sc, int32_t* flags, int64_t* pos, int64_t* tmp, int32_t* list,
                              cudaStream_t st, int64_t shard, int64_t nshards) {
  TileSched ts;
  const int64_t all_tiles = build_sched(n, n_pad, excl, ts);
  const int64_t total = all_tiles > shard ? (all_tiles - shard + nshards - 1) / nshards : 0;
  if (total > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "too many tiles for the pruned list");
  if (total == 0) {
    CPPGB_CUDA_TRY(cudaMemsetAsync(pos, 0, sizeof(int64_t), st));
    return CPPGB_OK;
  }
  const unsigned nb = (unsigned)((total + 255) / 256);
  prune_flags_kernel<<<nb, 256, 0, st>>>(ts, total, shard, nshards, blo, bhi, n_pad / BM, sc, flags);
  CPPGB_LAUNCH_CHECK();
  int rc = launch_exclusive_scan_i32(flags, total, pos, tmp, st);  // pos[total] = kept tiles
  if (rc) return rc;
  prune_compact_kernel<<<nb, 256, 0, st>>>(total, shard, nshards, flags, pos, list);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int launch_gram_tc(const void* X, int mode, int64_t n, int64_t n_pad, int64_t Kp, int64_t excl, const float* norms,
                   DenseScalars* sc, Candidate* cand, int64_t cap, cudaStream_t st, int64_t shard, int64_t nshards,
                   const int32_t* tlist, const int64_t* tcount, const int32_t* perm, int64_t excl_orig,
                   float* dump, int64_t dump_tiles, const unsigned int* gate) {
  if (Kp % BK || n_pad % BN) return set_error(CPPGB_ERR_ARG, "internal: tensor-core stage needs Kp %% 64 == 0");
  if (((uintptr_t)X & 15) != 0) return set_error(CPPGB_ERR_ARG, "internal: row matrix must be 16-byte aligned");
  if (n_pad > 0x7fffffffLL || Kp > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "problem too large for TMA coordinates");
  TileSched ts;  // kernel parameter (copied at launch)
  const int64_t all_tiles = build_sched(n, n_pad, excl, ts);
  // this shard's tiles are t = k * nshards + shard; the kernel walks k (or the pruned list's entries)
  const int64_t total = all_tiles > shard ? (all_tiles - shard + nshards - 1) / nshards : 0;
  if (dump ? dump_tiles == 0 : total == 0) return CPPGB_OK;

  EncodeTiledFn enc = tensor_map_encoder();
  if (!enc) return set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  CUtensorMap tmap;
  const cuuint64_t gdim[2] = {(cuuint64_t)Kp, (cuuint64_t)n_pad};
  const cuuint64_t gstride[1] = {(cuuint64_t)Kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapDataType dt =
      mode == CPPGB_MODE_FILTER_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult cr = enc(&tmap, dt, 2, const_cast<void*>(X), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);

  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint32_t ab = mode == CPPGB_MODE_FILTER_BF16 ? 1u : 0u;
  if (!dump && !perm && !tlist && tuned_dense_shape() == 2) {
    // 256 x 256 tiles on CTA pairs: the schedule's rows are pairs of 128-row blocks
    TileSched ts2;
    const int64_t all2 = build_sched(n, n_pad, excl, ts2, 2);
    const int64_t total2 = all2 > shard ? (all2 - shard + nshards - 1) / nshards : 0;
    if (total2 == 0) return CPPGB_OK;
    const size_t smem2 = (size_t)P_STAGES * P_STAGE_BYTES + sizeof(PairCtl) + 1024;
    CPPGB_CUDA_TRY(cudaFuncSetAttribute(gram_tc_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    int clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(sms & ~1));
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = smem2;
    cfg.stream = st;
    CPPGB_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, gram_tc_pair_kernel, &cfg));
    if (clusters < 1) return set_error(CPPGB_ERR_CUDA, "no CTA pair of the dense stage fits on the device");
    const int64_t ncl = total2 < clusters ? total2 : clusters;
    gram_tc_pair_kernel<<<(unsigned)(2 * ncl), NTHREADS, smem2, st>>>(tmap, ts2, total2, ab, norms, sc, cand, cap,
                                                                      Kp / BK, shard, nshards, gate);
    CPPGB_LAUNCH_CHECK();
    return CPPGB_OK;
  }
  const size_t smem = (size_t)STAGES * STAGE_BYTES + sizeof(SmemCtl) + 1024;
  const int64_t grid = total < sms ? total : sms;
  if (dump) {
    CPPGB_CUDA_TRY(
        cudaFuncSetAttribute(gram_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t g = dump_tiles < sms ? dump_tiles : sms;
    gram_tc_kernel<false, true><<<(unsigned)g, NTHREADS, smem, st>>>(
        tmap, ts, dump_tiles, ab, norms, sc, cand, cap, Kp / BK, 0, 1, tlist, nullptr, nullptr, 1, dump, nullptr);
  } else if (perm) {
    CPPGB_CUDA_TRY(
        cudaFuncSetAttribute(gram_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    gram_tc_kernel<true, false><<<(unsigned)grid, NTHREADS, smem, st>>>(
        tmap, ts, total, ab, norms, sc, cand, cap, Kp / BK, shard, nshards, tlist, tcount, perm, excl_orig, nullptr,
        gate);
  } else {
    CPPGB_CUDA_TRY(
        cudaFuncSetAttribute(gram_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    gram_tc_kernel<false, false><<<(unsigned)grid, NTHREADS, smem, st>>>(
        tmap, ts, total, ab, norms, sc, cand, cap, Kp / BK, shard, nshards, tlist, tcount, nullptr, 1, nullptr, gate);
  }
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

}  // namespace cppgb
