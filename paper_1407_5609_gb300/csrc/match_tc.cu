// Exact match counts of categorical rows on the tensor cores.
//
// Two rows of symbols are compared through the dot products of small-integer encodings: FP8 (E4M3)
// operands with values in {0, 1, 2, 4} (all exact in E4M3), tcgen05.mma kind::f8f6f4 accumulating in
// FP32.  Every product is at most 16 and every partial sum at most 16 m < 2^24 -- the entry points
// reject groups of 2^20 or more subjects (and strings of more than 2^23 positions) -- so the
// accumulators hold the exact integer counts.
//
//  * Two-locus (Sec. 6) with the one-hot planes of Sec. 5.3 (a = [g_i = 1], b = [g_i = 2],
//    c = [g_j = 1], d = [g_j = 2] per subject): the number of subjects whose genotypes match is
//      u = m - s_i - s_j + [a, b] . [2c + d, c + 2d],   s = sum (a + b),
//    because [g_i = g_j] = (1 - a - b)(1 - c - d) + ac + bd.  The score is |u_A m2 - u_B m1|.
//  * Pearson's correlation of the genotype values x = a + 2b: sum x_i x_j = [a, b] . [c + 2d, 2c + 4d];
//    r = (m Sxy - Sx_i Sx_j) / sqrt(vx_i vx_j), vx = m Sxx - Sx^2, and the score |r_A - r_B| is formed
//    in FP64 with the same operations as the oracle, so it is bit-identical.
//  * Strings over sigma symbols (Sec. 4), one-hot per position (the mapping of Sec. 5.5): the dot
//    product of two one-hot rows is the number of positions where the strings agree, so the pair
//    with the most (fewest) matches is the closest (least correlated) pair under the Hamming distance.
//
// Kernel: one persistent CTA per SM over the 128 x 128 tiles (bi <= bj) of the upper triangle; warp
// 0 loads K-chunks of the left and right rows with TMA (6 stages of 32 KB), warp 1 issues the MMAs
// into 128-column TMEM accumulators (four tiles in flight with one group, two with two groups), and
// eight epilogue warps (two per TMEM lane quarter, each on half the columns) turn each pair's counts
// into a 64-bit key (larger is better, ties to the smaller (i, j)) and keep the best per CTA.
#include <cuda_bf16.h>

#include <cstring>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace cppgb {
namespace {
using namespace tc;

// Operands are FP8 E4M3 (one byte; 0, 1, 2 and 4 are exact), so a stage holds 128 K values per row
// (one 128-byte swizzle atom) and one MMA covers K = 32.
constexpr int BM = 128, BN = 128, BK = 128, STAGES = 6;
constexpr int A_BYTES = BM * BK, B_BYTES = BN * BK, STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;                  // two per TMEM lane quarter, each on half the tile's columns
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;  // producer, MMA issuer, epilogue
constexpr uint32_t TMEM_COLS = 512;            // 4 tiles in flight (one group) or 2 (two groups) x 128 columns
constexpr int MAX_ACC = 4;

struct MatchMaps {
  CUtensorMap L[2], R[2];
};

struct MatchParams {
  int64_t S;              // rows
  int32_t groups, mode;   // 1 or 2 groups; MatchMode
  int64_t kch[2];         // K chunks of BK per group
  int64_t t0, tstride;    // shard: the tiles t = t0 + k tstride of the triangle's order (0, 1: all)
  int64_t m[2];           // two-locus: group sizes; strings: the length t (m[0])
  const int32_t* s[2];    // two-locus count: sum (a + b) per row
  const int64_t* sx[2];   // Pearson: sum x and m sum x^2 - (sum x)^2 per row
  const int64_t* vx[2];
};

// Fault injection for the tests of the bounded waits (cpp_set_fault_injection): when non-zero the TMA
// producer issues no copy, so the MMA issuer's and the epilogue's waits run out and the scan reports
// CPPGB_ERR_TIMEOUT.  Zero unless a test sets it.
__device__ int g_fault_skip_tma = 0;

struct Ctl {
  uint64_t full[STAGES], empty[STAGES], tfull[MAX_ACC], tempty[MAX_ACC], drain;
  MatchPartial red[EPI_WARPS];
  unsigned long long cta_best;  // strings: the best key any thread of the CTA has found
  uint32_t tmem_base;
  int abort_flag;
};
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + sizeof(Ctl) + 1024;

__device__ __forceinline__ void tri_tile(int64_t t, int64_t nb, int64_t* bi, int64_t* bj) {
  // row k holds nb - k tiles (bj = k .. nb - 1); the tiles before row k number k nb - k (k - 1) / 2
  int64_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (mid * nb - mid * (mid - 1) / 2 <= t) lo = mid;
    else hi = mid - 1;
  }
  *bi = lo;
  *bj = lo + (t - (lo * nb - lo * (lo - 1) / 2));
}

// the tile G further on in the same order (callers make sure it exists, so the loop ends inside the
// triangle): rows shrink as bi grows, so the position wraps row by row
__device__ __forceinline__ void tri_next(int64_t G, int64_t nb, int64_t& bi, int64_t& bj) {
  int64_t pos = bj - bi + G;
  while (pos >= nb - bi) {
    pos -= nb - bi;
    ++bi;
  }
  bj = bi + pos;
}

__device__ __forceinline__ bool better(unsigned long long k, int i, int j, unsigned long long bk, int bi, int bj) {
  if (bi < 0) return true;
  if (k != bk) return k > bk;
  if (i != bi) return i < bi;
  return j < bj;
}

// the best key a 32-column chunk of string matches can give: most agreeing positions (most) or
// most mismatches (t - fewest agreeing), from a max / min tree over the FP32 counts
template <bool MOST>
__device__ __forceinline__ unsigned long long chunk_key(const uint32_t (&r)[32], int64_t t) {
  float m[16];
#pragma unroll
  for (int k = 0; k < 16; ++k)
    m[k] = MOST ? fmaxf(__uint_as_float(r[k]), __uint_as_float(r[k + 16]))
                : fminf(__uint_as_float(r[k]), __uint_as_float(r[k + 16]));
#pragma unroll
  for (int w = 8; w >= 1; w >>= 1)
#pragma unroll
    for (int k = 0; k < w; ++k) m[k] = MOST ? fmaxf(m[k], m[k + w]) : fminf(m[k], m[k + w]);
  return MOST ? (unsigned long long)m[0] : (unsigned long long)(t - (int64_t)m[0]);
}

__device__ __forceinline__ double pearson_r(int64_t m, int64_t sxy, int64_t sxi, int64_t sxj, int64_t vxi, int64_t vxj) {
  if (vxi == 0 || vxj == 0) return 0.0;
  const double num = (double)(m * sxy - sxi * sxj);
  const double den = __dsqrt_rn(__dmul_rn((double)vxi, (double)vxj));
  return __ddiv_rn(num, den);
}

// One instantiation per measure (MatchMode): each carries only its own epilogue arithmetic.
template <int MODE>
__global__ void __launch_bounds__(NTHREADS, 1)
    match_tc_kernel(const __grid_constant__ MatchMaps maps, const __grid_constant__ MatchParams mp, int64_t total,  // tiles of the shard
                    int64_t nb, MatchPartial* __restrict__ partials, unsigned int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  Ctl* ctl = (Ctl*)(smem + STAGES * STAGE_BYTES);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int a = 0; a < MAX_ACC; ++a) {
      mbar_init(&ctl->tfull[a], 1);
      mbar_init(&ctl->tempty[a], EPI_WARPS);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_flag = 0;
    ctl->cta_best = 0ull;
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
  // accumulators in flight: TMEM holds 512 columns, a tile needs 128 per group
  const uint32_t nacc = mp.groups == 1 ? 4u : 2u, acc_cols = (uint32_t)mp.groups * (uint32_t)BN;

  if (warp == 0) {
    if (lane == 0) {  // ---------------------------------------------- TMA producer
      for (int g = 0; g < mp.groups; ++g) {
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.L[g]) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.R[g]) : "memory");
      }
      uint32_t stage = 0, phase = 0;
      int64_t issued = 0;
      bool ok = true;
      int64_t bi = 0, bj = 0;
      if ((int64_t)blockIdx.x < total) tri_tile(mp.t0 + (int64_t)blockIdx.x * mp.tstride, nb, &bi, &bj);
      const bool skip = *reinterpret_cast<volatile int*>(&g_fault_skip_tma) != 0;
      for (int64_t t = blockIdx.x; t < total && ok && !skip; t += gridDim.x) {
        if (t != (int64_t)blockIdx.x) tri_next((int64_t)gridDim.x * mp.tstride, nb, bi, bj);
        for (int g = 0; g < mp.groups && ok; ++g)
          for (int64_t kc = 0; kc < mp.kch[g]; ++kc) {
            if (!mbar_wait(&ctl->empty[stage], phase ^ 1u, abort_flag)) { ok = false; break; }
            uint8_t* sa = smem + stage * STAGE_BYTES;
            mbar_arrive_expect_tx(&ctl->full[stage], STAGE_BYTES);
            tma_load_2d(sa, &maps.L[g], &ctl->full[stage], (int)(kc * BK), (int)(bi * BM));
            tma_load_2d(sa + A_BYTES, &maps.R[g], &ctl->full[stage], (int)(kc * BK), (int)(bj * BN));
            ++issued;
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
          }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, 4u);
      }
      const int64_t last = issued < STAGES ? issued : STAGES;
      for (int64_t k = 1; k <= last; ++k) {  // drain: every issued copy lands before exit
        const int64_t u = issued - k;
        const uint32_t s = (uint32_t)(u % STAGES), par = (uint32_t)((u / STAGES) & 1);
        const uint64_t t0 = globaltimer();
        while (!mbar_try_wait(&ctl->full[s], par) && globaltimer() - t0 < WAIT_NS) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // ---------------------------------------------- MMA issuer
      const uint32_t idesc = make_idesc_f8(BM, BN);  // E4M3 operands, FP32 accumulator
      uint32_t stage = 0, phase = 0;
      int64_t it = 0;
      bool ok = true;
      uint32_t acc = 0, use = 0;
      for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
        if (t != (int64_t)blockIdx.x && ++acc == nacc) {
          acc = 0;
          use ^= 1u;
        }
        if (!mbar_wait(&ctl->tempty[acc], use ^ 1u, abort_flag)) { ok = false; break; }
        tc_fence_after();
        for (int g = 0; g < mp.groups && ok; ++g) {
          const uint32_t dtmem = tmem_base + acc * acc_cols + (uint32_t)g * (uint32_t)BN;
          for (int64_t kc = 0; kc < mp.kch[g]; ++kc) {
            if (!mbar_wait(&ctl->full[stage], phase, abort_flag)) { ok = false; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
            const uint64_t ad = sw128_desc(sa), bd = sw128_desc(sa + A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 32; ++kk)  // K = 32 bytes per MMA: +2 in 16-byte descriptor units
              mma_f8(dtmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, (kc | kk) != 0);
            mma_commit(&ctl->empty[stage]);
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
          }
        }
        if (!ok) break;
        mma_commit(&ctl->tfull[acc]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(status, 4u);
      }
      mma_commit(&ctl->drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < WAIT_NS) {
      }
    }
  } else {  // -------------------------------------------------------- epilogue (warps 2 .. 2 + EPI_WARPS - 1)
    // warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 (its lane quarter) and the half (w - 2) / 4
    // of the tile's columns
    const uint32_t quarter = (uint32_t)(warp & 3);
    const int half = (warp - 2) / 4;
    unsigned long long bk = 0ull;
    int bi_best = -1, bj_best = -1;
    int64_t it = 0;
    bool ok = true;
    constexpr bool ham = MODE == MATCH_HAMMING_MIN || MODE == MATCH_HAMMING_MAX;
    constexpr bool most = MODE == MATCH_HAMMING_MIN;
    int64_t bi = 0, bj = 0;
    if ((int64_t)blockIdx.x < total) tri_tile(mp.t0 + (int64_t)blockIdx.x * mp.tstride, nb, &bi, &bj);
    uint32_t acc = 0, use = 0;
    for (int64_t t = blockIdx.x; t < total && ok; t += gridDim.x, ++it) {
      if (t != (int64_t)blockIdx.x) {
        tri_next((int64_t)gridDim.x * mp.tstride, nb, bi, bj);
        if (++acc == nacc) {
          acc = 0;
          use ^= 1u;
        }
      }
      if (!__all_sync(0xffffffffu, mbar_wait(&ctl->tfull[acc], use, abort_flag))) { ok = false; break; }
      tc_fence_after();
      const int64_t i = bi * BM + quarter * 32 + lane;
      const bool row_ok = i < mp.S;
      const int64_t ii = row_ok ? i : 0;
      const uint32_t tb = tmem_base + ((quarter * 32u) << 16) + acc * acc_cols;
      int32_t sAi = 0, sBi = 0;
      int64_t sxAi = 0, sxBi = 0, vxAi = 0, vxBi = 0;
      if (MODE == MATCH_TL_COUNT) {
        sAi = mp.s[0][ii];
        sBi = mp.s[1][ii];
      } else if (MODE == MATCH_TL_PEARSON) {
        sxAi = mp.sx[0][ii];
        sxBi = mp.sx[1][ii];
        vxAi = mp.vx[0][ii];
        vxBi = mp.vx[1][ii];
      }
      // the pair (i, j) with the accumulators a (group A / strings) and b (group B) as FP32 bits
      auto consider = [&](int64_t j, uint32_t a, uint32_t b) {
        if (!(row_ok && j < mp.S && j > i)) return;
        const int64_t accA = (int64_t)__uint_as_float(a);
        unsigned long long key;
        if (MODE == MATCH_TL_COUNT) {
          const int64_t accB = (int64_t)__uint_as_float(b);
          const int64_t uA = mp.m[0] - sAi - mp.s[0][j] + accA;
          const int64_t uB = mp.m[1] - sBi - mp.s[1][j] + accB;
          const int64_t sc = uA * mp.m[1] - uB * mp.m[0];
          key = (unsigned long long)(sc < 0 ? -sc : sc);
        } else if (MODE == MATCH_TL_PEARSON) {
          const int64_t accB = (int64_t)__uint_as_float(b);
          const double rA = pearson_r(mp.m[0], accA, sxAi, mp.sx[0][j], vxAi, mp.vx[0][j]);
          const double rB = pearson_r(mp.m[1], accB, sxBi, mp.sx[1][j], vxBi, mp.vx[1][j]);
          key = (unsigned long long)__double_as_longlong(fabs(__dsub_rn(rA, rB)));
        } else if (MODE == MATCH_HAMMING_MIN) {
          key = (unsigned long long)accA;  // most agreeing positions = fewest mismatches
        } else {
          key = (unsigned long long)(mp.m[0] - accA);  // most mismatches
        }
        if (better(key, (int)i, (int)j, bk, bi_best, bj_best)) {
          bk = key;
          bi_best = (int)i;
          bj_best = (int)j;
          if (ham) atomicMax(&ctl->cta_best, key);
        }
      };
      if (ham) {
        // both 32-column chunks of this half in flight at once, one wait
        uint32_t ra[32], rb[32];
        const uint32_t c0 = (uint32_t)(half * 64);
        tmem_ld32_nowait(tb + c0, ra);
        tmem_ld32_nowait(tb + c0 + 32u, rb);
        tmem_wait_ld(ra);
        tmem_wait_ld(rb);
        const int64_t j0 = bj * BN + c0;
        // per chunk, its best count (a 31-op tree) decides whether any entry can reach or tie the
        // best key found so far in the CTA (a key some pair has, so a smaller one cannot win); the
        // tree also counts the masked entries of edge tiles, which can only raise it.  Most chunks
        // are skipped.
        const unsigned long long cb = *(volatile unsigned long long*)&ctl->cta_best;
        const unsigned long long bar = cb > bk ? cb : bk;
        if (chunk_key<most>(ra, mp.m[0]) >= bar) {
#pragma unroll
          for (int k = 0; k < 32; ++k) consider(j0 + k, ra[k], 0u);
        }
        if (chunk_key<most>(rb, mp.m[0]) >= bar) {
#pragma unroll
          for (int k = 0; k < 32; ++k) consider(j0 + 32 + k, rb[k], 0u);
        }
      } else {
#pragma unroll 1
        for (int c = 2 * half; c < 2 * half + 2; ++c) {
          uint32_t ra[32], rb[32];
          tmem_ld32(tb + (uint32_t)(c * 32), ra);
          if (mp.groups == 2) tmem_ld32(tb + (uint32_t)BN + (uint32_t)(c * 32), rb);
#pragma unroll
          for (int k = 0; k < 32; ++k) consider(bj * BN + c * 32 + k, ra[k], mp.groups == 2 ? rb[k] : 0u);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->tempty[acc]);
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(status, 4u);
    }
    // best of the warp, then of the epilogue warps
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok2 = __shfl_xor_sync(0xffffffffu, bk, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi_best, o), oj = __shfl_xor_sync(0xffffffffu, bj_best, o);
      if (oi >= 0 && better(ok2, oi, oj, bk, bi_best, bj_best)) {
        bk = ok2;
        bi_best = oi;
        bj_best = oj;
      }
    }
    if (lane == 0) ctl->red[warp - 2] = MatchPartial{(long long)bk, bi_best, bj_best};
    asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS) : "memory");  // the epilogue warps, once, after their loops
    if (warp == 2 && lane == 0) {
      MatchPartial b = ctl->red[0];
      for (int w = 1; w < EPI_WARPS; ++w) {
        const MatchPartial o = ctl->red[w];
        if (o.i >= 0 && better((unsigned long long)o.key, o.i, o.j, (unsigned long long)b.key, b.i, b.j)) b = o;
      }
      if (b.i < 0) b.key = -1;
      partials[blockIdx.x] = b;
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

// ---------------------------------------------------------------- preparation
__device__ __forceinline__ uint8_t e4m3_small(int v) {  // exact E4M3 bits of 0 .. 4 (exponent bias 7)
  return v == 0 ? 0x00 : v == 1 ? 0x38 : v == 2 ? 0x40 : v == 3 ? 0x44 : 0x48;
}

// Two-locus rows: one warp per (row, group).  L = [a bits, b bits] of the group's W words (K = 128 W);
// R = [2c + d, c + 2d] (count) or [c + 2d, 2c + 4d] (Pearson); rows >= S are zero.  Per-row sums:
// s = sum (a + b) (count); Sx = sum (a + 2b), vx = m Sxx - Sx^2 with Sxx = sum (a + 4b) (Pearson).
__global__ void tl_prep_kernel(const uint64_t* __restrict__ planes, int64_t S, int64_t S_pad, int64_t W, int64_t m1,
                               int64_t m2, int mode, uint8_t* L0, uint8_t* R0, uint8_t* L1, uint8_t* R1,
                               int32_t* s0, int32_t* s1, int64_t* sx0, int64_t* sx1, int64_t* vx0, int64_t* vx1) {
  const int lane = threadIdx.x & 31;
  const int64_t w_id = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w_id >= 2 * S_pad) return;
  const int64_t row = w_id >> 1;
  const int g = (int)(w_id & 1);
  const int64_t K = 128 * W;
  uint8_t* L = (g == 0 ? L0 : L1) + row * K;
  uint8_t* R = (g == 0 ? R0 : R1) + row * K;
  long long sa = 0, sb = 0;
  for (int64_t w = lane; w < W; w += 32) {
    uint64_t a = 0, b = 0;
    if (row < S) {
      a = planes[((row * 2 + g) * 2 + 0) * W + w];
      b = planes[((row * 2 + g) * 2 + 1) * W + w];
    }
    sa += __popcll(a);
    sb += __popcll(b);
    for (int q = 0; q < 64; q += 16) {  // 16 subjects per 16-byte store
      uint8_t la[16], lb[16], r1[16], r2[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int ab = (int)((a >> (q + e)) & 1), bb = (int)((b >> (q + e)) & 1);
        la[e] = e4m3_small(ab);
        lb[e] = e4m3_small(bb);
        if (mode == MATCH_TL_COUNT) {
          r1[e] = e4m3_small(2 * ab + bb);
          r2[e] = e4m3_small(ab + 2 * bb);
        } else {
          r1[e] = e4m3_small(ab + 2 * bb);
          r2[e] = e4m3_small(2 * ab + 4 * bb);
        }
      }
      *reinterpret_cast<uint4*>(L + 64 * w + q) = *reinterpret_cast<const uint4*>(la);
      *reinterpret_cast<uint4*>(L + 64 * W + 64 * w + q) = *reinterpret_cast<const uint4*>(lb);
      *reinterpret_cast<uint4*>(R + 64 * w + q) = *reinterpret_cast<const uint4*>(r1);
      *reinterpret_cast<uint4*>(R + 64 * W + 64 * w + q) = *reinterpret_cast<const uint4*>(r2);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
  }
  if (lane == 0) {
    if (mode == MATCH_TL_COUNT) {
      (g == 0 ? s0 : s1)[row] = (int32_t)(sa + sb);
    } else {
      const int64_t m = g == 0 ? m1 : m2;
      const int64_t sx = sa + 2 * sb, sxx = sa + 4 * sb;
      (g == 0 ? sx0 : sx1)[row] = sx;
      (g == 0 ? vx0 : vx1)[row] = m * sxx - sx * sx;
    }
  }
}

// One-hot rows of strings: X[row][p sigma + v] = 1 where s[row][p] = v (X zeroed before); one warp per row.
__global__ void ham_prep_kernel(const uint8_t* __restrict__ strs, int64_t n, int64_t t, int64_t ld, int sigma,
                                uint8_t* __restrict__ X, int64_t K, unsigned int* status) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  bool bad = false;
  for (int64_t p = lane; p < t; p += 32) {
    const int v = strs[row * ld + p];
    if (v >= sigma) {
      bad = true;
      continue;
    }
    X[row * K + p * sigma + v] = 0x38;  // E4M3 1.0
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, 1u);
}

// Best of the per-CTA partials (one block).
__global__ void match_finish_kernel(const MatchPartial* __restrict__ partials, int64_t np, MatchPartial* out) {
  __shared__ MatchPartial red[256];
  MatchPartial b{-1, -1, -1};
  for (int64_t q = threadIdx.x; q < np; q += blockDim.x) {
    const MatchPartial o = partials[q];
    if (o.i >= 0 && better((unsigned long long)o.key, o.i, o.j, (unsigned long long)b.key, b.i, b.j)) b = o;
  }
  red[threadIdx.x] = b;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) {
      const MatchPartial o = red[threadIdx.x + s], c = red[threadIdx.x];
      if (o.i >= 0 && better((unsigned long long)o.key, o.i, o.j, (unsigned long long)c.key, c.i, c.j))
        red[threadIdx.x] = o;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

int encode_rows(CUtensorMap* m, void* base, int64_t rows, int64_t K) {
  const EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) return set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)K};  // one byte per value; K is a multiple of 128
  const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)BM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return CPPGB_OK;
}

int launch_match(const MatchMaps& maps, const MatchParams& mp, MatchPartial* partials, int64_t* np_out,
                 unsigned int* status, cudaStream_t st) {
  const int64_t nb = (mp.S + BM - 1) / BM;
  const int64_t all = nb * (nb + 1) / 2;
  const int64_t total = mp.t0 < all ? (all - mp.t0 + mp.tstride - 1) / mp.tstride : 0;  // this shard's tiles
  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t grid = total < sms ? total : sms;
  *np_out = grid;
  if (grid == 0) return CPPGB_OK;
  auto kern = mp.mode == MATCH_TL_COUNT      ? match_tc_kernel<MATCH_TL_COUNT>
              : mp.mode == MATCH_TL_PEARSON  ? match_tc_kernel<MATCH_TL_PEARSON>
              : mp.mode == MATCH_HAMMING_MIN ? match_tc_kernel<MATCH_HAMMING_MIN>
                                             : match_tc_kernel<MATCH_HAMMING_MAX>;
  CPPGB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES));
  kern<<<(unsigned)grid, NTHREADS, SMEM_BYTES, st>>>(maps, mp, total, nb, partials, status);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

struct TLLayout {
  uint8_t *L[2], *R[2];
  int32_t* s[2];
  int64_t *sx[2], *vx[2];
  MatchPartial* partials;
  twolocus_result* dres;
  unsigned int* status;
  size_t bytes;
};

TLLayout tl_layout(void* ws, int64_t S, int64_t W) {
  TLLayout L;
  Carver c(ws);
  const int64_t S_pad = (S + BM - 1) / BM * BM, K = 128 * W;
  for (int g = 0; g < 2; ++g) {
    L.L[g] = c.take<uint8_t>((size_t)(S_pad > 0 ? S_pad : BM) * K);
    L.R[g] = c.take<uint8_t>((size_t)(S_pad > 0 ? S_pad : BM) * K);
    L.s[g] = c.take<int32_t>(S_pad + 1);
    L.sx[g] = c.take<int64_t>(S_pad + 1);
    L.vx[g] = c.take<int64_t>(S_pad + 1);
  }
  L.partials = c.take<MatchPartial>(1024);
  L.dres = c.take<twolocus_result>(1);
  L.status = c.take<unsigned int>(1);
  L.bytes = c.bytes();
  return L;
}

// The results on the device (copied to the caller's host struct): the Pearson score from its
// bits, the status from the kernels' flags (1: a symbol >= sigma, 4: a timed-out wait).
__global__ void tl_tc_result_kernel(twolocus_result* r, const unsigned int* status, int pearson) {
  twolocus_result v = *r;
  if (pearson && v.i >= 0) {
    v.score_real = __longlong_as_double((long long)v.score);
    v.score = -1;  // the Pearson measure has no integer score
  }
  v.status = (*status & 4u) ? CPPGB_ERR_TIMEOUT : CPPGB_OK;
  if (v.status != CPPGB_OK) {
    v.i = v.j = -1;
    v.score = -1;
    v.score_real = -1.0;
  }
  v.reserved = 0;
  *r = v;
}

__global__ void ham_result_kernel(const MatchPartial* best, const unsigned int* status, int least, int64_t t,
                                  hamming_result* out) {
  hamming_result r;
  r.i = r.j = -1;
  r.mismatches = -1;
  r.reserved = 0;
  const unsigned int s = *status;
  r.status = (s & 1u) ? CPPGB_ERR_ARG : (s & 4u) ? CPPGB_ERR_TIMEOUT : CPPGB_OK;
  if (r.status == CPPGB_OK && best->i >= 0) {
    r.i = best->i;
    r.j = best->j;
    r.mismatches = least ? best->key : t - best->key;
  }
  *out = r;
}

struct HamLayout {
  uint8_t* X;
  MatchPartial *partials, *best;
  unsigned int* status;
  hamming_result* res;
  size_t bytes;
};

HamLayout ham_layout(void* ws, int64_t n, int64_t K) {
  HamLayout L;
  Carver c(ws);
  const int64_t n_pad = (n + BM - 1) / BM * BM;
  L.X = c.take<uint8_t>((size_t)(n_pad > 0 ? n_pad : BM) * K);
  L.partials = c.take<MatchPartial>(1024);
  L.best = c.take<MatchPartial>(1);
  L.status = c.take<unsigned int>(1);
  L.res = c.take<hamming_result>(1);
  L.bytes = c.bytes();
  return L;
}

}  // namespace

int set_fault_match(int on) {
  CPPGB_CUDA_TRY(cudaMemcpyToSymbol(g_fault_skip_tma, &on, sizeof on));
  return CPPGB_OK;
}
}  // namespace cppgb

using namespace cppgb;

extern "C" {

size_t twolocus_scan_tc_workspace_size(int64_t S, int64_t W) {
  if (S < 0 || W < 1) return 0;
  return tl_layout(nullptr, S, W).bytes;
}

int twolocus_scan_tc_shard(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                           int measure, int64_t shard, int64_t nshards, twolocus_result* out, void* ws, size_t ws_bytes,
                           void* stream) {
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (nshards < 1 || shard < 0 || shard >= nshards) return set_error(CPPGB_ERR_ARG, "need 0 <= shard < nshards");
  if (measure != CPPGB_TL_MATCHES && measure != CPPGB_TL_PEARSON) return set_error(CPPGB_ERR_ARG, "unknown measure");
  if (S < 0 || S > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "S out of range");
  if (m_cases < 1 || m_controls < 1) return set_error(CPPGB_ERR_ARG, "group sizes must be >= 1");
  if (W < (m_cases + 63) / 64 || W < (m_controls + 63) / 64 || W > 4096)
    return set_error(CPPGB_ERR_ARG, "W = %lld words cannot hold the groups (or exceeds 4096)", (long long)W);
  if (m_cases >= (1 << 20) || m_controls >= (1 << 20)) return set_error(CPPGB_ERR_ARG, "groups must hold < 2^20 subjects");
  if (S > 0 && !planes) return set_error(CPPGB_ERR_ARG, "planes is NULL");
  if (!ws || ((uintptr_t)ws & 255)) return set_error(CPPGB_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
  TLLayout L = tl_layout(ws, S, W);
  if (ws_bytes < L.bytes) return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu given, %zu needed", ws_bytes, L.bytes);
  if (!gram_tc_available()) return set_error(CPPGB_ERR_ARG, "tensor-core kernels are not available in this build");
  cudaStream_t st = (cudaStream_t)stream;
  if (S < 2) {
    memset(out, 0, sizeof *out);
    out->i = out->j = -1;
    out->score = -1;
    out->score_real = -1.0;
    return CPPGB_OK;
  }
  const int mode = measure == CPPGB_TL_PEARSON ? MATCH_TL_PEARSON : MATCH_TL_COUNT;
  const int64_t S_pad = (S + BM - 1) / BM * BM, K = 128 * W;
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(unsigned int), st));
  const int64_t warps = 2 * S_pad;
  tl_prep_kernel<<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(planes, S, S_pad, W, m_cases, m_controls, mode, L.L[0],
                                                             L.R[0], L.L[1], L.R[1], L.s[0], L.s[1], L.sx[0], L.sx[1],
                                                             L.vx[0], L.vx[1]);
  CPPGB_LAUNCH_CHECK();
  MatchMaps maps;
  int rc;
  for (int g = 0; g < 2; ++g) {
    if ((rc = encode_rows(&maps.L[g], L.L[g], S_pad, K))) return rc;
    if ((rc = encode_rows(&maps.R[g], L.R[g], S_pad, K))) return rc;
  }
  MatchParams mp;
  mp.S = S;
  mp.groups = 2;
  mp.mode = mode;
  mp.kch[0] = mp.kch[1] = K / BK;
  mp.t0 = shard;
  mp.tstride = nshards;
  mp.m[0] = m_cases;
  mp.m[1] = m_controls;
  for (int g = 0; g < 2; ++g) {
    mp.s[g] = L.s[g];
    mp.sx[g] = L.sx[g];
    mp.vx[g] = L.vx[g];
  }
  int64_t np = 0;
  if ((rc = launch_match(maps, mp, L.partials, &np, L.status, st))) return rc;
  if ((rc = launch_twolocus_finish(planes, W, m_cases, m_controls, L.partials, np, L.dres, st))) return rc;
  tl_tc_result_kernel<<<1, 1, 0, st>>>(L.dres, L.status, mode == MATCH_TL_PEARSON ? 1 : 0);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out, L.dres, sizeof *out, cudaMemcpyDeviceToHost, st));
  return CPPGB_OK;
}

int twolocus_scan_tc(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls, int measure,
                     twolocus_result* out, void* ws, size_t ws_bytes, void* stream) {
  return twolocus_scan_tc_shard(planes, S, W, m_cases, m_controls, measure, 0, 1, out, ws, ws_bytes, stream);
}

size_t hamming_pair_workspace_size(int64_t n, int64_t t, int sigma) {
  if (n < 0 || t < 1 || sigma < 2 || sigma > 256) return 0;
  const int64_t K = (t * sigma + BK - 1) / BK * BK;
  return ham_layout(nullptr, n, K).bytes;
}

int hamming_pair_shard(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, int64_t shard,
                       int64_t nshards, hamming_result* out, void* ws, size_t ws_bytes, void* stream) {
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (nshards < 1 || shard < 0 || shard >= nshards) return set_error(CPPGB_ERR_ARG, "need 0 <= shard < nshards");
  out->i = out->j = -1;
  out->mismatches = -1;
  out->status = CPPGB_OK;
  out->reserved = 0;
  if (n < 0 || n > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "n out of range");
  if (t < 1 || sigma < 2 || sigma > 256 || ld < t) return set_error(CPPGB_ERR_ARG, "need t >= 1, 2 <= sigma <= 256, ld >= t");
  if (t > (1 << 23)) return set_error(CPPGB_ERR_ARG, "strings longer than 2^23 symbols are not supported");
  const int64_t K = (t * sigma + BK - 1) / BK * BK;
  if (K > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "t * sigma too large");
  if (n > 0 && !strs) return set_error(CPPGB_ERR_ARG, "strings is NULL");
  if (!ws || ((uintptr_t)ws & 255)) return set_error(CPPGB_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
  HamLayout L = ham_layout(ws, n, K);
  if (ws_bytes < L.bytes) return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu given, %zu needed", ws_bytes, L.bytes);
  if (!gram_tc_available()) return set_error(CPPGB_ERR_ARG, "tensor-core kernels are not available in this build");
  if (n < 2) return CPPGB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n_pad = (n + BM - 1) / BM * BM;
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.X, 0, (size_t)n_pad * K, st));
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.status, 0, sizeof(unsigned int), st));
  ham_prep_kernel<<<(unsigned)((n + 7) / 8), 256, 0, st>>>(strs, n, t, ld, sigma, L.X, K, L.status);
  CPPGB_LAUNCH_CHECK();
  MatchMaps maps;
  int rc;
  if ((rc = encode_rows(&maps.L[0], L.X, n_pad, K))) return rc;
  maps.R[0] = maps.L[0];
  maps.L[1] = maps.R[1] = maps.L[0];
  MatchParams mp;
  memset(&mp, 0, sizeof mp);
  mp.S = n;
  mp.groups = 1;
  mp.mode = least ? MATCH_HAMMING_MAX : MATCH_HAMMING_MIN;
  mp.kch[0] = K / BK;
  mp.t0 = shard;
  mp.tstride = nshards;
  mp.m[0] = t;
  int64_t np = 0;
  if ((rc = launch_match(maps, mp, L.partials, &np, L.status, st))) return rc;
  match_finish_kernel<<<1, 256, 0, st>>>(L.partials, np, L.best);
  CPPGB_LAUNCH_CHECK();
  ham_result_kernel<<<1, 1, 0, st>>>(L.best, L.status, least ? 1 : 0, t, L.res);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out, L.res, sizeof *out, cudaMemcpyDeviceToHost, st));
  return CPPGB_OK;
}

int hamming_pair(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, hamming_result* out,
                 void* ws, size_t ws_bytes, void* stream) {
  return hamming_pair_shard(strs, n, t, ld, sigma, least, 0, 1, out, ws, ws_bytes, stream);
}

}  // extern "C"
