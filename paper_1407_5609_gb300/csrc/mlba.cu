// MLBA -- the modified light-bulb algorithm of Sec. 4 (closest pair of strings over an alphabet of
// sigma symbols) and its least correlated form over the one-hot strings and their complements
// (Sec. 5.4-5.5).  All iterations run at once:
//
//   pack     strings -> b-bit symbols in 64-bit words (b = ceil(log2 sigma)), symbol check
//   keys     per (iteration, row) the characters in that iteration's sampled columns, packed into
//            one 64-bit key; rows are the n strings, or the n one-hot strings followed by their n
//            complements (a sampled column c of the one-hot matrix is the bit [s_{c/sigma} = c%sigma],
//            flipped for a complement row)
//   sort     segmented LSD radix sort of (key, row), 8-bit digits, one segment per iteration;
//            stable, so within a bucket the originals precede the complements
//   runs     bucket starts (flags + exclusive scan), the split between originals and complements
//   pairs    per bucket the number of candidate pairs: len(len-1)/2, or originals x complements in
//            the buckets whose key has its last sampled bit 0 (a bucket K and its mirror ~K hold the
//            same unordered pairs, so one of the two is enough); exclusive scan -> pair offsets
//   verify   every candidate pair, load-balanced over the offsets: Hamming distance by XOR, an OR-fold
//            of each b-bit field and a popcount; per-block best, then one block reduces
//
// The work per iteration is O(m log sigma) for the keys and sort plus O(candidates) for the verification,
// instead of the n^2/2 pairs of the exact scan.
#include <mutex>

#include "common.cuh"

namespace cppgb {
namespace {

constexpr int RS_NT = 256, RS_PER = 8, RS_TILE = RS_NT * RS_PER, RS_WARPS = RS_NT / 32;
constexpr int RS_SCAN_NT = 1024;
constexpr int VF_NT = 256, VF_CH = 8;

struct MlbaBest {
  long long h, i, j;  // mismatches and the pair; i < 0 when empty
};

__device__ __forceinline__ bool mlba_better(int least, long long h, long long i, long long j, const MlbaBest& b) {
  if (i < 0) return false;
  if (b.i < 0) return true;
  if (h != b.h) return least ? h > b.h : h < b.h;
  return i < b.i || (i == b.i && j < b.j);
}

__device__ __forceinline__ MlbaBest mlba_pick(int least, const MlbaBest& a, const MlbaBest& b) {
  return mlba_better(least, b.h, b.i, b.j, a) ? b : a;
}

// ---- pack ------------------------------------------------------------------------------------------

// P[r][w]: symbols w*spw .. w*spw + spw - 1 of string r, symbol k at bits (k % spw) * b; the pad is 0.
__global__ void mlba_pack_kernel(const uint8_t* __restrict__ s, int64_t n, int64_t t, int64_t ld, int sigma, int b,
                                 int spw, int W, uint64_t* __restrict__ P, unsigned* __restrict__ status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * W) return;
  const int64_t r = e / W;
  const int w = (int)(e % W);
  const uint8_t* row = s + r * ld;
  uint64_t word = 0;
  bool bad = false;
  for (int k = 0; k < spw; ++k) {
    const int64_t c = (int64_t)w * spw + k;
    if (c >= t) break;
    const unsigned v = row[c];
    bad |= (int)v >= sigma;
    word |= (uint64_t)v << (k * b);
  }
  if (bad) atomicOr(status, 1u);
  P[e] = word;
}

__device__ __forceinline__ unsigned mlba_sym(const uint64_t* __restrict__ P, int W, int b, int spw, int64_t r, int64_t c) {
  const uint64_t word = P[r * W + c / spw];
  return (unsigned)(word >> ((c % spw) * b)) & ((1u << b) - 1u);
}

// ---- keys ------------------------------------------------------------------------------------------

__global__ void mlba_key_kernel(const uint64_t* __restrict__ P, int W, int b, int spw, int64_t n, int64_t m,
                                int sigma, int least, int64_t width, const int32_t* __restrict__ cols, int L,
                                int64_t E, uint64_t* __restrict__ keys, uint32_t* __restrict__ ids,
                                unsigned* __restrict__ status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int64_t it = e / m, r = e - it * m;
  const int32_t* cl = cols + it * L;
  uint64_t key = 0;
  bool bad = false;
  if (!least) {
    for (int k = 0; k < L; ++k) {
      const int64_t c = cl[k];
      if (c < 0 || c >= width) { bad = true; continue; }
      key |= (uint64_t)mlba_sym(P, W, b, spw, r, c) << (k * b);
    }
  } else {
    const int64_t i = r < n ? r : r - n;
    const uint64_t flip = r < n ? 0u : 1u;
    for (int k = 0; k < L; ++k) {
      const int64_t c = cl[k];
      if (c < 0 || c >= width) { bad = true; continue; }
      const uint64_t bit = mlba_sym(P, W, b, spw, i, c / sigma) == (unsigned)(c % sigma) ? 1u : 0u;
      key |= (bit ^ flip) << k;
    }
  }
  if (bad) atomicOr(status, 2u);
  keys[e] = key;
  ids[e] = (uint32_t)r;
}

// ---- segmented LSD radix sort ------------------------------------------------------------------------

// hist[(seg * 256 + digit) * bps + blk] = count of the digit in the block's tile
__global__ void __launch_bounds__(RS_NT) rs_hist_kernel(const uint64_t* __restrict__ keys, int64_t m, int bps,
                                                        int shift, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[256];
  const int blk = blockIdx.x, seg = blockIdx.y;
  h[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t* k = keys + (int64_t)seg * m;
  const int64_t base = (int64_t)blk * RS_TILE;
  for (int q = threadIdx.x; q < RS_TILE; q += RS_NT) {
    const int64_t p = base + q;
    if (p < m) atomicAdd(&h[(unsigned)(k[p] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[((int64_t)seg * 256 + threadIdx.x) * bps + blk] = h[threadIdx.x];
}

// exclusive scan of one segment's 256 * bps counts (digit-major), in place
__global__ void __launch_bounds__(RS_SCAN_NT) rs_scan_kernel(uint32_t* __restrict__ hist, int cnt) {
  __shared__ uint32_t wsum[32];
  uint32_t* h = hist + (int64_t)blockIdx.x * cnt;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  uint32_t carry = 0;
  for (int base = 0; base < cnt; base += RS_SCAN_NT * 4) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = base + tid * 4 + q;
      v[q] = idx < cnt ? h[idx] : 0u;
      s += v[q];
    }
    uint32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
      uint32_t z = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      wsum[lane] = z;
    }
    __syncthreads();
    uint32_t ex = x - s + (w > 0 ? wsum[w - 1] : 0u) + carry;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = base + tid * 4 + q;
      if (idx < cnt) h[idx] = ex;
      ex += v[q];
    }
    carry += wsum[31];
    __syncthreads();
  }
}

// Stable scatter of one tile.  Warp w owns tile positions [256 w, 256 w + 256), taken 32 at a time
// in order; __match_any_sync groups the lanes of a round by digit, and a per-warp digit count in
// shared memory carries the rank across rounds.  The per-digit counts are then scanned across warps.
__global__ void __launch_bounds__(RS_NT) rs_scatter_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ iin,
                                                           uint64_t* __restrict__ kout, uint32_t* __restrict__ iout,
                                                           int64_t m, int bps, int shift,
                                                           const uint32_t* __restrict__ hist) {
  __shared__ uint32_t wh[RS_WARPS][256];
  __shared__ uint32_t boff[256];
  const int blk = blockIdx.x, seg = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int q = 0; q < RS_WARPS; ++q) wh[q][tid] = 0;
  boff[tid] = hist[((int64_t)seg * 256 + tid) * bps + blk];
  __syncthreads();
  const int64_t sbase = (int64_t)seg * m;
  const int64_t base = (int64_t)blk * RS_TILE + w * (RS_TILE / RS_WARPS);
  const unsigned lt = (1u << lane) - 1u;
  uint64_t k[RS_PER];
  uint32_t id[RS_PER], rank[RS_PER];
  int dg[RS_PER];
#pragma unroll
  for (int r = 0; r < RS_PER; ++r) {
    const int64_t p = base + r * 32 + lane;
    const bool valid = p < m;
    k[r] = valid ? kin[sbase + p] : 0ull;
    id[r] = valid ? iin[sbase + p] : 0u;
    const int d = valid ? (int)((unsigned)(k[r] >> shift) & 255u) : 256;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? wh[w][d] : 0u;
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wh[w][d] = before + (uint32_t)__popc(peers);
    __syncwarp();
    rank[r] = before + (uint32_t)__popc(peers & lt);
    dg[r] = d;
  }
  __syncthreads();
  {
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < RS_WARPS; ++q) {
      const uint32_t c = wh[q][tid];
      wh[q][tid] = s;
      s += c;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RS_PER; ++r) {
    if (dg[r] < 256) {
      const int64_t dst = sbase + boff[dg[r]] + wh[w][dg[r]] + rank[r];
      kout[dst] = k[r];
      iout[dst] = id[r];
    }
  }
}

// ---- buckets ---------------------------------------------------------------------------------------

__global__ void mlba_flag_kernel(const uint64_t* __restrict__ keys, int64_t m, int64_t E, int32_t* __restrict__ flag) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  flag[e] = (e % m == 0 || keys[e] != keys[e - 1]) ? 1 : 0;
}

// rstart[run] = first element (rstart[R] = E); rsplit[run] = first complement row of the run, or -1
__global__ void mlba_runs_kernel(const int32_t* __restrict__ flag, const int64_t* __restrict__ rscan,
                                 const uint32_t* __restrict__ ids, int64_t n, int least, int64_t E,
                                 int64_t* __restrict__ rstart, int64_t* __restrict__ rsplit) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int f = flag[e];
  const int64_t run = rscan[e] + f - 1;
  if (f) rstart[run] = e;
  if (e == E - 1) rstart[run + 1] = E;
  if (least && ids[e] >= (uint32_t)n && (f || ids[e - 1] < (uint32_t)n)) rsplit[run] = e;
}

__global__ void mlba_run_pairs_kernel(const int64_t* __restrict__ rstart, const int64_t* __restrict__ rsplit,
                                      const int64_t* __restrict__ rscan, const uint64_t* __restrict__ keys, int least,
                                      int L, int64_t E, int64_t* __restrict__ rpairs) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= E) return;
  const int64_t R = rscan[E];
  int64_t c = 0;
  if (r < R) {
    const int64_t s = rstart[r], len = rstart[r + 1] - s;
    if (!least) {
      c = len * (len - 1) / 2;
    } else if (((keys[s] >> (L - 1)) & 1ull) == 0) {
      const int64_t sp = rsplit[r];
      const int64_t o = sp < 0 ? len : sp - s;
      c = o * (len - o);
    }
  }
  rpairs[r] = c;
}

// ---- verification ----------------------------------------------------------------------------------

__device__ __forceinline__ int64_t mlba_run_of(const int64_t* __restrict__ poff, int64_t E, int64_t g) {
  int64_t lo = 0, hi = E;  // poff[lo] <= g < poff[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (poff[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

// row x of the pair (x, y), x < y < len, enumerated row by row: the largest x with T(x) <= q,
// T(x) = x len - x (x + 1) / 2 pairs before row x
__device__ __forceinline__ int64_t mlba_tri_row(int64_t len, int64_t q) {
  int64_t lo = 0, hi = len - 1;  // T(lo) <= q < T(hi)
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (mid * len - mid * (mid + 1) / 2 <= q) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(VF_NT) mlba_verify_kernel(const uint64_t* __restrict__ P, int W, int b,
                                                            uint64_t lsb, const uint32_t* __restrict__ ids,
                                                            const int64_t* __restrict__ rstart,
                                                            const int64_t* __restrict__ rsplit,
                                                            const int64_t* __restrict__ poff, int64_t E, int least,
                                                            int64_t n, MlbaBest* __restrict__ partials) {
  __shared__ MlbaBest red[VF_NT / 32];
  const int64_t total = poff[E];
  MlbaBest best{-1, -1, -1};
  const int64_t stride = (int64_t)gridDim.x * VF_NT * VF_CH;
  for (int64_t g0 = ((int64_t)blockIdx.x * VF_NT + threadIdx.x) * VF_CH; g0 < total; g0 += stride) {
    const int64_t g1 = min(g0 + (int64_t)VF_CH, total);
    int64_t r = mlba_run_of(poff, E, g0);
    int64_t s = rstart[r], len = rstart[r + 1] - s, rend = poff[r + 1];
    int64_t o = 0, x, y;
    int64_t q = g0 - poff[r];
    if (!least) {
      x = mlba_tri_row(len, q);
      y = q - (x * len - x * (x + 1) / 2) + x + 1;
    } else {
      const int64_t sp = rsplit[r];
      o = sp < 0 ? len : sp - s;
      x = q / (len - o);
      y = q % (len - o);
    }
    for (int64_t g = g0; g < g1; ++g) {
      if (g == rend) {  // next non-empty bucket
        r = mlba_run_of(poff, E, g);
        s = rstart[r];
        len = rstart[r + 1] - s;
        rend = poff[r + 1];
        x = 0;
        if (!least) {
          y = 1;
        } else {
          const int64_t sp = rsplit[r];
          o = sp < 0 ? len : sp - s;
          y = 0;
        }
      }
      int64_t a, c;
      if (!least) {
        a = ids[s + x];
        c = ids[s + y];
        if (++y == len) { ++x; y = x + 1; }
      } else {
        a = ids[s + x];
        c = (int64_t)ids[s + o + y] - n;
        if (++y == len - o) { ++x; y = 0; }
      }
      const int64_t i = a < c ? a : c, j = a < c ? c : a;
      const uint64_t* pi = P + i * W;
      const uint64_t* pj = P + j * W;
      long long h = 0;
      for (int w = 0; w < W; ++w) {
        const uint64_t d = pi[w] ^ pj[w];
        uint64_t f = d;
        for (int sh = 1; sh < b; ++sh) f |= d >> sh;
        h += __popcll(f & lsb);
      }
      if (mlba_better(least, h, i, j, best)) best = MlbaBest{h, i, j};
    }
  }
  // block reduction
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    MlbaBest other{__shfl_down_sync(0xffffffffu, best.h, o), __shfl_down_sync(0xffffffffu, best.i, o),
                   __shfl_down_sync(0xffffffffu, best.j, o)};
    best = mlba_pick(least, best, other);
  }
  if (lane == 0) red[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    MlbaBest b0 = red[0];
    for (int q = 1; q < VF_NT / 32; ++q) b0 = mlba_pick(least, b0, red[q]);
    partials[blockIdx.x] = b0;
  }
}

struct MlbaOut {
  long long i, j, h, cand;
};

__global__ void mlba_finish_kernel(const MlbaBest* __restrict__ partials, int np, int least,
                                   const int64_t* __restrict__ poff, int64_t E, MlbaOut* __restrict__ out) {
  __shared__ MlbaBest red[32];
  MlbaBest best{-1, -1, -1};
  for (int q = threadIdx.x; q < np; q += blockDim.x) best = mlba_pick(least, best, partials[q]);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    MlbaBest other{__shfl_down_sync(0xffffffffu, best.h, o), __shfl_down_sync(0xffffffffu, best.i, o),
                   __shfl_down_sync(0xffffffffu, best.j, o)};
    best = mlba_pick(least, best, other);
  }
  if (lane == 0) red[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    MlbaBest b0 = red[0];
    for (int q = 1; q < (int)(blockDim.x / 32); ++q) b0 = mlba_pick(least, b0, red[q]);
    out->i = b0.i;
    out->j = b0.j;
    out->h = b0.i < 0 ? -1 : b0.h;
    out->cand = poff[E];
  }
}

// ---- host ------------------------------------------------------------------------------------------

int sym_bits(int sigma) {
  int b = 1;
  while ((1 << b) < sigma) ++b;
  return b;
}

// bit 0 of each of the spw b-bit fields
uint64_t lsb_mask(int b, int spw) {
  uint64_t m = 0;
  for (int k = 0; k < spw; ++k) m |= 1ull << (k * b);
  return m;
}

int verify_blocks() {
  static int nb = 0;
  if (!nb) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
      sms = 152;
    nb = sms * 4;
  }
  return nb;
}

constexpr int VF_MAX_BLOCKS = 4096;

// stage events: [pack + keys, radix sort, buckets + pair offsets, verification]
cudaEvent_t g_mev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
std::mutex g_mev_mu;

struct MlbaLayout {
  uint64_t* P;
  uint64_t* keys[2];
  uint32_t* ids[2];
  uint32_t* hist;
  int32_t* flag;
  int64_t *rscan, *rstart, *rsplit, *rpairs, *poff, *tmp;
  MlbaBest* partials;
  MlbaOut* out;
  unsigned* status;
  size_t bytes;
};

MlbaLayout mlba_layout(void* ws, int64_t n, int64_t t, int sigma, int least, int64_t iters) {
  MlbaLayout L;
  memset(&L, 0, sizeof L);
  const int b = sym_bits(sigma), spw = 64 / b;
  const int64_t W = (t + spw - 1) / spw;
  const int64_t m = least ? 2 * n : n, E = iters * m;
  const int64_t bps = (m + RS_TILE - 1) / RS_TILE;
  char* base = (char*)ws;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += (bytes + 255) / 256 * 256;
    return (void*)p;
  };
  L.P = (uint64_t*)take(sizeof(uint64_t) * (size_t)(n * W));
  L.keys[0] = (uint64_t*)take(sizeof(uint64_t) * (size_t)E);
  L.keys[1] = (uint64_t*)take(sizeof(uint64_t) * (size_t)E);
  L.ids[0] = (uint32_t*)take(sizeof(uint32_t) * (size_t)E);
  L.ids[1] = (uint32_t*)take(sizeof(uint32_t) * (size_t)E);
  L.hist = (uint32_t*)take(sizeof(uint32_t) * (size_t)(iters * 256 * bps));
  L.flag = (int32_t*)take(sizeof(int32_t) * (size_t)E);
  L.rscan = (int64_t*)take(sizeof(int64_t) * (size_t)(E + 1));
  L.rstart = (int64_t*)take(sizeof(int64_t) * (size_t)(E + 1));
  L.rsplit = (int64_t*)take(sizeof(int64_t) * (size_t)E);
  L.rpairs = (int64_t*)take(sizeof(int64_t) * (size_t)E);
  L.poff = (int64_t*)take(sizeof(int64_t) * (size_t)(E + 1));
  L.tmp = (int64_t*)take(sizeof(int64_t) * scan_temp_elems(E > 0 ? E : 1));
  L.partials = (MlbaBest*)take(sizeof(MlbaBest) * VF_MAX_BLOCKS);
  L.out = (MlbaOut*)take(sizeof(MlbaOut));
  L.status = (unsigned*)take(sizeof(unsigned));
  L.bytes = off;
  return L;
}

}  // namespace
}  // namespace cppgb

using namespace cppgb;

extern "C" {

size_t mlba_pair_workspace_size(int64_t n, int64_t t, int sigma, int least, int64_t iters) {
  if (n < 0 || t < 1 || sigma < 2 || sigma > 256 || iters < 0) return 0;
  return mlba_layout(nullptr, n, t, sigma, least ? 1 : 0, iters).bytes;
}

int mlba_pair(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, const int32_t* cols,
              int64_t iters, int64_t L, mlba_result* out, void* ws, size_t ws_bytes, void* stream) {
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  out->i = out->j = -1;
  out->mismatches = -1;
  out->candidates = 0;
  least = least ? 1 : 0;
  if (n < 0 || t < 1 || sigma < 2 || sigma > 256 || ld < t || iters < 0)
    return set_error(CPPGB_ERR_ARG, "need n >= 0, t >= 1, 2 <= sigma <= 256, ld >= t, iters >= 0");
  const int b = sym_bits(sigma), spw = 64 / b;
  if (L < (least ? 1 : 0) || (least ? L : L * b) > 64)
    return set_error(CPPGB_ERR_ARG, "the sampled characters must fit one 64-bit key: L <= %d (and L >= 1 for least)",
                     least ? 64 : 64 / b);
  const int64_t m = least ? 2 * n : n;
  if (m > 0x7fffffffLL || iters * m > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "iters x rows must be below 2^31");
  if (n > 0 && !strs) return set_error(CPPGB_ERR_ARG, "strings is NULL");
  if (iters > 0 && L > 0 && !cols) return set_error(CPPGB_ERR_ARG, "cols is NULL");
  if (!ws || ((uintptr_t)ws & 255)) return set_error(CPPGB_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
  MlbaLayout Lo = mlba_layout(ws, n, t, sigma, least, iters);
  if (ws_bytes < Lo.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu given, %zu needed", ws_bytes, Lo.bytes);
  if (n < 2 || iters == 0) return CPPGB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int W = (int)((t + spw - 1) / spw);
  const int64_t E = iters * m, width = least ? (int64_t)sigma * t : t;
  const int bps = (int)((m + RS_TILE - 1) / RS_TILE);
  bool timing = stage_timing_on();
  std::unique_lock<std::mutex> tlock(g_mev_mu, std::defer_lock);
  if (timing) {
    tlock.lock();
    if (!g_mev[0])
      for (auto& e : g_mev)
        if (cudaEventCreate(&e) != cudaSuccess) timing = false;
  }
  auto mark = [&](int k) -> int {
    if (timing) CPPGB_CUDA_TRY(cudaEventRecord(g_mev[k], st));
    return CPPGB_OK;
  };
  int rc;
  if ((rc = mark(0))) return rc;
  CPPGB_CUDA_TRY(cudaMemsetAsync(Lo.status, 0, sizeof(unsigned), st));
  mlba_pack_kernel<<<(unsigned)((n * W + 255) / 256), 256, 0, st>>>(strs, n, t, ld, sigma, b, spw, W, Lo.P, Lo.status);
  CPPGB_LAUNCH_CHECK();
  mlba_key_kernel<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(Lo.P, W, b, spw, n, m, sigma, least, width, cols,
                                                              (int)L, E, Lo.keys[0], Lo.ids[0], Lo.status);
  CPPGB_LAUNCH_CHECK();
  if ((rc = mark(1))) return rc;
  const int kbits = (int)(least ? L : L * b);
  const int passes = (kbits + 7) / 8;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const dim3 grid((unsigned)bps, (unsigned)iters);
    rs_hist_kernel<<<grid, RS_NT, 0, st>>>(Lo.keys[cur], m, bps, 8 * p, Lo.hist);
    CPPGB_LAUNCH_CHECK();
    rs_scan_kernel<<<(unsigned)iters, RS_SCAN_NT, 0, st>>>(Lo.hist, 256 * bps);
    CPPGB_LAUNCH_CHECK();
    rs_scatter_kernel<<<grid, RS_NT, 0, st>>>(Lo.keys[cur], Lo.ids[cur], Lo.keys[cur ^ 1], Lo.ids[cur ^ 1], m, bps,
                                              8 * p, Lo.hist);
    CPPGB_LAUNCH_CHECK();
    cur ^= 1;
  }
  if ((rc = mark(2))) return rc;
  const unsigned eb = (unsigned)((E + 255) / 256);
  mlba_flag_kernel<<<eb, 256, 0, st>>>(Lo.keys[cur], m, E, Lo.flag);
  CPPGB_LAUNCH_CHECK();
  if ((rc = launch_exclusive_scan_i32(Lo.flag, E, Lo.rscan, Lo.tmp, st))) return rc;
  if (least) CPPGB_CUDA_TRY(cudaMemsetAsync(Lo.rsplit, 0xff, sizeof(int64_t) * (size_t)E, st));
  mlba_runs_kernel<<<eb, 256, 0, st>>>(Lo.flag, Lo.rscan, Lo.ids[cur], n, least, E, Lo.rstart, Lo.rsplit);
  CPPGB_LAUNCH_CHECK();
  mlba_run_pairs_kernel<<<eb, 256, 0, st>>>(Lo.rstart, Lo.rsplit, Lo.rscan, Lo.keys[cur], least, (int)L, E, Lo.rpairs);
  CPPGB_LAUNCH_CHECK();
  if ((rc = launch_exclusive_scan_i64(Lo.rpairs, E, Lo.poff, Lo.tmp, st))) return rc;
  if ((rc = mark(3))) return rc;
  const int nb = verify_blocks() < VF_MAX_BLOCKS ? verify_blocks() : VF_MAX_BLOCKS;
  mlba_verify_kernel<<<(unsigned)nb, VF_NT, 0, st>>>(Lo.P, W, b, lsb_mask(b, spw), Lo.ids[cur], Lo.rstart, Lo.rsplit,
                                                     Lo.poff, E, least, n, Lo.partials);
  CPPGB_LAUNCH_CHECK();
  mlba_finish_kernel<<<1, 1024, 0, st>>>(Lo.partials, nb, least, Lo.poff, E, Lo.out);
  CPPGB_LAUNCH_CHECK();
  if ((rc = mark(4))) return rc;
  MlbaOut o;
  unsigned status = 0;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&o, Lo.out, sizeof o, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&status, Lo.status, sizeof status, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  if (timing) {
    double ms[4];
    for (int k = 0; k < 4; ++k) {
      float v = 0.f;
      CPPGB_CUDA_TRY(cudaEventElapsedTime(&v, g_mev[k], g_mev[k + 1]));
      ms[k] = v;
    }
    set_stage_times(ms, 4);
  }
  if (status & 1u) return set_error(CPPGB_ERR_ARG, "a symbol is >= sigma");
  if (status & 2u) return set_error(CPPGB_ERR_ARG, "a sampled column is out of range");
  out->i = o.i;
  out->j = o.j;
  out->mismatches = o.h;
  out->candidates = o.cand;
  return CPPGB_OK;
}

}  // extern "C"
