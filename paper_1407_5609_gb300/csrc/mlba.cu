// MLBA -- the modified light-bulb algorithm of Sec. 4 (closest pair of strings over an alphabet of
// sigma symbols) and its least correlated form over the one-hot strings and their complements
// (Sec. 5.4-5.5).  All iterations run at once, as one captured graph:
//
//   prep     strings -> b-bit symbols in 64-bit words (b = ceil(log2 sigma)), symbol check; each
//            sampled column -> (word, shift, symbol) so that no later step divides
//   keys     per (iteration, row) the characters in that iteration's sampled columns, packed into
//            one 64-bit key; rows are the n strings, or the n one-hot strings followed by their n
//            complements (a sampled column c of the one-hot matrix is the bit [s_{c/sigma} = c%sigma],
//            flipped for a complement row)
//   sort     segmented LSD radix sort of (key, row), 8-bit digits, one segment per iteration; stable,
//            so within a bucket the rows stay in ascending order and originals precede complements
//   buckets  at each bucket's first element: its end and its original/complement split by binary
//            search in the sorted segment, and its candidate pairs -- len(len-1)/2, or originals x
//            complements in the buckets whose key has its last sampled bit 0 (a bucket K and its
//            mirror ~K hold the same unordered pairs, so one of the two is enough)
//   verify   small buckets one thread each; the pairs of large buckets numbered by an exclusive scan
//            and dealt out evenly.  Hamming distance by XOR, an OR-fold of each b-bit field and a
//            popcount; per-block best, then one block reduces
//
// The work per iteration is O(m log sigma) for the keys and sort plus O(candidates) for the
// verification, instead of the n^2/2 pairs of the exact scan.
#include <mutex>

#include "common.cuh"

namespace cppgb {
namespace {

constexpr int RS_NT = 256, RS_PER = 8, RS_TILE = RS_NT * RS_PER, RS_WARPS = RS_NT / 32;
constexpr int RS_SCAN_NT = 1024;
constexpr int RS_FUSE_MAX_BPS = 64;  // up to this many tiles per segment, the scatter scans the counts itself
constexpr int VF_NT = 256, VF_CH = 8;
constexpr int64_t VF_SMALL = 64;     // buckets with at most this many pairs are verified by one thread each
constexpr int VF_MAX_BLOCKS = 4096;

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

// ---- prep ------------------------------------------------------------------------------------------

// P[r][w]: symbols w*spw .. w*spw + spw - 1 of string r, symbol k at bits (k % spw) * b; the pad is 0.
// desc[it][k]: (word << 16) | (shift << 8) | symbol of the k-th sampled column of iteration it (the
// symbol is the one a one-hot column tests; 0 for string columns).
__global__ void mlba_prep_kernel(const uint8_t* __restrict__ s, int64_t n, int64_t t, int64_t ld, int sigma, int b,
                                 int spw, int W, uint64_t* __restrict__ P, const int32_t* __restrict__ cols,
                                 int64_t ncols, int least, int64_t width, uint64_t* __restrict__ desc,
                                 unsigned* __restrict__ status) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n * W) {
    const int64_t r = e / W;
    const int w = (int)(e - r * W);
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
  if (e < ncols) {
    const int64_t c = cols[e];
    uint64_t d = 0;
    if (c < 0 || c >= width) {
      atomicOr(status, 2u);
    } else {
      const int64_t p = least ? c / sigma : c;
      const uint64_t v = least ? (uint64_t)(c - p * sigma) : 0u;
      d = ((uint64_t)(p / spw) << 16) | ((uint64_t)((p % spw) * b) << 8) | v;
    }
    desc[e] = d;
  }
}

// ---- keys ------------------------------------------------------------------------------------------

__global__ void mlba_key_kernel(const uint64_t* __restrict__ P, int W, int b, uint32_t n, uint32_t m, int least,
                                const uint64_t* __restrict__ desc, int L, uint32_t E, uint64_t* __restrict__ keys,
                                uint32_t* __restrict__ ids) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  const uint32_t it = e / m, r = e - it * m;
  const uint64_t* dl = desc + (size_t)it * L;
  const uint64_t mask = (1ull << b) - 1ull;
  uint64_t key = 0;
  if (!least) {
    const uint64_t* row = P + (size_t)r * W;
    for (int k = 0; k < L; ++k) {
      const uint64_t d = dl[k];
      key |= ((row[d >> 16] >> ((d >> 8) & 255u)) & mask) << (k * b);
    }
  } else {
    const uint64_t* row = P + (size_t)(r < n ? r : r - n) * W;
    const uint64_t flip = r < n ? 0u : 1u;
    for (int k = 0; k < L; ++k) {
      const uint64_t d = dl[k];
      const uint64_t bit = ((row[d >> 16] >> ((d >> 8) & 255u)) & mask) == (d & 255u) ? 1u : 0u;
      key |= (bit ^ flip) << k;
    }
  }
  keys[e] = key;
  ids[e] = r;
}

// ---- segmented LSD radix sort ------------------------------------------------------------------------

// Per tile, the count of each digit.  Layout: digit-major [seg][digit][tile] when a separate scan
// follows, tile-major [seg][tile][digit] when the scatter scans the counts itself (fused).
__global__ void __launch_bounds__(RS_NT) rs_hist_kernel(const uint64_t* __restrict__ keys, int64_t m, int bps,
                                                        int shift, int fused, uint32_t* __restrict__ hist) {
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
  const int64_t idx = fused ? ((int64_t)seg * bps + blk) * 256 + threadIdx.x
                            : ((int64_t)seg * 256 + threadIdx.x) * bps + blk;
  hist[idx] = h[threadIdx.x];
}

// exclusive scan of one segment's 256 * bps counts (digit-major), in place (the unfused path)
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

// Stable scatter of one tile.  The tile's output offset per digit comes either from the scanned
// counts (unfused) or from the raw counts of the segment's tiles: all tiles' totals of the smaller
// digits plus the earlier tiles' counts of this digit (fused).  Warp w owns tile positions
// [256 w, 256 w + 256), taken 32 at a time in order; __match_any_sync groups the lanes of a round by
// digit, and a per-warp digit count in shared memory carries the rank across rounds.  The per-digit
// counts are then scanned across warps.
__global__ void __launch_bounds__(RS_NT) rs_scatter_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ iin,
                                                           uint64_t* __restrict__ kout, uint32_t* __restrict__ iout,
                                                           int64_t m, int bps, int shift, int fused,
                                                           const uint32_t* __restrict__ hist) {
  __shared__ uint32_t wh[RS_WARPS][256];
  __shared__ uint32_t boff[256];
  __shared__ uint32_t dsum[RS_WARPS];
  const int blk = blockIdx.x, seg = blockIdx.y;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int q = 0; q < RS_WARPS; ++q) wh[q][tid] = 0;
  if (fused) {
    const uint32_t* hb = hist + (int64_t)seg * bps * 256 + tid;
    uint32_t before = 0, tot = 0;
    for (int q = 0; q < bps; ++q) {
      const uint32_t c = hb[(int64_t)q * 256];
      tot += c;
      before += q < blk ? c : 0u;
    }
    uint32_t x = tot;  // inclusive scan over the digits: within the warp, then across warps
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) dsum[w] = x;
    __syncthreads();
    uint32_t ex = x - tot;
    for (int q = 0; q < w; ++q) ex += dsum[q];
    boff[tid] = ex + before;
  } else {
    boff[tid] = hist[((int64_t)seg * 256 + tid) * bps + blk];
  }
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

// At a bucket's first element e: rlen[e] = its length, rsplit[e] = its originals (least = 1), and its
// candidate pairs; rpairs / bpairs (large buckets only) are 0 elsewhere; cand accumulates the total.
__global__ void mlba_bucket_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ids, uint32_t n,
                                   uint32_t m, uint32_t E, int least, int L, int32_t* __restrict__ rlen,
                                   int32_t* __restrict__ rsplit, int64_t* __restrict__ rpairs,
                                   int64_t* __restrict__ bpairs, unsigned long long* __restrict__ cand) {
  const uint32_t e = blockIdx.x * blockDim.x + threadIdx.x;
  int64_t c = 0;
  if (e < E) {
    const uint32_t seg = e / m, segend = (seg + 1) * m;
    const uint64_t K = keys[e];
    if (e == seg * m || keys[e - 1] != K) {
      uint32_t lo = e, hi = segend;  // keys[lo] == K; hi is past the bucket
      while (hi - lo > 1) {
        const uint32_t mid = lo + (hi - lo) / 2;
        if (keys[mid] == K) lo = mid;
        else hi = mid;
      }
      const int64_t len = hi - e;
      int64_t o = len;
      if (!least) {
        c = len * (len - 1) / 2;
      } else if (((K >> (L - 1)) & 1ull) == 0) {
        int64_t a = (int64_t)e - 1, z = hi;  // ids ascend in a bucket: the first complement row
        while (z - a > 1) {
          const int64_t mid = a + (z - a) / 2;
          if (ids[mid] >= n) z = mid;
          else a = mid;
        }
        o = z - e;
        c = o * (len - o);
      }
      rlen[e] = (int32_t)len;
      rsplit[e] = (int32_t)o;
    }
    rpairs[e] = c;
    bpairs[e] = c > VF_SMALL ? c : 0;
  }
  unsigned long long wsum = (unsigned long long)c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) wsum += __shfl_down_sync(0xffffffffu, wsum, o);
  if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(cand, wsum);
}

// ---- verification ----------------------------------------------------------------------------------

// the bucket (its first element) of large-bucket pair g: poff[lo] <= g < poff[lo + 1]
__device__ __forceinline__ int64_t mlba_run_of(const int64_t* __restrict__ poff, int64_t E, int64_t g) {
  int64_t lo = 0, hi = E;
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

// Hamming distance of strings a and c (packed), folded into the running best
__device__ __forceinline__ void mlba_eval(const uint64_t* __restrict__ P, int W, int b, uint64_t lsb, int least,
                                          int64_t a, int64_t c, MlbaBest& best) {
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

// Phase 1: every bucket with 1 .. VF_SMALL candidate pairs is enumerated by one thread.  Phase 2: the
// pairs of the larger buckets are numbered by the scan of their counts (boff) and dealt out VF_CH at
// a time; a thread finds its bucket by a binary search and walks on from there.
__global__ void __launch_bounds__(VF_NT) mlba_verify_kernel(const uint64_t* __restrict__ P, int W, int b,
                                                            uint64_t lsb, const uint32_t* __restrict__ ids,
                                                            const int32_t* __restrict__ rlen,
                                                            const int32_t* __restrict__ rsplit,
                                                            const int64_t* __restrict__ rpairs,
                                                            const int64_t* __restrict__ boff, int64_t E, int least,
                                                            int64_t n, MlbaBest* __restrict__ partials) {
  __shared__ MlbaBest red[VF_NT / 32];
  MlbaBest best{-1, -1, -1};
  const int64_t gtid = (int64_t)blockIdx.x * VF_NT + threadIdx.x, nthreads = (int64_t)gridDim.x * VF_NT;
  for (int64_t s = gtid; s < E; s += nthreads) {
    const int64_t c = rpairs[s];
    if (c == 0 || c > VF_SMALL) continue;
    const int64_t len = rlen[s];
    if (!least) {
      for (int64_t x = 0; x + 1 < len; ++x) {
        const int64_t a = ids[s + x];
        for (int64_t y = x + 1; y < len; ++y) mlba_eval(P, W, b, lsb, least, a, ids[s + y], best);
      }
    } else {
      const int64_t o = rsplit[s];
      for (int64_t x = 0; x < o; ++x) {
        const int64_t a = ids[s + x];
        for (int64_t y = o; y < len; ++y) mlba_eval(P, W, b, lsb, least, a, (int64_t)ids[s + y] - n, best);
      }
    }
  }
  const int64_t total = boff[E];
  for (int64_t g0 = gtid * VF_CH; g0 < total; g0 += nthreads * VF_CH) {
    const int64_t g1 = min(g0 + (int64_t)VF_CH, total);
    int64_t s = mlba_run_of(boff, E, g0);
    int64_t len = rlen[s], rend = boff[s + 1];
    int64_t o = 0, x, y;
    const int64_t q = g0 - boff[s];
    if (!least) {
      x = mlba_tri_row(len, q);
      y = q - (x * len - x * (x + 1) / 2) + x + 1;
    } else {
      o = rsplit[s];
      x = q / (len - o);
      y = q % (len - o);
    }
    for (int64_t g = g0; g < g1; ++g) {
      if (g == rend) {  // the next large bucket
        s = mlba_run_of(boff, E, g);
        len = rlen[s];
        rend = boff[s + 1];
        x = 0;
        y = least ? 0 : 1;
        if (least) o = rsplit[s];
      }
      if (!least) {
        mlba_eval(P, W, b, lsb, least, ids[s + x], ids[s + y], best);
        if (++y == len) { ++x; y = x + 1; }
      } else {
        mlba_eval(P, W, b, lsb, least, ids[s + x], (int64_t)ids[s + o + y] - n, best);
        if (++y == len - o) { ++x; y = 0; }
      }
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
                                   const unsigned long long* __restrict__ cand, MlbaOut* __restrict__ out) {
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
    out->cand = (long long)*cand;
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
    nb = sms * 4 < VF_MAX_BLOCKS ? sms * 4 : VF_MAX_BLOCKS;
  }
  return nb;
}

struct MlbaLayout {
  uint64_t* P;
  uint64_t* desc;
  uint64_t* keys[2];
  uint32_t* ids[2];
  uint32_t* hist;
  int32_t *rlen, *rsplit;
  int64_t *rpairs, *bpairs, *boff, *tmp;
  unsigned long long* cand;
  MlbaBest* partials;
  MlbaOut* out;
  unsigned* status;
  size_t bytes;
};

MlbaLayout mlba_layout(void* ws, int64_t n, int64_t t, int sigma, int least, int64_t iters, int64_t L) {
  MlbaLayout Lo;
  memset(&Lo, 0, sizeof Lo);
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
  Lo.P = (uint64_t*)take(sizeof(uint64_t) * (size_t)(n * W));
  Lo.desc = (uint64_t*)take(sizeof(uint64_t) * (size_t)(iters * L));
  Lo.keys[0] = (uint64_t*)take(sizeof(uint64_t) * (size_t)E);
  Lo.keys[1] = (uint64_t*)take(sizeof(uint64_t) * (size_t)E);
  Lo.ids[0] = (uint32_t*)take(sizeof(uint32_t) * (size_t)E);
  Lo.ids[1] = (uint32_t*)take(sizeof(uint32_t) * (size_t)E);
  Lo.hist = (uint32_t*)take(sizeof(uint32_t) * (size_t)(iters * 256 * bps));
  Lo.rlen = (int32_t*)take(sizeof(int32_t) * (size_t)E);
  Lo.rsplit = (int32_t*)take(sizeof(int32_t) * (size_t)E);
  Lo.rpairs = (int64_t*)take(sizeof(int64_t) * (size_t)E);
  Lo.bpairs = (int64_t*)take(sizeof(int64_t) * (size_t)E);
  Lo.boff = (int64_t*)take(sizeof(int64_t) * (size_t)(E + 1));
  Lo.cand = (unsigned long long*)take(sizeof(unsigned long long));
  Lo.tmp = (int64_t*)take(sizeof(int64_t) * scan_temp_elems(E > 0 ? E : 1));
  Lo.partials = (MlbaBest*)take(sizeof(MlbaBest) * VF_MAX_BLOCKS);
  Lo.out = (MlbaOut*)take(sizeof(MlbaOut));
  Lo.status = (unsigned*)take(sizeof(unsigned));
  Lo.bytes = off;
  return Lo;
}

struct MlbaArgs {
  const uint8_t* strs;
  int64_t n, t, ld;
  int sigma, least;
  const int32_t* cols;
  int64_t iters, L;
  void* ws;
  size_t ws_bytes;
  bool operator==(const MlbaArgs& o) const {
    return strs == o.strs && n == o.n && t == o.t && ld == o.ld && sigma == o.sigma && least == o.least &&
           cols == o.cols && iters == o.iters && L == o.L && ws == o.ws && ws_bytes == o.ws_bytes;
  }
};

// stage events: [prep + keys, radix sort, buckets + pair offsets, verification]
cudaEvent_t g_mev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

// Every kernel of one search, in stream order (captured into a graph by the caller).
int enqueue_mlba(const MlbaArgs& a, const MlbaLayout& Lo, bool timing, cudaStream_t st) {
  const int b = sym_bits(a.sigma), spw = 64 / b;
  const int W = (int)((a.t + spw - 1) / spw);
  const int64_t n = a.n, m = a.least ? 2 * n : n, E = a.iters * m, width = a.least ? (int64_t)a.sigma * a.t : a.t;
  const int bps = (int)((m + RS_TILE - 1) / RS_TILE);
  const int fused = bps <= RS_FUSE_MAX_BPS;
  auto mark = [&](int k) -> int {
    if (timing) CPPGB_CUDA_TRY(cudaEventRecordWithFlags(g_mev[k], st, cudaEventRecordExternal));
    return CPPGB_OK;
  };
  int rc;
  if ((rc = mark(0))) return rc;
  CPPGB_CUDA_TRY(cudaMemsetAsync(Lo.status, 0, sizeof(unsigned), st));
  CPPGB_CUDA_TRY(cudaMemsetAsync(Lo.cand, 0, sizeof(unsigned long long), st));
  const int64_t ncols = a.iters * a.L, prep = n * W > ncols ? n * W : ncols;
  mlba_prep_kernel<<<(unsigned)((prep + 255) / 256), 256, 0, st>>>(a.strs, n, a.t, a.ld, a.sigma, b, spw, W, Lo.P,
                                                                   a.cols, ncols, a.least, width, Lo.desc, Lo.status);
  CPPGB_LAUNCH_CHECK();
  mlba_key_kernel<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(Lo.P, W, b, (uint32_t)n, (uint32_t)m, a.least, Lo.desc,
                                                              (int)a.L, (uint32_t)E, Lo.keys[0], Lo.ids[0]);
  CPPGB_LAUNCH_CHECK();
  if ((rc = mark(1))) return rc;
  const int kbits = (int)(a.least ? a.L : a.L * b);
  const int passes = (kbits + 7) / 8;
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const dim3 grid((unsigned)bps, (unsigned)a.iters);
    rs_hist_kernel<<<grid, RS_NT, 0, st>>>(Lo.keys[cur], m, bps, 8 * p, fused, Lo.hist);
    CPPGB_LAUNCH_CHECK();
    if (!fused) {
      rs_scan_kernel<<<(unsigned)a.iters, RS_SCAN_NT, 0, st>>>(Lo.hist, 256 * bps);
      CPPGB_LAUNCH_CHECK();
    }
    rs_scatter_kernel<<<grid, RS_NT, 0, st>>>(Lo.keys[cur], Lo.ids[cur], Lo.keys[cur ^ 1], Lo.ids[cur ^ 1], m, bps,
                                              8 * p, fused, Lo.hist);
    CPPGB_LAUNCH_CHECK();
    cur ^= 1;
  }
  if ((rc = mark(2))) return rc;
  mlba_bucket_kernel<<<(unsigned)((E + 255) / 256), 256, 0, st>>>(Lo.keys[cur], Lo.ids[cur], (uint32_t)n,
                                                                 (uint32_t)m, (uint32_t)E, a.least, (int)a.L, Lo.rlen,
                                                                 Lo.rsplit, Lo.rpairs, Lo.bpairs, Lo.cand);
  CPPGB_LAUNCH_CHECK();
  if ((rc = launch_exclusive_scan_i64(Lo.bpairs, E, Lo.boff, Lo.tmp, st))) return rc;
  if ((rc = mark(3))) return rc;
  const int nb = verify_blocks();
  mlba_verify_kernel<<<(unsigned)nb, VF_NT, 0, st>>>(Lo.P, W, b, lsb_mask(b, spw), Lo.ids[cur], Lo.rlen, Lo.rsplit,
                                                     Lo.rpairs, Lo.boff, E, a.least, n, Lo.partials);
  CPPGB_LAUNCH_CHECK();
  mlba_finish_kernel<<<1, 1024, 0, st>>>(Lo.partials, nb, a.least, Lo.cand, Lo.out);
  CPPGB_LAUNCH_CHECK();
  return mark(4);
}

// Graph cache: one instantiated graph per argument set (all kernel arguments are baked in).
std::mutex g_mgraph_mu;
MlbaArgs g_mkey{};
bool g_mkey_timing = false;
cudaGraphExec_t g_mexec = nullptr;
int g_mdev = -1;
long long g_mgraph_kernels = 0;

}  // namespace
}  // namespace cppgb

using namespace cppgb;

extern "C" {

size_t mlba_pair_workspace_size(int64_t n, int64_t t, int sigma, int least, int64_t iters, int64_t L) {
  if (n < 0 || t < 1 || sigma < 2 || sigma > 256 || iters < 0 || L < 0) return 0;
  return mlba_layout(nullptr, n, t, sigma, least ? 1 : 0, iters, L).bytes;
}

int mlba_pair(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, const int32_t* cols,
              int64_t iters, int64_t L, mlba_result* out, void* ws, size_t ws_bytes, void* stream) {
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  out->i = out->j = -1;
  out->mismatches = -1;
  out->candidates = 0;
  out->status = CPPGB_OK;
  out->reserved = 0;
  least = least ? 1 : 0;
  if (n < 0 || t < 1 || sigma < 2 || sigma > 256 || ld < t || iters < 0)
    return set_error(CPPGB_ERR_ARG, "need n >= 0, t >= 1, 2 <= sigma <= 256, ld >= t, iters >= 0");
  const int b = sym_bits(sigma);
  if (L < (least ? 1 : 0) || (least ? L : L * b) > 64)
    return set_error(CPPGB_ERR_ARG, "the sampled characters must fit one 64-bit key: L <= %d (and L >= 1 for least)",
                     least ? 64 : 64 / b);
  const int64_t m = least ? 2 * n : n;
  if (m > 0x7fffffffLL || iters * m > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "iters x rows must be below 2^31");
  if (least && (int64_t)sigma * t > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "sigma * t must be below 2^31");
  if (n > 0 && !strs) return set_error(CPPGB_ERR_ARG, "strings is NULL");
  if (iters > 0 && L > 0 && !cols) return set_error(CPPGB_ERR_ARG, "cols is NULL");
  if (!ws || ((uintptr_t)ws & 255)) return set_error(CPPGB_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
  MlbaLayout Lo = mlba_layout(ws, n, t, sigma, least, iters, L);
  if (ws_bytes < Lo.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu given, %zu needed", ws_bytes, Lo.bytes);
  if (n < 2 || iters == 0) return CPPGB_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const MlbaArgs args{strs, n, t, ld, sigma, least, cols, iters, L, ws, ws_bytes};
  int dev = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_mgraph_mu);
  bool timing = stage_timing_on();
  if (timing && !g_mev[0])
    for (auto& e : g_mev)
      if (cudaEventCreate(&e) != cudaSuccess) timing = false;
  if (!(g_mexec && args == g_mkey && timing == g_mkey_timing && g_mdev == dev)) {
    if (g_mexec) {
      cudaGraphExecDestroy(g_mexec);
      g_mexec = nullptr;
    }
    cudaStream_t cap_st;
    CPPGB_CUDA_TRY(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    CPPGB_CUDA_TRY(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
    const long long before = (long long)cpp_launch_count();
    const int rc = enqueue_mlba(args, Lo, timing, cap_st);
    g_mgraph_kernels = (long long)cpp_launch_count() - before;
    note_launches(-g_mgraph_kernels);  // captured, not launched
    cudaError_t ce = cudaStreamEndCapture(cap_st, &graph);
    cudaStreamDestroy(cap_st);
    if (rc) {  // a failed enqueue: drop whatever the capture recorded
      if (ce == cudaSuccess && graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (ce != cudaSuccess) return set_error(CPPGB_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&g_mexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      g_mexec = nullptr;
      return set_error(CPPGB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
    }
    g_mkey = args;
    g_mkey_timing = timing;
    g_mdev = dev;
  }
  CPPGB_CUDA_TRY(cudaGraphLaunch(g_mexec, st));
  note_launches(g_mgraph_kernels);
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
  if (status & 3u) {
    out->status = CPPGB_ERR_ARG;
    return set_error(CPPGB_ERR_ARG, (status & 1u) ? "a symbol is >= sigma" : "a sampled column is out of range");
  }
  out->i = o.i;
  out->j = o.j;
  out->mismatches = o.h;
  out->candidates = o.cand;
  return CPPGB_OK;
}

}  // extern "C"
