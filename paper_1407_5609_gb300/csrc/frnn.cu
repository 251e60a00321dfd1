// Fixed-radius near neighbours (Sec. 3.5): N(i) = { j != i : d(p_i, p_j) <= R } for every point,
// symmetric, as CSR with ascending columns.  The decision for a pair is the FP64 value of
// sum_k (x_ik - x_jk)^2 (coordinate order) compared with R*R.
//
// d <= 4: uniform grid with the floor function (the grid idea the paper cites in Sec. 1 for
//   constant dimension).  Cells have side s >= R (1 + delta), so every pair within R lies in the
//   same or adjacent cells; occupied cells live in an open-addressing hash table of 64-bit cell
//   keys; points are grouped by cell with a counting sort; one warp per occupied cell stages the
//   points of its 3^d neighbour cells in shared memory and tests the cell's points against them
//   twice (count, then fill).  A pair is decided in FP32 unless its FP32 squared distance lies
//   within a 2^-16 relative band of R^2, where the FP64 test decides.
// d > 4: the FP32 Gram tiles with a radius epilogue emit every pair whose lower bound can be <= R;
//   each emitted pair is decided by the FP64 test.
#include "common.cuh"

namespace cppgb {
namespace {

constexpr uint64_t EMPTY_KEY = ~0ull;

struct GridParams {
  float o[4];       // grid origin (bounding-box minimum)
  float inv_s;      // 1 / cell side
  int32_t d, bits;  // dimension, key bits per dimension
  int64_t lim;      // valid cell coordinates are [0, lim)
  double rr;        // R * R in FP64 (the decision value)
  float rr_lo, rr_hi;  // FP32 band around R^2: below -> inside, above -> outside, else FP64
  int32_t use64;    // 1: decide every pair in FP64
  int32_t pad;
  int64_t ncx;      // cells along x that hold points (slabs of a sharded query: see slab_table_kernel)
};

struct FrnnState {
  GridParams gp;
  unsigned int mm[8];   // ordered-float keys: min of dim k at [k], max at [4 + k]
  unsigned int status;  // 1: non-finite coordinate, 8: hash table full
  unsigned int spill;   // 1: the row buffer overflowed (the rows are then written by a second pass)
  unsigned long long cursor;  // entries of the row buffer handed out
  long long n_rows;           // points whose rows this call writes (its slab's, or all of them)
};

__device__ __forceinline__ unsigned int ord_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_val(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
// Slot of a cell key in a table of T = 2^tbits slots: the key folded to 32 bits, then Fibonacci
// hashing (multiply by 2^32 / golden ratio, keep the top tbits bits).
__device__ __forceinline__ uint64_t slot_hash(uint64_t key, int tbits) {
  const uint32_t f = (uint32_t)key ^ ((uint32_t)(key >> 32) * 0x85EBCA6Bu);
  return (uint64_t)((f * 0x9E3779B1u) >> (32 - tbits));
}

// A cell of the grid in the hash table: its 64-bit key, and (after the counting sort) its first
// position in the cell-sorted point arrays and its number of points; one 16-byte load per probe.
struct __align__(16) CellRec {
  unsigned long long key;
  int32_t start, cnt;
};

__global__ void frnn_init_kernel(FrnnState* fs, uint32_t* counters, int64_t n) {
  for (int k = 0; k < 4; ++k) {
    fs->mm[k] = 0xffffffffu;
    fs->mm[4 + k] = 0u;
  }
  fs->status = 0u;
  fs->spill = 0u;
  fs->cursor = 0ull;
  fs->n_rows = n;  // a sharded query's slab table sets its own count
  if (counters) counters[0] = counters[1] = 0u;
}

// Bounding box (ordered-float keys) and the non-finite flag: warp, then block reductions, then one
// atomic per block and bound.
__global__ void __launch_bounds__(256) bbox_kernel(const float* __restrict__ pts, int64_t n, int d, int64_t ld,
                                                   FrnnState* fs) {
  __shared__ unsigned int red[8][8];
  __shared__ int bad_any;
  unsigned int lo[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[4] = {0u, 0u, 0u, 0u};
  bool bad = false;
  if (threadIdx.x == 0) bad_any = 0;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < d; ++k) {
      const float x = pts[p * ld + k];
      bad |= !isfinite(x);
      const unsigned int key = ord_key(x);
      lo[k] = min(lo[k], key);
      hi[k] = max(hi[k], key);
    }
  }
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) {
    for (int k = 0; k < 4; ++k) {
      red[w][k] = lo[k];
      red[w][4 + k] = hi[k];
    }
    if (bad) atomicOr(&bad_any, 1);
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    const int k = threadIdx.x;
    unsigned int v = red[0][k];
    for (int q = 1; q < (int)(blockDim.x >> 5); ++q) v = k < 4 ? min(v, red[q][k]) : max(v, red[q][k]);
    if ((k & 3) < d) {
      if (k < 4) atomicMin(&fs->mm[k], v);
      else atomicMax(&fs->mm[k], v);
    }
    if (k == 0 && bad_any) atomicOr(&fs->status, 1u);
  }
}

// Cell side s = R (1 + delta) with delta >= 2^-10 and >= 16 u (extent / R): the FP32 cell
// coordinates (x - o) / s of two points within R then differ by at most 1 in every dimension.
// s is also raised so that every coordinate fits the key's bits.
__global__ void grid_params_kernel(FrnnState* fs, int d, double R) {
  GridParams gp;
  float ext = 0.f;
  for (int k = 0; k < 4; ++k) gp.o[k] = 0.f;
  for (int k = 0; k < d; ++k) {
    gp.o[k] = ord_val(fs->mm[k]);
    ext = fmaxf(ext, ord_val(fs->mm[4 + k]) - gp.o[k]);
  }
  gp.d = d;
  gp.bits = 63 / d < 21 ? 63 / d : 21;
  const float lim = (float)((1ll << gp.bits) - 4);
  const float Rf = (float)R;
  const float delta = fmaxf(0x1p-10f, Rf > 0.f ? 16.f * 0x1p-24f * (ext / Rf) : 0.f);
  float s = Rf * (1.f + delta);
  s = fmaxf(s, ext / lim * (1.f + 0x1p-10f));
  if (!(s > 0.f) || !isfinite(s)) s = 1.f;
  gp.inv_s = __frcp_rd(s * (1.f + 0x1p-20f));
  gp.lim = (1ll << gp.bits) - 1;
  gp.rr = __dmul_rn(R, R);
  const float rf = (float)gp.rr;
  gp.use64 = !(rf >= 1e-30f && rf <= 1e30f);
  gp.rr_lo = rf * (1.f - 0x1p-16f);
  gp.rr_hi = rf * (1.f + 0x1p-16f);
  gp.pad = 0;
  gp.ncx = (int64_t)floorf(__fmul_rn(__fsub_rn(ord_val(fs->mm[4]), gp.o[0]), gp.inv_s)) + 1;
  fs->gp = gp;
}

template <int D>
__device__ __forceinline__ void cell_of(const GridParams& gp, const float* x, int64_t* c) {
#pragma unroll
  for (int k = 0; k < D; ++k) c[k] = (int64_t)floorf(__fmul_rn(__fsub_rn(x[k], gp.o[k]), gp.inv_s));
}
template <int D>
__device__ __forceinline__ uint64_t key_of(const GridParams& gp, const int64_t* c) {
  uint64_t key = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) key |= (uint64_t)c[k] << (k * gp.bits);
  return key;
}

// Every point joins its cell's record (created on first sight) and takes a rank inside the cell;
// the threads that create cells append them (key and slot) to the list of occupied cells, one
// atomic per warp.
template <int D>
__global__ void __launch_bounds__(256) hash_insert_kernel(const float* __restrict__ pts, int64_t n, int64_t ld,
                                                          FrnnState* fs, CellRec* __restrict__ tab, int64_t T,
                                                          uint32_t* __restrict__ slot_of,
                                                          uint32_t* __restrict__ rank_of,
                                                          uint32_t* __restrict__ occ_slot,
                                                          unsigned long long* __restrict__ occ_key,
                                                          uint32_t* __restrict__ n_occ) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool valid = p < n;
  const GridParams gp = fs->gp;
  uint64_t key = 0;
  int64_t h = -1;
  bool created = false;
  if (valid) {
    float x[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < D; ++k) x[k] = pts[p * ld + k];
    int64_t c[4];
    cell_of<D>(gp, x, c);
    key = key_of<D>(gp, c);
    uint64_t g = slot_hash(key, __ffsll(T) - 1);
    for (int64_t probe = 0; probe < T; ++probe) {
      const unsigned long long prev = atomicCAS(&tab[g].key, EMPTY_KEY, key);
      if (prev == EMPTY_KEY || prev == key) {
        created = prev == EMPTY_KEY;
        h = (int64_t)g;
        break;
      }
      g = (g + 1) & (uint64_t)(T - 1);
    }
    if (h >= 0) {
      slot_of[p] = (uint32_t)h;
      rank_of[p] = (uint32_t)atomicAdd(&tab[h].cnt, 1);
    } else {
      atomicOr(&fs->status, 8u);
      slot_of[p] = 0xffffffffu;
    }
  }
  const uint32_t mask = __ballot_sync(0xffffffffu, created);
  if (mask) {
    uint32_t base = 0;
    if (lane == __ffs(mask) - 1) base = atomicAdd(n_occ, (uint32_t)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
    if (created) {
      const uint32_t idx = base + (uint32_t)__popc(mask & ((1u << lane) - 1u));
      occ_slot[idx] = (uint32_t)h;
      occ_key[idx] = key;
    }
  }
}

// occ_cnt[c] = points of occupied cell c (0 past the occupied cells), for the scan of cell starts
__global__ void occ_count_kernel(int64_t n, const uint32_t* __restrict__ occ_slot, const uint32_t* __restrict__ n_occ,
                                 const CellRec* __restrict__ tab, int32_t* __restrict__ occ_cnt) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) occ_cnt[c] = c < (int64_t)*n_occ ? tab[occ_slot[c]].cnt : 0;
}
__global__ void occ_start_kernel(int64_t n, const uint32_t* __restrict__ occ_slot, const uint32_t* __restrict__ n_occ,
                                 const int64_t* __restrict__ occ_start, CellRec* __restrict__ tab) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n && c < (int64_t)*n_occ) tab[occ_slot[c]].start = (int32_t)occ_start[c];
}

__global__ void scatter_kernel(const float* __restrict__ pts, int64_t n, int64_t ld, const FrnnState* fs,
                               const uint32_t* __restrict__ slot_of, const uint32_t* __restrict__ rank_of,
                               const CellRec* __restrict__ tab, int32_t* __restrict__ sorted_idx,
                               float4* __restrict__ sorted_pts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || slot_of[p] == 0xffffffffu) return;
  const int d = fs->gp.d;
  float x[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < d; ++k) x[k] = pts[p * ld + k];
  const int64_t pos = (int64_t)tab[slot_of[p]].start + rank_of[p];
  sorted_idx[pos] = (int32_t)p;
  sorted_pts[pos] = make_float4(x[0], x[1], x[2], x[3]);
}

// The FP64 test of Sec. 3.5's "d <= R", summed in coordinate order without contraction.
template <int D>
__device__ __forceinline__ bool within_fp64(const float* x, const float* y, double rr) {
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const double t = __dsub_rn((double)x[k], (double)y[k]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s <= rr;
}
// The record of the cell with this key: (start, cnt), cnt = 0 when the cell holds no point.
__device__ __forceinline__ int2 find_cell(const CellRec* __restrict__ tab, int64_t T, uint64_t key) {
  uint64_t h = slot_hash(key, __ffsll(T) - 1);
  for (int64_t probe = 0; probe < T; ++probe) {
    const CellRec r = tab[h];
    if (r.key == key) return make_int2(r.start, r.cnt);
    if (r.key == EMPTY_KEY) break;
    h = (h + 1) & (uint64_t)(T - 1);
  }
  return make_int2(0, 0);
}

// The FP64 test as a call of its own: FP64 runs at a small fraction of the FP32 rate here, so it
// must never be if-converted into the common path.
template <int D>
__device__ __noinline__ int within_fp64_call(float x0, float x1, float x2, float x3, float y0, float y1, float y2,
                                             float y3, double rr) {
  const float x[4] = {x0, x1, x2, x3}, y[4] = {y0, y1, y2, y3};
  return within_fp64<D>(x, y, rr) ? 1 : 0;
}

// Pair decision (called by all 32 lanes together): FP32 squared distance, with the FP64 test inside a
// 2^-16 relative band of R^2 (or always when R^2 is outside the FP32 range), entered only when some
// lane of the warp needs it.  x[D] and y[D] are the two points.
// The FP32 value has a relative error below 6 u (one rounding per difference, one per fused
// multiply-add), far inside the 2^-16 band, so every pair outside the band is decided as the FP64
// test would decide it.
template <int D>
__device__ __forceinline__ int decide(const float* x, const float* y, const GridParams& gp, bool live) {
  const float d0 = x[0] - y[0];
  float s = d0 * d0;
#pragma unroll
  for (int t = 1; t < D; ++t) {
    const float dv = x[t] - y[t];
    s = fmaf(dv, dv, s);
  }
  int in = s < gp.rr_lo ? 1 : 0;
  const bool band = live && (gp.use64 || (!(s < gp.rr_lo) && !(s > gp.rr_hi)));
  if (__any_sync(0xffffffffu, band)) {
    if (band)
      in = within_fp64_call<D>(x[0], D > 1 ? x[1] : 0.f, D > 2 ? x[2] : 0.f, D > 3 ? x[3] : 0.f, y[0],
                               D > 1 ? y[1] : 0.f, D > 2 ? y[2] : 0.f, D > 3 ? y[3] : 0.f, gp.rr);
  }
  return live ? in : 0;
}

// Lanes look up the 3^D neighbour cells of cell c (lane handles codes lane PER .. lane PER + PER - 1,
// code = sum_e (offset_e + 1) 3^e, so the offsets below increase with the code) and the warp lays
// their points out one after another: off[code] = position of the cell's first candidate, st[code]
// = its first sorted position, off[S] = the total, which is returned.
template <int D>
__device__ __forceinline__ int neighbour_layout(const GridParams& gp, uint64_t key, const int64_t* c,
                                                const CellRec* __restrict__ tab, int64_t T, int lane, int32_t* off,
                                                int32_t* st) {
  constexpr int S = D == 1 ? 3 : D == 2 ? 9 : D == 3 ? 27 : 81, PER = (S + 31) / 32;
  int2 rec[PER];
  int mine = 0;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int code = lane * PER + r;
    rec[r] = make_int2(0, 0);
    if (code < S) {
      // neighbour key = key + sum_e delta_e 2^(e bits): every field stays inside [0, lim)
      int rem = code;
      bool inside = true;
      int64_t koff = 0;
#pragma unroll
      for (int e = 0; e < D; ++e) {
        const int delta = rem % 3 - 1;
        rem /= 3;
        const int64_t ce = c[e] + delta;
        inside &= ce >= 0 && ce < gp.lim;
        koff += (int64_t)delta << (e * gp.bits);
      }
      if (inside) rec[r] = find_cell(tab, T, key + (uint64_t)koff);
    }
    mine += rec[r].y;
  }
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  int run = incl - mine;
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int code = lane * PER + r;
    if (code < S) {
      off[code] = run;
      st[code] = rec[r].x;
    }
    run += rec[r].y;
  }
  if (lane == 0) off[S] = total;
  __syncwarp();
  return total;
}

// Sorted position of the candidate at laid-out position t: the last cell whose offset is <= t.
template <int S>
__device__ __forceinline__ int64_t cand_pos(const int32_t* off, const int32_t* st, int t) {
  int lo = 0, hi = S;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= t) lo = mid;
    else hi = mid;
  }
  return (int64_t)st[lo] + (t - off[lo]);
}

__device__ void sort_segment(int32_t* a, int64_t m) {
  if (m <= 32) {
    for (int64_t u = 1; u < m; ++u) {
      const int32_t v = a[u];
      int64_t w = u - 1;
      while (w >= 0 && a[w] > v) {
        a[w + 1] = a[w];
        --w;
      }
      a[w + 1] = v;
    }
    return;
  }
  // heap sort for long rows
  auto sift = [&](int64_t root, int64_t end) {
    while (2 * root + 1 < end) {
      int64_t child = 2 * root + 1;
      if (child + 1 < end && a[child] < a[child + 1]) ++child;
      if (a[root] >= a[child]) return;
      const int32_t t = a[root];
      a[root] = a[child];
      a[child] = t;
      root = child;
    }
  };
  for (int64_t r = m / 2 - 1; r >= 0; --r) sift(r, m);
  for (int64_t e = m - 1; e > 0; --e) {
    const int32_t t = a[0];
    a[0] = a[e];
    a[e] = t;
    sift(0, e);
  }
}

// Slabs of a sharded query: the x cells [0, ncx) fall into SLAB_BINS bins of equal width; each bin
// goes to the slab in which its first point falls when the points are ranked by bin (slab s takes
// ranks [s n / nshards, (s + 1) n / nshards)), so the slabs hold equal numbers of points up to one
// bin's worth, whatever the distribution along x.  A slab is a range of whole bins, contiguous in x.
constexpr int SLAB_BINS = 4096;
__device__ __forceinline__ int slab_bin(const GridParams& gp, int64_t cx) {
  int64_t b = gp.ncx > 0 ? cx * SLAB_BINS / gp.ncx : 0;
  return (int)(b < 0 ? 0 : b >= SLAB_BINS ? SLAB_BINS - 1 : b);
}

// Points per slab bin: the occupied cells' counts (occ_cnt) added by the bin of their x cell, in
// shared memory first, then one global atomic per non-empty bin and block.
__global__ void __launch_bounds__(256) slab_hist_kernel(const FrnnState* fs, const unsigned long long* __restrict__ occ_key,
                                                        const int32_t* __restrict__ occ_cnt,
                                                        const uint32_t* __restrict__ n_occ, int32_t* __restrict__ hist) {
  __shared__ int32_t h[SLAB_BINS];
  for (int b = threadIdx.x; b < SLAB_BINS; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const GridParams gp = fs->gp;
  const uint64_t cmask = (1ull << gp.bits) - 1ull;
  const int64_t ncell = *n_occ;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[slab_bin(gp, (int64_t)(occ_key[c] & cmask))], occ_cnt[c]);
  __syncthreads();
  for (int b = threadIdx.x; b < SLAB_BINS; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// One block of 1024 threads: the exclusive scan of the bin counts, each bin's slab from the rank of
// its first point, and the number of points of this call's slab.
__global__ void __launch_bounds__(1024) slab_table_kernel(FrnnState* fs, const int32_t* __restrict__ hist,
                                                          int32_t* __restrict__ slab_tab, int64_t n, int shard,
                                                          int nshards) {
  constexpr int PER = SLAB_BINS / 1024;
  __shared__ int64_t wsum[32];
  __shared__ unsigned long long mine;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) mine = 0ull;
  int64_t v[PER], loc = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    v[k] = hist[t * PER + k];
    loc += v[k];
  }
  int64_t incl = loc;  // inclusive scan over the block
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[w] = incl;
  __syncthreads();
  if (w == 0) {
    int64_t x = wsum[lane], xi = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, xi, o);
      if (lane >= o) xi += y;
    }
    wsum[lane] = xi - x;  // exclusive prefix of the warps
  }
  __syncthreads();
  int64_t run = wsum[w] + incl - loc;  // points before this thread's first bin
  const int64_t total = n > 0 ? n : 1;
  unsigned long long cnt = 0ull;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    int64_t sl = run * nshards / total;
    sl = sl >= nshards ? nshards - 1 : sl;
    slab_tab[t * PER + k] = (int32_t)sl;
    if (sl == shard) cnt += (unsigned long long)v[k];
    run += v[k];
  }
  atomicAdd(&mine, cnt);
  __syncthreads();
  if (t == 0) fs->n_rows = (long long)mine;
}

// ------------------------------------------------------------------ cell-parallel query
// One warp per occupied cell: lanes look up the 3^D neighbour cells at once, the warp stages every
// candidate point of those cells in shared memory (copies of contiguous cell ranges), then takes
// the cell's points one after another: each lane tests one staged candidate and a ballot compacts
// the neighbours into a list whose entries each lane places by rank, so a row is written once,
// ascending.  The next cell's key is loaded one iteration ahead.  Cells with more candidates than
// the staging buffer holds are listed for the warp-per-point kernel below.
//
// ROWS pass (the query's only neighbour search when the row buffer suffices): every row goes to
// the row buffer at a position the warp takes from its current chunk (chunks of ROW_CHUNK entries
// come from one global cursor), and the point's count and position are recorded; past the buffer's
// capacity the row is dropped and the spill flag set.  FILL pass (only after a spill): every row
// goes straight to its place in the CSR, whose row pointers are then known.
constexpr int QW = 8;            // warps per block
constexpr int STAGE_CAP = 256;   // staged candidates per warp
constexpr int ROW_CHUNK = 1024;  // row-buffer entries a warp takes at a time
constexpr int ROWS_PER_POINT = 24;  // row-buffer capacity per point
static_assert(STAGE_CAP <= ROW_CHUNK, "a row must fit one chunk");

template <int D>
struct CellStage {
  static constexpr int S = D == 1 ? 3 : D == 2 ? 9 : D == 3 ? 27 : 81;
  static constexpr bool PACK = D <= 3;  // the point index rides in the unused fourth coordinate
  float4 p[STAGE_CAP];
  int32_t j[PACK ? 1 : STAGE_CAP];
  int32_t nb[STAGE_CAP];
  int32_t off[S + 1];
  int32_t st[S];
};

template <int D, bool FILL>
__global__ void __launch_bounds__(QW * 32) cell_query_kernel(
    FrnnState* fs, const CellRec* __restrict__ tab, int64_t T, const unsigned long long* __restrict__ occ_key,
    const uint32_t* __restrict__ n_occ, const int32_t* __restrict__ sorted_idx, const float4* __restrict__ sorted_pts,
    int32_t* __restrict__ counts, int64_t* __restrict__ row_at, int32_t* __restrict__ rowbuf, int64_t rowbuf_cap,
    const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cols, int64_t n, int64_t cols_cap,
    uint32_t* __restrict__ fb, uint32_t* __restrict__ n_fb, const int32_t* __restrict__ slab_tab, int shard,
    int nshards) {
  using Stage = CellStage<D>;
  constexpr int S = Stage::S, CENTER = (S - 1) / 2;
  extern __shared__ __align__(16) uint8_t cq_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Stage& sm = reinterpret_cast<Stage*>(cq_smem)[warp];
  if (FILL && (!fs->spill || row_ptr[n] > cols_cap)) return;  // no spill, or the host reports the capacity error
  const GridParams gp = fs->gp;
  const uint64_t cmask = (1ull << gp.bits) - 1ull;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t ncell = *n_occ;
  const int64_t stride = (int64_t)gridDim.x * QW;
  int64_t chunk = 0, chunk_left = 0;  // ROWS pass: the warp's free range of the row buffer
  int64_t ci = (int64_t)blockIdx.x * QW + warp;
  uint64_t key = ci < ncell ? occ_key[ci] : 0;
  for (; ci < ncell; ci += stride) {
    const uint64_t next = ci + stride < ncell ? occ_key[ci + stride] : 0;  // prefetch
    int64_t c[4];
#pragma unroll
    for (int e = 0; e < D; ++e) c[e] = (int64_t)((key >> (e * gp.bits)) & cmask);
    const int total = neighbour_layout<D>(gp, key, c, tab, T, lane, sm.off, sm.st);
    const int c0 = sm.off[CENTER], m = sm.off[CENTER + 1] - c0;  // the cell's own points
    if (nshards > 1 && slab_tab[slab_bin(gp, c[0])] != shard) {
      if (!FILL)
        for (int a = lane; a < m; a += 32) counts[sorted_idx[sm.st[CENTER] + a]] = 0;
    } else if (total > STAGE_CAP) {  // too many candidates for the staging buffer
      if (!FILL) {
        const uint32_t base = lane == 0 ? atomicAdd(n_fb, (uint32_t)m) : 0u;
        const uint32_t b = __shfl_sync(0xffffffffu, base, 0);
        for (int a = lane; a < m; a += 32) fb[b + a] = (uint32_t)(sm.st[CENTER] + a);
      }
    } else {
      for (int t = lane; t < total; t += 32) {
        const int64_t src = cand_pos<S>(sm.off, sm.st, t);
        float4 v = sorted_pts[src];
        const int32_t jj = sorted_idx[src];
        if (Stage::PACK) v.w = __int_as_float(jj);
        else sm.j[t] = jj;
        sm.p[t] = v;
      }
      __syncwarp();
      for (int a = 0; a < m; ++a) {
        const float4 xv = sm.p[c0 + a];
        const float x[4] = {xv.x, xv.y, xv.z, xv.w};
        const int32_t q = Stage::PACK ? __float_as_int(xv.w) : sm.j[c0 + a];
        int found = 0;
        for (int t0 = 0; t0 < total; t0 += 32) {
          const int t = t0 + lane;
          const bool live = t < total;
          const float4 yv = sm.p[live ? t : 0];
          const float y[4] = {yv.x, yv.y, yv.z, yv.w};
          const int32_t j = Stage::PACK ? __float_as_int(yv.w) : sm.j[live ? t : 0];
          const int in = decide<D>(x, y, gp, live && j != q);
          const uint32_t mask = __ballot_sync(0xffffffffu, in);
          if (in) sm.nb[found + __popc(mask & lt)] = j;
          found += __popc(mask);
        }
        __syncwarp();
        int32_t* out = nullptr;
        if (FILL) {
          out = cols + row_ptr[q];
        } else {
          // the row's place in the row buffer (warp-uniform: every lane keeps the same chunk)
          int64_t at = 0;
          if (found > 0) {
            if (found > chunk_left) {  // a fresh chunk (a row never exceeds STAGE_CAP <= ROW_CHUNK)
              unsigned long long base = 0;
              if (lane == 0) base = atomicAdd(&fs->cursor, (unsigned long long)ROW_CHUNK);
              chunk = (int64_t)__shfl_sync(0xffffffffu, base, 0);
              chunk_left = ROW_CHUNK;
            }
            at = chunk;
            chunk += found;
            chunk_left -= found;
          }
          if (lane == 0) {
            counts[q] = found;
            row_at[q] = at;
          }
          if (at + found <= rowbuf_cap) {
            out = rowbuf + at;
          } else if (lane == 0) {
            fs->spill = 1u;
          }
        }
        if (out) {
          for (int e = lane; e < found; e += 32) {  // rank among the row's (distinct) entries
            const int32_t v = sm.nb[e];
            int r = 0;
            for (int f = 0; f < found; ++f) r += sm.nb[f] < v ? 1 : 0;
            out[r] = v;
          }
        }
        __syncwarp();
      }
    }
    __syncwarp();
    key = next;
  }
}

// The rows of the row buffer copied to their places in the CSR, when nothing spilled and the CSR
// fits: each warp takes 32 consecutive points, whose rows are one contiguous range of cols, and its
// lanes walk that range 32 entries at a time (each entry's row found by a search over the 33 row
// pointers held one per lane).  Rows with row_at < 0 (points of crowded cells) are left to the
// crowded fill pass.
__global__ void __launch_bounds__(256) rows_copy_kernel(const FrnnState* fs, const int64_t* __restrict__ row_ptr,
                                                        const int64_t* __restrict__ row_at,
                                                        const int32_t* __restrict__ rowbuf, int32_t* __restrict__ cols,
                                                        int64_t n, int64_t cols_cap) {
  if (fs->spill || row_ptr[n] > cols_cap) return;
  const int lane = threadIdx.x & 31;
  const int64_t wpb = blockDim.x >> 5;
  for (int64_t q0 = ((int64_t)blockIdx.x * wpb + (threadIdx.x >> 5)) * 32; q0 < n; q0 += (int64_t)gridDim.x * wpb * 32) {
    const int64_t q = q0 + lane;
    const int64_t rp = row_ptr[q < n ? q : n];          // lanes past the last point hold row_ptr[n]
    const int64_t at = q < n ? row_at[q] : -1;
    const int64_t end = row_ptr[q0 + 32 < n ? q0 + 32 : n];
    const int64_t first = __shfl_sync(0xffffffffu, rp, 0);
    for (int64_t e0 = first; e0 < end; e0 += 32) {
      const int64_t e = e0 + lane;
      int r = 0;  // the last lane whose row starts at or before e
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int64_t v = __shfl_sync(0xffffffffu, rp, r + step);
        if (v <= e) r += step;
      }
      const int64_t src_at = __shfl_sync(0xffffffffu, at, r);
      const int64_t src_rp = __shfl_sync(0xffffffffu, rp, r);
      if (e < end && src_at >= 0) cols[e] = rowbuf[src_at + (e - src_rp)];
    }
  }
}

// One warp per point of a crowded cell (listed by the rows pass): the warp walks the laid-out
// candidates 32 at a time straight from global memory.  Count pass: counts[q], and row_at[q] = -1
// (the row is not in the row buffer).  Fill pass: the row is appended unordered, then sorted in
// place (rank placement through shared memory for rows of up to SORT_CAP entries, else a heap sort
// by one lane).
constexpr int PW = 4;          // warps per block
constexpr int SORT_CAP = 1024;

template <int D>
struct PointStage {
  static constexpr int S = D == 1 ? 3 : D == 2 ? 9 : D == 3 ? 27 : 81;
  int32_t off[S + 1];
  int32_t st[S];
  int32_t buf[SORT_CAP];
};

template <int D, bool FILL>
__global__ void __launch_bounds__(PW * 32) crowded_query_kernel(
    const FrnnState* fs, const CellRec* __restrict__ tab, int64_t T, const int32_t* __restrict__ sorted_idx,
    const float4* __restrict__ sorted_pts, int32_t* __restrict__ counts, int64_t* __restrict__ row_at,
    const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cols, int64_t n, int64_t cols_cap,
    const uint32_t* __restrict__ fb, const uint32_t* __restrict__ n_fb) {
  using Stage = PointStage<D>;
  constexpr int S = Stage::S;
  __shared__ Stage stage[PW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Stage& sm = stage[warp];
  if (FILL && row_ptr[n] > cols_cap) return;
  const GridParams gp = fs->gp;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t m = *n_fb;
  for (int64_t w = (int64_t)blockIdx.x * PW + warp; w < m; w += (int64_t)gridDim.x * PW) {
    const int64_t k = fb[w];
    const int32_t q = sorted_idx[k];
    const float4 xv = sorted_pts[k];
    const float x[4] = {xv.x, xv.y, xv.z, xv.w};
    int64_t c[4];
    cell_of<D>(gp, x, c);
    const int total = neighbour_layout<D>(gp, key_of<D>(gp, c), c, tab, T, lane, sm.off, sm.st);
    int32_t* out = FILL ? cols + row_ptr[q] : nullptr;
    int64_t found = 0;
    for (int t0 = 0; t0 < total; t0 += 32) {
      const int t = t0 + lane;
      const bool live = t < total;
      const int64_t src = live ? cand_pos<S>(sm.off, sm.st, t) : 0;
      const float4 yv = sorted_pts[src];
      const float y[4] = {yv.x, yv.y, yv.z, yv.w};
      const int32_t j = sorted_idx[src];
      const int in = decide<D>(x, y, gp, live && j != q);
      const uint32_t mask = __ballot_sync(0xffffffffu, in);
      if (FILL && in) out[found + __popc(mask & lt)] = j;
      found += __popc(mask);
    }
    if (!FILL) {
      if (lane == 0) {
        counts[q] = (int32_t)found;
        row_at[q] = -1;
      }
    } else if (found <= SORT_CAP) {
      __syncwarp();
      for (int e = lane; e < found; e += 32) sm.buf[e] = out[e];
      __syncwarp();
      for (int e = lane; e < found; e += 32) {
        const int32_t v = sm.buf[e];
        int r = 0;
        for (int f = 0; f < found; ++f) r += sm.buf[f] < v ? 1 : 0;
        out[r] = v;
      }
      __syncwarp();
    } else {
      __syncwarp();
      if (lane == 0) sort_segment(out, found);
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------- dense path (d > 4)
// The high-d path's candidates (grid-stride over the live count on the device): the FP64 test,
// then the rows, once the counts are scanned and only when every candidate was kept and the
// neighbour entries fit cols_cap.
__global__ void radius_check_kernel(const float* __restrict__ pts, int64_t d, int64_t ld, double rr,
                                    const DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                    uint8_t* __restrict__ keep, int32_t* __restrict__ counts) {
  const int64_t live = (int64_t)sc->n_cand < cap ? (int64_t)sc->n_cand : cap;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < live; c += (int64_t)gridDim.x * blockDim.x) {
    const Candidate cd = cand[c];
    const float* x = pts + (int64_t)cd.i * ld;
    const float* y = pts + (int64_t)cd.j * ld;
    double s = 0.0;
    for (int64_t k = 0; k < d; ++k) {
      const double t = __dsub_rn((double)x[k], (double)y[k]);
      s = __dadd_rn(s, __dmul_rn(t, t));
    }
    const bool in = s <= rr;
    keep[c] = in ? 1 : 0;
    if (in) {
      atomicAdd(&counts[cd.i], 1);
      atomicAdd(&counts[cd.j], 1);
    }
  }
}

__global__ void radius_fill_kernel(const DenseScalars* sc, const Candidate* __restrict__ cand, int64_t cap,
                                   const uint8_t* __restrict__ keep, const int64_t* __restrict__ row_ptr, int64_t n,
                                   int64_t cols_cap, int32_t* __restrict__ cursor, int32_t* __restrict__ cols) {
  if ((int64_t)sc->n_cand > cap || row_ptr[n] > cols_cap) return;
  const int64_t live = (int64_t)sc->n_cand;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < live; c += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[c]) continue;
    const Candidate cd = cand[c];
    cols[row_ptr[cd.i] + atomicAdd(&cursor[cd.i], 1)] = cd.j;
    cols[row_ptr[cd.j] + atomicAdd(&cursor[cd.j], 1)] = cd.i;
  }
}

__global__ void sort_rows_kernel(int64_t n, const int64_t* __restrict__ row_ptr, int64_t cols_cap,
                                 int32_t* __restrict__ cols) {
  if (row_ptr[n] > cols_cap) return;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) sort_segment(cols + row_ptr[r], row_ptr[r + 1] - row_ptr[r]);
}

// The query's result: the directed pair count and the status (grid path: fs, high-d path: sc).
__global__ void frnn_result_kernel(const FrnnState* fs, const DenseScalars* sc, int64_t cap,
                                   const int64_t* __restrict__ row_ptr, int64_t n, int64_t cols_cap,
                                   frnn_result* res) {
  frnn_result r;
  r.n_pairs = row_ptr[n];
  const long long rows = fs ? fs->n_rows : (long long)n;
  r.n_rows = (int32_t)(rows < 0x7fffffffLL ? rows : 0x7fffffffLL);
  const unsigned int st = fs ? fs->status : sc->status;
  r.status = (st & 1u) ? CPPGB_ERR_NUMERIC : (st & 8u) ? CPPGB_ERR_CUDA
             : ((sc && (int64_t)sc->n_cand > cap) || r.n_pairs > cols_cap) ? CPPGB_ERR_CAPACITY : CPPGB_OK;
  *res = r;
}

int64_t table_size(int64_t n) {
  int64_t T = 1024;
  while (T < 2 * n) T <<= 1;
  return T;
}

struct GridLayout {
  FrnnState* fs;
  CellRec* tab;        // hash table of the occupied cells
  uint32_t *slot_of, *rank_of;
  int32_t* sorted_idx;
  float4* sorted_pts;
  int32_t* counts;
  uint32_t* counters;  // [0] occupied cells, [1] points of crowded cells
  uint32_t *occ_slot, *fb;
  unsigned long long* occ_key;
  int32_t* occ_cnt;
  int64_t* occ_start;
  int64_t* tmp;
  int64_t* row_at;     // each point's row in the row buffer (-1: written by the crowded fill pass)
  int32_t* rowbuf;     // the rows pass's output, ROWS_PER_POINT entries per point
  int32_t *slab_hist, *slab_tab;  // sharded queries: points per slab bin, slab of each bin
  frnn_result* res;
  int64_t T, rowbuf_cap;
  size_t bytes;
};

GridLayout grid_layout(void* ws, int64_t n) {
  GridLayout L;
  Carver c(ws);
  L.T = table_size(n);
  L.fs = c.take<FrnnState>(1);
  L.tab = c.take<CellRec>(L.T);
  L.slot_of = c.take<uint32_t>(n);
  L.rank_of = c.take<uint32_t>(n);
  L.sorted_idx = c.take<int32_t>(n);
  L.sorted_pts = c.take<float4>(n);
  L.counts = c.take<int32_t>(n);
  L.counters = c.take<uint32_t>(2);
  L.occ_slot = c.take<uint32_t>(n);
  L.occ_key = c.take<unsigned long long>(n);
  L.fb = c.take<uint32_t>(n);
  L.occ_cnt = c.take<int32_t>(n);
  L.occ_start = c.take<int64_t>(n + 1);
  L.tmp = c.take<int64_t>(scan_temp_elems(n));
  L.row_at = c.take<int64_t>(n);
  L.rowbuf_cap = (int64_t)ROWS_PER_POINT * n;
  L.rowbuf = c.take<int32_t>(L.rowbuf_cap);
  L.slab_hist = c.take<int32_t>(SLAB_BINS);
  L.slab_tab = c.take<int32_t>(SLAB_BINS);
  L.res = c.take<frnn_result>(1);
  L.bytes = c.bytes();
  return L;
}

// Dense path layout: the closest-pair layout (rows, norms, eps, candidates) plus keep flags,
// counts/cursors and scan space.
struct RadiusLayout {
  DenseScalars* sc;
  float *norms, *eps;
  float* X;
  Candidate* cand;
  uint8_t* keep;
  int32_t* counts;
  int32_t* cursor;
  int64_t* tmp;
  frnn_result* res;
  int64_t n_pad, Kp, cap;
  size_t bytes;
};

RadiusLayout radius_layout(void* ws, int64_t n, int64_t d, size_t ws_bytes) {
  RadiusLayout L;
  L.n_pad = (n + 255) / 256 * 256;
  if (L.n_pad == 0) L.n_pad = 256;
  L.Kp = (d + 15) / 16 * 16;
  Carver c(ws);
  L.sc = c.take<DenseScalars>(1);
  L.norms = c.take<float>(L.n_pad);
  L.eps = c.take<float>(L.n_pad);
  L.X = c.take<float>((size_t)L.n_pad * L.Kp);
  L.counts = c.take<int32_t>(n + 1);
  L.cursor = c.take<int32_t>(n + 1);
  L.tmp = c.take<int64_t>(scan_temp_elems(n + 1));
  L.res = c.take<frnn_result>(1);
  int64_t cap = 16 * n;
  cap = cap < (1 << 16) ? (1 << 16) : cap;
  const size_t fixed = c.bytes() + 512;
  if (ws_bytes > fixed) {
    const int64_t fit = (int64_t)((ws_bytes - fixed) / (sizeof(Candidate) + 1));
    if (fit > cap) cap = fit;
  }
  L.cap = cap;
  L.cand = c.take<Candidate>(cap);
  L.keep = c.take<uint8_t>(cap);
  L.bytes = c.bytes();
  return L;
}

// Empty hash table: every key EMPTY_KEY, every count 0.
__global__ void tab_clear_kernel(CellRec* __restrict__ tab, int64_t T) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h < T) {
    CellRec r;
    r.key = EMPTY_KEY;
    r.start = 0;
    r.cnt = 0;
    tab[h] = r;
  }
}

template <int D>
int grid_path(const float* pts, int64_t n, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
              int64_t cols_cap, frnn_result* out, void* ws, size_t ws_bytes, cudaStream_t st, int shard = 0,
              int nshards = 1) {
  const int d = D;
  GridLayout L = grid_layout(ws, n);
  if (ws_bytes < L.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.bytes);
  if (n >= 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "the grid path needs n < 2^31 - 1");
  const unsigned nb = (unsigned)((n + 255) / 256);
  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  frnn_init_kernel<<<1, 1, 0, st>>>(L.fs, L.counters, n);
  CPPGB_LAUNCH_CHECK();
  tab_clear_kernel<<<(unsigned)((L.T + 255) / 256), 256, 0, st>>>(L.tab, L.T);
  CPPGB_LAUNCH_CHECK();
  bbox_kernel<<<nb < (unsigned)(2 * sms) ? nb : (unsigned)(2 * sms), 256, 0, st>>>(pts, n, d, ld, L.fs);
  CPPGB_LAUNCH_CHECK();
  grid_params_kernel<<<1, 1, 0, st>>>(L.fs, d, R);
  CPPGB_LAUNCH_CHECK();
  // the grid: cells hashed by key, points grouped by cell (counting sort over the occupied cells)
  hash_insert_kernel<D><<<nb, 256, 0, st>>>(pts, n, ld, L.fs, L.tab, L.T, L.slot_of, L.rank_of, L.occ_slot,
                                            L.occ_key, L.counters);
  CPPGB_LAUNCH_CHECK();
  occ_count_kernel<<<nb, 256, 0, st>>>(n, L.occ_slot, L.counters, L.tab, L.occ_cnt);
  CPPGB_LAUNCH_CHECK();
  if (nshards > 1) {  // slabs of equal point counts (slab_table_kernel)
    CPPGB_CUDA_TRY(cudaMemsetAsync(L.slab_hist, 0, sizeof(int32_t) * SLAB_BINS, st));
    slab_hist_kernel<<<nb < (unsigned)(2 * sms) ? nb : (unsigned)(2 * sms), 256, 0, st>>>(L.fs, L.occ_key, L.occ_cnt,
                                                                                         L.counters, L.slab_hist);
    CPPGB_LAUNCH_CHECK();
    slab_table_kernel<<<1, 1024, 0, st>>>(L.fs, L.slab_hist, L.slab_tab, n, shard, nshards);
    CPPGB_LAUNCH_CHECK();
  }
  int rc = launch_exclusive_scan_i32(L.occ_cnt, n, L.occ_start, L.tmp, st);
  if (rc) return rc;
  occ_start_kernel<<<nb, 256, 0, st>>>(n, L.occ_slot, L.counters, L.occ_start, L.tab);
  CPPGB_LAUNCH_CHECK();
  scatter_kernel<<<nb, 256, 0, st>>>(pts, n, ld, L.fs, L.slot_of, L.rank_of, L.tab, L.sorted_idx, L.sorted_pts);
  CPPGB_LAUNCH_CHECK();
  // rows pass (counts, rows into the row buffer), crowded counts, scan, copy of the buffered rows;
  // then the crowded cells' rows, and, only after a spill, the fill pass of every other row
  const size_t smem = (size_t)QW * sizeof(CellStage<D>);
  CPPGB_CUDA_TRY(cudaFuncSetAttribute(cell_query_kernel<D, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  CPPGB_CUDA_TRY(cudaFuncSetAttribute(cell_query_kernel<D, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  int per_sm = 0;
  CPPGB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_query_kernel<D, false>, QW * 32, smem));
  const unsigned cgrid = (unsigned)sms * (unsigned)(per_sm > 0 ? per_sm : 1), pgrid = (unsigned)sms * 4u;
  const uint32_t* n_occ = L.counters;
  uint32_t* n_fb = L.counters + 1;
  cell_query_kernel<D, false><<<cgrid, QW * 32, smem, st>>>(
      L.fs, L.tab, L.T, L.occ_key, n_occ, L.sorted_idx, L.sorted_pts, L.counts, L.row_at, L.rowbuf, L.rowbuf_cap,
      nullptr, nullptr, n, 0, L.fb, n_fb, L.slab_tab, shard, nshards);
  CPPGB_LAUNCH_CHECK();
  crowded_query_kernel<D, false><<<pgrid, PW * 32, 0, st>>>(L.fs, L.tab, L.T, L.sorted_idx, L.sorted_pts, L.counts,
                                                            L.row_at, nullptr, nullptr, n, 0, L.fb, n_fb);
  CPPGB_LAUNCH_CHECK();
  if ((rc = launch_exclusive_scan_i32(L.counts, n, row_ptr, L.tmp, st))) return rc;
  // the copy and fill kernels check row_ptr[n] <= cols_cap on the device and write nothing otherwise
  const int64_t copy_blocks = (n + 255) / 256;
  rows_copy_kernel<<<(unsigned)(copy_blocks < (int64_t)sms * 8 ? copy_blocks : (int64_t)sms * 8), 256, 0, st>>>(
      L.fs, row_ptr, L.row_at, L.rowbuf, cols, n, cols_cap);
  CPPGB_LAUNCH_CHECK();
  crowded_query_kernel<D, true><<<pgrid, PW * 32, 0, st>>>(L.fs, L.tab, L.T, L.sorted_idx, L.sorted_pts, nullptr,
                                                           nullptr, row_ptr, cols, n, cols_cap, L.fb, n_fb);
  CPPGB_LAUNCH_CHECK();
  cell_query_kernel<D, true><<<cgrid, QW * 32, smem, st>>>(
      L.fs, L.tab, L.T, L.occ_key, n_occ, L.sorted_idx, L.sorted_pts, nullptr, nullptr, nullptr, 0, row_ptr, cols,
      n, cols_cap, L.fb, n_fb, L.slab_tab, shard, nshards);
  CPPGB_LAUNCH_CHECK();
  frnn_result_kernel<<<1, 1, 0, st>>>(L.fs, nullptr, 0, row_ptr, n, cols_cap, L.res);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out, L.res, sizeof *out, cudaMemcpyDeviceToHost, st));
  return CPPGB_OK;
}

int dense_path(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
               int64_t cols_cap, frnn_result* out, void* ws, size_t ws_bytes, cudaStream_t st) {
  RadiusLayout L = radius_layout(ws, n, d, ws_bytes);
  if (ws_bytes < L.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.bytes);
  int rc;
  if ((rc = launch_init_scalars(L.sc, st))) return rc;
  if ((rc = launch_prep_points(pts, CPPGB_F32, n, d, ld, CPPGB_MODE_PLAIN_FP32, L.X, L.n_pad, L.Kp, L.norms, L.eps,
                               L.sc, st)))
    return rc;
  const double K = (double)L.Kp, u = 0x1p-24, g = K * u / (1.0 - K * u);
  if ((rc = launch_bounds(L.sc, (float)((4.0 * g + 8.0 * u) * 1.01), st))) return rc;
  const float rr32 = (float)(R * R) * (1.f + 0x1p-20f);
  if ((rc = launch_gram_simt_radius(L.X, n, L.Kp, L.norms, L.sc, L.cand, L.cap, rr32, st))) return rc;
  // every candidate's FP64 test, the row counts, their scan, the rows, then each row sorted
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.counts, 0, sizeof(int32_t) * (n + 1), st));
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.cursor, 0, sizeof(int32_t) * (n + 1), st));
  const int64_t cb = (L.cap + 255) / 256;
  const unsigned cgrid = (unsigned)(cb < 152 * 8 ? cb : 152 * 8);
  radius_check_kernel<<<cgrid, 256, 0, st>>>(pts, d, ld, R * R, L.sc, L.cand, L.cap, L.keep, L.counts);
  CPPGB_LAUNCH_CHECK();
  if ((rc = launch_exclusive_scan_i32(L.counts, n, row_ptr, L.tmp, st))) return rc;
  radius_fill_kernel<<<cgrid, 256, 0, st>>>(L.sc, L.cand, L.cap, L.keep, row_ptr, n, cols_cap, L.cursor, cols);
  CPPGB_LAUNCH_CHECK();
  sort_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, row_ptr, cols_cap, cols);
  CPPGB_LAUNCH_CHECK();
  frnn_result_kernel<<<1, 1, 0, st>>>(nullptr, L.sc, L.cap, row_ptr, n, cols_cap, L.res);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out, L.res, sizeof *out, cudaMemcpyDeviceToHost, st));
  return CPPGB_OK;
}

}  // namespace
}  // namespace cppgb

using namespace cppgb;

static int frnn_common(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
                int64_t cols_cap, frnn_result* out, void* ws, size_t ws_bytes, void* stream, int64_t shard,
                int64_t nshards) {
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  out->n_pairs = 0;
  out->status = CPPGB_OK;
  out->n_rows = 0;
  if (n < 0 || n > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "n out of range");
  if (d < 1 || d > 4096 || ld < d) return set_error(CPPGB_ERR_ARG, "need 1 <= d <= 4096 and ld >= d");
  if (!(R >= 0.0) || !isfinite(R)) return set_error(CPPGB_ERR_ARG, "R must be finite and >= 0");
  if (!row_ptr) return set_error(CPPGB_ERR_ARG, "row_ptr is NULL");
  if (cols_cap < 0 || (cols_cap > 0 && !cols)) return set_error(CPPGB_ERR_ARG, "bad cols / cols_cap");
  if (n > 0 && !pts) return set_error(CPPGB_ERR_ARG, "pts is NULL");
  if (!ws || ((uintptr_t)ws & 255)) return set_error(CPPGB_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  if (n == 0) {
    CPPGB_CUDA_TRY(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), st));
    return CPPGB_OK;
  }
  const int sh = (int)shard, ns = (int)nshards;
  switch (d) {
    case 1: return grid_path<1>(pts, n, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, st, sh, ns);
    case 2: return grid_path<2>(pts, n, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, st, sh, ns);
    case 3: return grid_path<3>(pts, n, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, st, sh, ns);
    case 4: return grid_path<4>(pts, n, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, st, sh, ns);
  }
  return dense_path(pts, n, d, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, st);
}

extern "C" {

size_t frnn_query_workspace_size(int64_t n, int d) {
  if (n < 0 || d < 1 || d > 4096) return 0;
  if (d <= 4) return grid_layout(nullptr, n).bytes;
  return radius_layout(nullptr, n, d, 0).bytes;
}


int frnn_query(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
               int64_t cols_cap, frnn_result* out, void* ws, size_t ws_bytes, void* stream) {
  return frnn_common(pts, n, d, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, stream, 0, 1);
}

int frnn_query_shard(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t shard, int64_t nshards,
                     int64_t* row_ptr, int32_t* cols, int64_t cols_cap, frnn_result* out, void* ws,
                     size_t ws_bytes, void* stream) {
  if (d < 1 || d > 4) return set_error(CPPGB_ERR_ARG, "frnn_query_shard needs 1 <= d <= 4 (the grid path)");
  if (nshards < 1 || nshards > 65536 || shard < 0 || shard >= nshards)
    return set_error(CPPGB_ERR_ARG, "need 0 <= shard < nshards <= 65536");
  return frnn_common(pts, n, d, ld, R, row_ptr, cols, cols_cap, out, ws, ws_bytes, stream, shard, nshards);
}

}  // extern "C"
