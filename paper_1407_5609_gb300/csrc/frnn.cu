// Fixed-radius near neighbours (Sec. 3.5): N(i) = { j != i : d(p_i, p_j) <= R } for every point,
// symmetric, as CSR with ascending columns.  The decision for a pair is the FP64 value of
// sum_k (x_ik - x_jk)^2 (coordinate order) compared with R*R.
//
// d <= 4: uniform grid with the floor function (the grid idea the paper cites in Sec. 1 for
//   constant dimension).  Cells have side s >= R (1 + delta), so every pair within R lies in the
//   same or adjacent cells; occupied cells live in an open-addressing hash table of 64-bit cell
//   keys; points are grouped by cell with a counting sort; each point scans its 3^d neighbour cells
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
  int64_t ncx;      // cells along x that hold points (slabs of a sharded query split them evenly)
};

struct FrnnState {
  GridParams gp;
  unsigned int mm[8];   // ordered-float keys: min of dim k at [k], max at [4 + k]
  unsigned int status;  // 1: non-finite coordinate, 8: hash table full
  unsigned int pad;
};

__device__ __forceinline__ unsigned int ord_key(float f) {
  const unsigned int u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord_val(unsigned int k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}
__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

__global__ void frnn_init_kernel(FrnnState* fs) {
  for (int k = 0; k < 4; ++k) {
    fs->mm[k] = 0xffffffffu;
    fs->mm[4 + k] = 0u;
  }
  fs->status = 0u;
}

__global__ void bbox_kernel(const float* __restrict__ pts, int64_t n, int d, int64_t ld, FrnnState* fs) {
  unsigned int lo[4] = {0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[4] = {0u, 0u, 0u, 0u};
  bool bad = false;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < d; ++k) {
      const float x = pts[p * ld + k];
      bad |= !isfinite(x);
      const unsigned int key = ord_key(x);
      lo[k] = min(lo[k], key);
      hi[k] = max(hi[k], key);
    }
  }
  for (int k = 0; k < d; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
  }
  bad = __any_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0) {
    for (int k = 0; k < d; ++k) {
      atomicMin(&fs->mm[k], lo[k]);
      atomicMax(&fs->mm[4 + k], hi[k]);
    }
    if (bad) atomicOr(&fs->status, 1u);
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

template <int D>
__global__ void hash_insert_kernel(const float* __restrict__ pts, int64_t n, int64_t ld, FrnnState* fs,
                                   uint64_t* __restrict__ keys, int64_t T, uint32_t* __restrict__ slot_of,
                                   int32_t* __restrict__ cnt, uint32_t* __restrict__ rank_of) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const GridParams gp = fs->gp;
  float x[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < D; ++k) x[k] = pts[p * ld + k];
  int64_t c[4];
  cell_of<D>(gp, x, c);
  const uint64_t key = key_of<D>(gp, c);
  uint64_t h = mix64(key) & (uint64_t)(T - 1);
  for (int64_t probe = 0; probe < T; ++probe) {
    const unsigned long long prev = atomicCAS((unsigned long long*)&keys[h], EMPTY_KEY, key);
    if (prev == EMPTY_KEY || prev == key) {
      slot_of[p] = (uint32_t)h;
      rank_of[p] = (uint32_t)atomicAdd(&cnt[h], 1);
      return;
    }
    h = (h + 1) & (uint64_t)(T - 1);
  }
  atomicOr(&fs->status, 8u);
  slot_of[p] = 0xffffffffu;
}

__global__ void scatter_kernel(const float* __restrict__ pts, int64_t n, int64_t ld, const FrnnState* fs,
                               const uint32_t* __restrict__ slot_of, const uint32_t* __restrict__ rank_of,
                               const int64_t* __restrict__ start, int32_t* __restrict__ sorted_idx,
                               float4* __restrict__ sorted_pts) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || slot_of[p] == 0xffffffffu) return;
  const int d = fs->gp.d;
  float x[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k = 0; k < d; ++k) x[k] = pts[p * ld + k];
  const int64_t pos = start[slot_of[p]] + rank_of[p];
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
__device__ __forceinline__ int64_t find_slot(const uint64_t* __restrict__ keys, int64_t T, uint64_t key) {
  uint64_t h = mix64(key) & (uint64_t)(T - 1);
  for (int64_t probe = 0; probe < T; ++probe) {
    const uint64_t k = keys[h];
    if (k == key) return (int64_t)h;
    if (k == EMPTY_KEY) return -1;
    h = (h + 1) & (uint64_t)(T - 1);
  }
  return -1;
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

// FILL = false: counts[q] = |N(q)|.  FILL = true: writes N(q) at cols[row_ptr[q] ..], sorted.
// With nshards > 1 only the points of slab `shard` (x cells [shard, shard + 1) * ncx / nshards) are
// answered; the others get empty rows.  The grid holds every point, so no neighbour is missed.
// The neighbour loop uses 32-bit indices (n < 2^31) and a branch-free FP32 test with the FP64 test
// only inside the band: an earlier form with 64-bit indices and an early-return test produced wrong
// counts for a few warps whose lanes spanned several cells (nvcc 13.0, sm_103a); this form matches
// the oracle at 2^20 points.
template <int D, bool FILL>
__global__ void grid_query_kernel(int n, const FrnnState* fs, const uint64_t* __restrict__ keys, int64_t T,
                                  const int32_t* __restrict__ cnt, const int64_t* __restrict__ start,
                                  const int32_t* __restrict__ sorted_idx, const float4* __restrict__ sorted_pts,
                                  int32_t* __restrict__ counts, const int64_t* __restrict__ row_ptr,
                                  int32_t* __restrict__ cols, int shard, int nshards) {
  const int k = (int)(blockIdx.x * blockDim.x + threadIdx.x);
  if (k >= n) return;
  const GridParams gp = fs->gp;
  const int32_t q = sorted_idx[k];
  const float4 xv = sorted_pts[k];
  const float x[4] = {xv.x, xv.y, xv.z, xv.w};
  int64_t c[4];
  cell_of<D>(gp, x, c);
  if (nshards > 1) {
    int64_t slab = c[0] * nshards / gp.ncx;
    slab = slab < 0 ? 0 : slab >= nshards ? nshards - 1 : slab;
    if (slab != shard) {
      if (!FILL) counts[q] = 0;
      return;
    }
  }
  constexpr int stencil = D == 1 ? 3 : D == 2 ? 9 : D == 3 ? 27 : 81;
  int found = 0;
  int32_t* out = FILL ? cols + row_ptr[q] : nullptr;
  for (int code = 0; code < stencil; ++code) {
    int64_t cc[4];
    int rem = code;
    bool inside = true;
#pragma unroll
    for (int e = 0; e < D; ++e) {
      cc[e] = c[e] + (rem % 3) - 1;
      rem /= 3;
      inside &= cc[e] >= 0 && cc[e] < gp.lim;
    }
    if (!inside) continue;
    const int h = (int)find_slot(keys, T, key_of<D>(gp, cc));
    if (h < 0) continue;
    const int b = (int)start[h], e = b + cnt[h];
    for (int m = b; m < e; ++m) {
      const int32_t j = sorted_idx[m];
      const float4 yv = sorted_pts[m];
      const float y[4] = {yv.x, yv.y, yv.z, yv.w};
      float s = 0.f;
#pragma unroll
      for (int t = 0; t < D; ++t) {
        const float dv = __fsub_rn(x[t], y[t]);
        s = __fadd_rn(s, __fmul_rn(dv, dv));
      }
      int in = s < gp.rr_lo ? 1 : 0;
      if (gp.use64 || (!(s < gp.rr_lo) && !(s > gp.rr_hi))) in = within_fp64<D>(x, y, gp.rr) ? 1 : 0;
      in = (j != q) ? in : 0;
      if (FILL && in) out[found] = j;
      found += in;
    }
  }
  if (FILL)
    sort_segment(out, found);
  else
    counts[q] = found;
}

// ---------------------------------------------------------------- dense path (d > 4)
__global__ void radius_check_kernel(const float* __restrict__ pts, int64_t d, int64_t ld, double rr,
                                    const DenseScalars* sc, const Candidate* __restrict__ cand, int64_t n_live,
                                    float th_unused, uint8_t* __restrict__ keep, int32_t* __restrict__ counts) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_live) return;
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

__global__ void radius_fill_kernel(const Candidate* __restrict__ cand, int64_t n_live, const uint8_t* __restrict__ keep,
                                   const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cursor,
                                   int32_t* __restrict__ cols) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_live || !keep[c]) return;
  const Candidate cd = cand[c];
  cols[row_ptr[cd.i] + atomicAdd(&cursor[cd.i], 1)] = cd.j;
  cols[row_ptr[cd.j] + atomicAdd(&cursor[cd.j], 1)] = cd.i;
}

__global__ void sort_rows_kernel(int64_t n, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ cols) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) sort_segment(cols + row_ptr[r], row_ptr[r + 1] - row_ptr[r]);
}

int64_t table_size(int64_t n) {
  int64_t T = 1024;
  while (T < 2 * n) T <<= 1;
  return T;
}

struct GridLayout {
  FrnnState* fs;
  uint64_t* keys;
  int32_t* cnt;
  int64_t* start;
  uint32_t *slot_of, *rank_of;
  int32_t* sorted_idx;
  float4* sorted_pts;
  int32_t* counts;
  int64_t* tmp;
  int64_t T;
  size_t bytes;
};

GridLayout grid_layout(void* ws, int64_t n) {
  GridLayout L;
  Carver c(ws);
  L.T = table_size(n);
  L.fs = c.take<FrnnState>(1);
  L.keys = c.take<uint64_t>(L.T);
  L.cnt = c.take<int32_t>(L.T);
  L.start = c.take<int64_t>(L.T + 1);
  L.slot_of = c.take<uint32_t>(n);
  L.rank_of = c.take<uint32_t>(n);
  L.sorted_idx = c.take<int32_t>(n);
  L.sorted_pts = c.take<float4>(n);
  L.counts = c.take<int32_t>(n);
  L.tmp = c.take<int64_t>(scan_temp_elems(L.T > n ? L.T : n));
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
  int64_t* tmp;
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
  L.tmp = c.take<int64_t>(scan_temp_elems(n + 1));
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

template <int D>
int grid_path(const float* pts, int64_t n, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
              int64_t cols_cap, int64_t* n_pairs_out, void* ws, size_t ws_bytes, cudaStream_t st, int shard = 0,
              int nshards = 1) {
  const int d = D;
  GridLayout L = grid_layout(ws, n);
  if (ws_bytes < L.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.bytes);
  const unsigned nb = (unsigned)((n + 255) / 256);
  frnn_init_kernel<<<1, 1, 0, st>>>(L.fs);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.keys, 0xff, sizeof(uint64_t) * L.T, st));
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.cnt, 0, sizeof(int32_t) * L.T, st));
  bbox_kernel<<<nb < 1024u ? nb : 1024u, 256, 0, st>>>(pts, n, d, ld, L.fs);
  CPPGB_LAUNCH_CHECK();
  grid_params_kernel<<<1, 1, 0, st>>>(L.fs, d, R);
  CPPGB_LAUNCH_CHECK();
  hash_insert_kernel<D><<<nb, 256, 0, st>>>(pts, n, ld, L.fs, L.keys, L.T, L.slot_of, L.cnt, L.rank_of);
  CPPGB_LAUNCH_CHECK();
  int rc = launch_exclusive_scan_i32(L.cnt, L.T, L.start, L.tmp, st);
  if (rc) return rc;
  scatter_kernel<<<nb, 256, 0, st>>>(pts, n, ld, L.fs, L.slot_of, L.rank_of, L.start, L.sorted_idx, L.sorted_pts);
  CPPGB_LAUNCH_CHECK();
  const unsigned nq = (unsigned)((n + 127) / 128);
  grid_query_kernel<D, false><<<nq, 128, 0, st>>>((int)n, L.fs, L.keys, L.T, L.cnt, L.start, L.sorted_idx, L.sorted_pts,
                                                L.counts, nullptr, nullptr, shard, nshards);
  CPPGB_LAUNCH_CHECK();
  if ((rc = launch_exclusive_scan_i32(L.counts, n, row_ptr, L.tmp, st))) return rc;
  int64_t total = 0;
  unsigned int status = 0;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&total, row_ptr + n, sizeof total, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&status, &L.fs->status, sizeof status, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  if (status & 1u) return set_error(CPPGB_ERR_NUMERIC, "non-finite coordinate");
  if (status & 8u) return set_error(CPPGB_ERR_CUDA, "internal: cell hash table full");
  *n_pairs_out = total;
  if (total > cols_cap)
    return set_error(CPPGB_ERR_CAPACITY, "cols_cap %lld is smaller than the %lld neighbour entries",
                     (long long)cols_cap, (long long)total);
  if (total > 0) {
    grid_query_kernel<D, true><<<nq, 128, 0, st>>>((int)n, L.fs, L.keys, L.T, L.cnt, L.start, L.sorted_idx, L.sorted_pts,
                                                 nullptr, row_ptr, cols, shard, nshards);
    CPPGB_LAUNCH_CHECK();
  }
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  return CPPGB_OK;
}

int dense_path(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
               int64_t cols_cap, int64_t* n_pairs_out, void* ws, size_t ws_bytes, cudaStream_t st) {
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
  DenseScalars h;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&h, L.sc, sizeof h, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.status & 1u) return set_error(CPPGB_ERR_NUMERIC, "non-finite coordinate");
  if ((int64_t)h.n_cand > L.cap)
    return set_error(CPPGB_ERR_CAPACITY,
                     "%llu candidate pairs lie within the radius bound; pass a workspace of %zu bytes",
                     (unsigned long long)h.n_cand,
                     L.bytes + (size_t)((int64_t)h.n_cand - L.cap) * (sizeof(Candidate) + 1) + 4096);
  const int64_t n_live = (int64_t)h.n_cand;
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.counts, 0, sizeof(int32_t) * (n + 1), st));
  if (n_live > 0) {
    radius_check_kernel<<<(unsigned)((n_live + 255) / 256), 256, 0, st>>>(pts, d, ld, R * R, L.sc, L.cand,
                                                                           n_live, 0.f, L.keep, L.counts);
    CPPGB_LAUNCH_CHECK();
  }
  if ((rc = launch_exclusive_scan_i32(L.counts, n, row_ptr, L.tmp, st))) return rc;
  int64_t total = 0;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&total, row_ptr + n, sizeof total, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  *n_pairs_out = total;
  if (total > cols_cap)
    return set_error(CPPGB_ERR_CAPACITY, "cols_cap %lld is smaller than the %lld neighbour entries",
                     (long long)cols_cap, (long long)total);
  if (total > 0) {
    CPPGB_CUDA_TRY(cudaMemsetAsync(L.counts, 0, sizeof(int32_t) * (n + 1), st));
    radius_fill_kernel<<<(unsigned)((n_live + 255) / 256), 256, 0, st>>>(L.cand, n_live, L.keep, row_ptr, L.counts,
                                                                          cols);
    CPPGB_LAUNCH_CHECK();
    sort_rows_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, row_ptr, cols);
    CPPGB_LAUNCH_CHECK();
  }
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  return CPPGB_OK;
}

}  // namespace
}  // namespace cppgb

using namespace cppgb;

static int frnn_common(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
                int64_t cols_cap, int64_t* n_pairs_out, void* ws, size_t ws_bytes, void* stream, int64_t shard,
                int64_t nshards) {
  if (!n_pairs_out) return set_error(CPPGB_ERR_ARG, "n_pairs_out is NULL");
  *n_pairs_out = 0;
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
    CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
    return CPPGB_OK;
  }
  const int sh = (int)shard, ns = (int)nshards;
  switch (d) {
    case 1: return grid_path<1>(pts, n, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, st, sh, ns);
    case 2: return grid_path<2>(pts, n, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, st, sh, ns);
    case 3: return grid_path<3>(pts, n, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, st, sh, ns);
    case 4: return grid_path<4>(pts, n, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, st, sh, ns);
  }
  return dense_path(pts, n, d, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, st);
}

extern "C" {

size_t frnn_query_workspace_size(int64_t n, int d) {
  if (n < 0 || d < 1 || d > 4096) return 0;
  if (d <= 4) return grid_layout(nullptr, n).bytes;
  return radius_layout(nullptr, n, d, 0).bytes;
}


int frnn_query(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
               int64_t cols_cap, int64_t* n_pairs_out, void* ws, size_t ws_bytes, void* stream) {
  return frnn_common(pts, n, d, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, stream, 0, 1);
}

int frnn_query_shard(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t shard, int64_t nshards,
                     int64_t* row_ptr, int32_t* cols, int64_t cols_cap, int64_t* n_pairs_out, void* ws,
                     size_t ws_bytes, void* stream) {
  if (n_pairs_out) *n_pairs_out = 0;
  if (d < 1 || d > 4) return set_error(CPPGB_ERR_ARG, "frnn_query_shard needs 1 <= d <= 4 (the grid path)");
  if (nshards < 1 || nshards > 65536 || shard < 0 || shard >= nshards)
    return set_error(CPPGB_ERR_ARG, "need 0 <= shard < nshards <= 65536");
  return frnn_common(pts, n, d, ld, R, row_ptr, cols, cols_cap, n_pairs_out, ws, ws_bytes, stream, shard, nshards);
}

}  // extern "C"
