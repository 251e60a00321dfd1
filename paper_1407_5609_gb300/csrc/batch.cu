// Batched closest pair + fixed-radius pairs over many independent instances (the problems of
// Sec. 3 and Sec. 3.5, instance by instance), in one persistent launch.
//
// Every instance q (n_q points in R^{d_q}, radius R_q) gets the FP32 Gram tiles of the dense stage
// (128 x 128 tiles of its upper triangle).  The tile lists of all instances are concatenated; a
// persistent kernel walks them round-robin, so small and large instances share the machine and no
// per-instance launch is needed.  Each tile's epilogue uses its own instance's bound: pairs whose
// lower bound can be <= R_q are emitted (radius candidates); the tile minimum tightens the
// instance's upper bound U_q, and the tile itself is recorded when its minimum could still reach
// the bound published before it.  A second pass recomputes only the recorded tiles that can reach
// the final U_q and emits their closest-pair candidates.  A batched FP64 recheck then yields each
// instance's exact closest pair (lexicographic (d^2, i, j)) and its exact pair list
// { (i, j) : i < j, d <= R_q } (ascending).  The whole sequence is captured once into a CUDA graph
// per argument set and replayed.
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tile_simt.cuh"

namespace cppgb {
namespace {

struct BatchInst {
  const float* pts;  // caller's FP32 [n][d]
  int32_t n, d, Kp, has_r;
  int64_t x_off;     // floats before this instance's rows in the packed X
  int64_t row_off;   // rows before this instance (norms)
  int64_t tile_off;  // tiles before this instance
  double rr;         // R * R (FP64 decision value)
  float rr32;        // R^2 rounded up to FP32 (radius emission)
  float kappa;       // accumulation bound coefficient for Kp
};

struct BatchState {
  BoundParams bp;
  unsigned int U_bits, n2_bits, status, ferr_bits;
  unsigned long long best_bits, best_ij;
  int32_t n_rech, cursor;
  int64_t pad;
};

// candidate pair; the top bit of qk marks a closest-pair candidate (else a radius candidate)
struct BatchCand {
  int32_t qk, i, j;
  float d2f;
};
constexpr int32_t CPP_FLAG = (int32_t)0x80000000;

// a tile whose minimum may reach its instance's closest pair
struct TileRec {
  int32_t q, bi, bj;
  float tmin;
};

struct BatchGlobals {
  unsigned long long n_cand, n_trec;
  unsigned int status;
  unsigned int pad;
};

__device__ __forceinline__ int find_inst(const int64_t* __restrict__ offs, int count, int64_t v) {
  int lo = 0, hi = count - 1;  // largest q with offs[q] <= v
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (offs[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void batch_init_kernel(BatchState* st, int count, BatchGlobals* g) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q == 0) {
    g->n_cand = 0ull;
    g->n_trec = 0ull;
    g->status = 0u;
  }
  if (q >= count) return;
  BatchState s;
  s.bp.eps_pair = 0.f;
  s.bp.e_acc = 0.f;
  s.U_bits = 0x7f800000u;
  s.n2_bits = 0u;
  s.status = 0u;
  s.ferr_bits = 0u;
  s.best_bits = 0x7ff0000000000000ull;
  s.best_ij = ~0ull;
  s.n_rech = 0;
  s.cursor = 0;
  s.pad = 0;
  st[q] = s;
}

// one warp per padded row of every instance; rows located through row_off by binary search
__global__ void __launch_bounds__(256) batch_prep_kernel(const BatchInst* __restrict__ inst, const int64_t* __restrict__ row_offs,
                                                         int count, int64_t total_rows, float* __restrict__ X,
                                                         float* __restrict__ norms, BatchState* st, BatchGlobals* g) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= total_rows) return;
  const int q = find_inst(row_offs, count, r);
  const BatchInst in = inst[q];
  const int64_t lr = r - in.row_off;
  float* out = X + in.x_off + lr * in.Kp;
  float n2 = 0.f;
  bool bad = false;
  for (int k = lane; k < in.Kp; k += 32) {
    float v = 0.f;
    if (lr < in.n && k < in.d) {
      v = in.pts[lr * in.d + k];
      bad |= !isfinite(v);
    }
    out[k] = v;
    n2 = fmaf(v, v, n2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  bad = __any_sync(0xffffffffu, bad);
  if (lane == 0) {
    norms[r] = n2;
    atomic_max_nonneg(&st[q].n2_bits, n2 * (1.f + 0x1p-12f));
    if (bad) atomicOr(&g->status, 1u);
  }
}

__global__ void batch_bounds_kernel(const BatchInst* __restrict__ inst, BatchState* st, int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  st[q].bp.eps_pair = 0.f;  // FP32 input stored exactly
  st[q].bp.e_acc = inst[q].kappa * __uint_as_float(st[q].n2_bits) * (1.f + 0x1p-20f);
}

// Persistent FP32 tile kernel over the concatenated tile lists.
__global__ void __launch_bounds__(TILE_NT, 2)
    batch_dense_kernel(const BatchInst* __restrict__ inst, const int64_t* __restrict__ tile_offs, int count,
                       int64_t total_tiles, const float* __restrict__ X, const float* __restrict__ norms,
                       BatchState* st, BatchGlobals* g, BatchCand* __restrict__ cand, int64_t cap,
                       TileRec* __restrict__ trec, int64_t trec_cap) {
  __shared__ __align__(16) TileSmem sm;
  __shared__ float red[TILE_NT / 32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    const int q = find_inst(tile_offs, count, t);
    const BatchInst in = inst[q];
    int64_t bi, bj;
    tri_decode(t - in.tile_off, 0, &bi, &bj);
    const int64_t row0 = bi * TILE_BM, col0 = bj * TILE_BM;
    float acc[8][8];
    simt_tile_mainloop(X + in.x_off, in.Kp, row0, col0, sm, acc);

    const float* nr = norms + in.row_off;
    int64_t gi[8], gj[8];
    float nx[8], ny[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      gi[r] = row0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
      gj[r] = col0 + (r < 4 ? tx * 4 + r : 64 + tx * 4 + r - 4);
      nx[r] = nr[gi[r]];
      ny[r] = nr[gj[r]];
    }
    float tmin = __int_as_float(0x7f800000);
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const bool ok = gi[r] < in.n && gj[c] < in.n && gj[c] > gi[r];
        float D = fmaf(-2.f, acc[r][c], nx[r] + ny[c]);
        D = ok ? D : __int_as_float(0x7f800000);
        acc[r][c] = D;
        tmin = fminf(tmin, D);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
    if ((tid & 31) == 0) red[tid >> 5] = tmin;
    __syncthreads();
    tmin = red[0];
#pragma unroll
    for (int w = 1; w < TILE_NT / 32; ++w) tmin = fminf(tmin, red[w]);
    __syncthreads();  // red is reused by the next tile
    if (tmin == __int_as_float(0x7f800000)) continue;  // uniform: no valid pair in this tile

    const BoundParams bp = st[q].bp;
    const float ub = upper_d2(tmin, bp);
    const float Ug = __uint_as_float(*reinterpret_cast<volatile unsigned int*>(&st[q].U_bits));
    if (in.has_r) {
      const float th = theta_of(in.rr32, bp);
      if (tmin <= th) {
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if (acc[r][c] <= th) {
              const unsigned long long k = atomicAdd(&g->n_cand, 1ull);
              if ((int64_t)k < cap) {
                BatchCand cd;
                cd.qk = q;
                cd.i = (int32_t)gi[r];
                cd.j = (int32_t)gj[c];
                cd.d2f = acc[r][c];
                cand[k] = cd;
              }
            }
          }
      }
    }
    if (tid == 0) {
      // record the tile if its minimum can reach the bound published before it
      if (tmin <= theta_of(Ug, bp)) {
        const unsigned long long k = atomicAdd(&g->n_trec, 1ull);
        if ((int64_t)k < trec_cap) trec[k] = TileRec{q, (int32_t)bi, (int32_t)bj, tmin};
      }
      if (ub < Ug) atomic_min_nonneg(&st[q].U_bits, ub);
    }
  }
}

// Pass 2: recompute the recorded tiles that can still reach their instance's final bound and emit
// their closest-pair candidates (D~ <= theta(U_final)).
__global__ void __launch_bounds__(TILE_NT, 2)
    batch_tile_recheck_kernel(const BatchInst* __restrict__ inst, const float* __restrict__ X,
                              const float* __restrict__ norms, const BatchState* st, BatchGlobals* g,
                              const TileRec* __restrict__ trec, int64_t trec_cap, BatchCand* __restrict__ cand,
                              int64_t cap) {
  __shared__ __align__(16) TileSmem sm;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t nrec = (int64_t)g->n_trec < trec_cap ? (int64_t)g->n_trec : trec_cap;
  for (int64_t t = blockIdx.x; t < nrec; t += gridDim.x) {
    const TileRec tr = trec[t];
    const BoundParams bp = st[tr.q].bp;
    const float th = theta_of(__uint_as_float(st[tr.q].U_bits), bp);
    if (!(tr.tmin <= th)) continue;  // uniform across the block
    const BatchInst in = inst[tr.q];
    const int64_t row0 = (int64_t)tr.bi * TILE_BM, col0 = (int64_t)tr.bj * TILE_BM;
    float acc[8][8];
    simt_tile_mainloop(X + in.x_off, in.Kp, row0, col0, sm, acc);
    const float* nr = norms + in.row_off;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t i = row0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
      const float nx = nr[i];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t j = col0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4);
        const float D = fmaf(-2.f, acc[r][c], nx + nr[j]);
        if (i < in.n && j < in.n && j > i && D <= th) {
          const unsigned long long k = atomicAdd(&g->n_cand, 1ull);
          if ((int64_t)k < cap) {
            BatchCand cd;
            cd.qk = tr.q | CPP_FLAG;
            cd.i = (int32_t)i;
            cd.j = (int32_t)j;
            cd.d2f = D;
            cand[k] = cd;
          }
        }
      }
    }
  }
}

__device__ __forceinline__ double exact_d2(const float* __restrict__ p, int d, int32_t i, int32_t j) {
  const float* x = p + (int64_t)i * d;
  const float* y = p + (int64_t)j * d;
  double s = 0.0;
  for (int k = 0; k < d; ++k) {
    const double t = __dsub_rn((double)x[k], (double)y[k]);
    s = __dadd_rn(s, __dmul_rn(t, t));
  }
  return s;
}

// d2buf[c] = FP64 d^2 (or -1 when the candidate needs no recheck); keep[c] = 1: within R_q.
__global__ void batch_recheck_kernel(const BatchInst* __restrict__ inst, BatchState* st, const BatchGlobals* g,
                                     const BatchCand* __restrict__ cand, int64_t cap, double* __restrict__ d2buf,
                                     uint8_t* __restrict__ keep, int32_t* __restrict__ pair_counts) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t live = (int64_t)g->n_cand < cap ? (int64_t)g->n_cand : cap;
  if (c >= live) return;
  const BatchCand cd = cand[c];
  const int q = cd.qk & ~CPP_FLAG;
  const BatchInst in = inst[q];
  const BoundParams bp = st[q].bp;
  const bool cpp = (cd.qk & CPP_FLAG) && cd.d2f <= theta_of(__uint_as_float(st[q].U_bits), bp);
  const bool rad = !(cd.qk & CPP_FLAG);
  keep[c] = 0;
  d2buf[c] = -1.0;
  if (!cpp && !rad) return;
  const double s = exact_d2(in.pts, in.d, cd.i, cd.j);
  if (cpp) {
    d2buf[c] = s;
    atomicMin(&st[q].best_bits, (unsigned long long)__double_as_longlong(s));
    atomicAdd(&st[q].n_rech, 1);
    atomic_max_nonneg(&st[q].ferr_bits, (float)fabs(__dsub_rn(s, (double)cd.d2f)));
  }
  if (rad && s <= in.rr) {
    keep[c] = 1;
    atomicAdd(&pair_counts[q], 1);
  }
}

__global__ void batch_argmin_kernel(BatchState* st, const BatchGlobals* g, const BatchCand* __restrict__ cand,
                                    int64_t cap, const double* __restrict__ d2buf) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t live = (int64_t)g->n_cand < cap ? (int64_t)g->n_cand : cap;
  if (c >= live) return;
  const double s = d2buf[c];
  if (s < 0.0) return;
  const BatchCand cd = cand[c];
  const int q = cd.qk & ~CPP_FLAG;
  if ((unsigned long long)__double_as_longlong(s) == st[q].best_bits)
    atomicMin(&st[q].best_ij, ((unsigned long long)(uint32_t)cd.i << 32) | (uint32_t)cd.j);
}

__global__ void batch_fill_kernel(const BatchGlobals* g, const BatchCand* __restrict__ cand, int64_t cap,
                                  const uint8_t* __restrict__ keep, const int64_t* __restrict__ pair_offs,
                                  BatchState* st, int32_t* __restrict__ pairs, int64_t pairs_cap) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t live = (int64_t)g->n_cand < cap ? (int64_t)g->n_cand : cap;
  if (c >= live || !keep[c]) return;
  const BatchCand cd = cand[c];
  const int64_t pos = pair_offs[cd.qk] + atomicAdd(&st[cd.qk].cursor, 1);  // radius candidates only
  if (pos < pairs_cap) {
    pairs[2 * pos] = cd.i;
    pairs[2 * pos + 1] = cd.j;
  }
}

// one thread per instance: sort its (i, j) pairs ascending; write its result record
__global__ void batch_finish_kernel(const BatchState* st, int count, const int64_t* __restrict__ pair_offs,
                                    int32_t* __restrict__ pairs, int64_t pairs_cap, const BatchGlobals* g,
                                    cpp_pair_result* __restrict__ res) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const int64_t b = pair_offs[q], e = pair_offs[q + 1];
  if (e <= pairs_cap) {
    uint64_t* P = reinterpret_cast<uint64_t*>(pairs);  // (i, j) as one little-endian word: j high, i low
    for (int64_t u = b + 1; u < e; ++u) {             // insertion sort on (i, j)
      const int32_t vi = pairs[2 * u], vj = pairs[2 * u + 1];
      int64_t w = u - 1;
      while (w >= b && (pairs[2 * w] > vi || (pairs[2 * w] == vi && pairs[2 * w + 1] > vj))) {
        P[w + 1] = P[w];
        --w;
      }
      pairs[2 * (w + 1)] = vi;
      pairs[2 * (w + 1) + 1] = vj;
    }
  }
  const BatchState s = st[q];
  cpp_pair_result r;
  const double best = __longlong_as_double((long long)s.best_bits);
  if (s.best_ij == ~0ull || !(best < __longlong_as_double(0x7ff0000000000000ll))) {
    r.i = -1;
    r.j = -1;
    r.dist2 = __longlong_as_double(0x7ff0000000000000ll);
    r.dist = r.dist2;
  } else {
    r.i = (int64_t)(s.best_ij >> 32);
    r.j = (int64_t)(s.best_ij & 0xffffffffu);
    r.dist2 = best;
    r.dist = __dsqrt_rn(best);
  }
  r.filter_err = __uint_as_float(s.ferr_bits);
  r.filter_bound = __uint_as_float(s.U_bits);
  r.n_emitted = (int64_t)g->n_cand;
  r.n_rechecked = s.n_rech;
  res[q] = r;
}

// ---------------------------------------------------------------- host side
struct BatchLayout {
  BatchInst* inst;
  int64_t *row_offs, *tile_offs;
  BatchState* st;
  BatchGlobals* g;
  int32_t* pair_counts;
  int64_t* pair_offs;
  int64_t* tmp;
  float* X;
  float* norms;
  BatchCand* cand;
  double* d2buf;
  uint8_t* keep;
  TileRec* trec;
  cpp_pair_result* res;
  int64_t cap, trec_cap;
  size_t bytes;
};

struct Totals {
  int64_t rows = 0, xfloats = 0, tiles = 0;
};

Totals totals_of(const cpp_instance* inst, int64_t count) {
  Totals t;
  for (int64_t q = 0; q < count; ++q) {
    const int64_t n = inst[q].n, Kp = (inst[q].d + 15) / 16 * 16;
    const int64_t npad = (n + TILE_BM - 1) / TILE_BM * TILE_BM;
    const int64_t nb = npad / TILE_BM;
    t.rows += npad;
    t.xfloats += npad * Kp;
    t.tiles += n >= 2 ? nb * (nb + 1) / 2 : 0;
  }
  return t;
}

BatchLayout batch_layout(void* ws, int64_t count, const Totals& t, size_t ws_bytes) {
  BatchLayout L;
  Carver c(ws);
  L.inst = c.take<BatchInst>(count);
  L.row_offs = c.take<int64_t>(count + 1);
  L.tile_offs = c.take<int64_t>(count + 1);
  L.st = c.take<BatchState>(count);
  L.g = c.take<BatchGlobals>(1);
  L.pair_counts = c.take<int32_t>(count + 1);
  L.pair_offs = c.take<int64_t>(count + 1);
  L.tmp = c.take<int64_t>(scan_temp_elems(count + 1));
  L.res = c.take<cpp_pair_result>(count);
  L.X = c.take<float>(t.xfloats + 16);
  L.norms = c.take<float>(t.rows + 1);
  L.trec_cap = t.tiles > 0 ? t.tiles : 1;  // at most one record per tile
  L.trec = c.take<TileRec>(L.trec_cap);
  int64_t cap = t.rows / 4;
  cap = cap < (1 << 20) ? (1 << 20) : cap;
  const size_t fixed = c.bytes() + 512;
  const size_t per = sizeof(BatchCand) + sizeof(double) + 1;
  if (ws_bytes > fixed) {
    const int64_t fit = (int64_t)((ws_bytes - fixed) / per);
    if (fit > cap) cap = fit;
  }
  L.cap = cap;
  L.cand = c.take<BatchCand>(cap);
  L.d2buf = c.take<double>(cap);
  L.keep = c.take<uint8_t>(cap);
  L.bytes = c.bytes();
  return L;
}

float kappa_fp32(int64_t Kp) {
  const double K = (double)Kp, u = 0x1p-24, g = K * u / (1.0 - K * u);
  return (float)((4.0 * g + 8.0 * u) * 1.01);
}

// Graph cache: one instantiated graph per argument set (all kernel arguments are baked in).
struct GraphKey {
  void* ws;
  size_t ws_bytes;
  int64_t count, rows, tiles, cap;
  int32_t* pairs;
  int64_t pairs_cap;
  bool operator==(const GraphKey& o) const {
    return ws == o.ws && ws_bytes == o.ws_bytes && count == o.count && rows == o.rows && tiles == o.tiles &&
           cap == o.cap && pairs == o.pairs && pairs_cap == o.pairs_cap;
  }
};
std::mutex g_graph_mu;
GraphKey g_key{};
cudaGraphExec_t g_exec = nullptr;
int g_dev = -1;
long long g_graph_kernels = 0;  // kernels in the instantiated graph

int enqueue_batch(const BatchLayout& L, int64_t count, const Totals& t, int32_t* pairs, int64_t pairs_cap, int sms,
                  cudaStream_t st) {
  const int ci = (int)count;
  batch_init_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(L.st, ci, L.g);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.pair_counts, 0, sizeof(int32_t) * (count + 1), st));
  batch_prep_kernel<<<(unsigned)((t.rows + 7) / 8), 256, 0, st>>>(L.inst, L.row_offs, ci, t.rows, L.X, L.norms, L.st,
                                                                  L.g);
  CPPGB_LAUNCH_CHECK();
  batch_bounds_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(L.inst, L.st, ci);
  CPPGB_LAUNCH_CHECK();
  if (t.tiles > 0) {
    const int64_t grid = t.tiles < 2 * sms ? t.tiles : 2 * sms;
    batch_dense_kernel<<<(unsigned)grid, TILE_NT, 0, st>>>(L.inst, L.tile_offs, ci, t.tiles, L.X, L.norms, L.st, L.g,
                                                           L.cand, L.cap, L.trec, L.trec_cap);
    CPPGB_LAUNCH_CHECK();
    batch_tile_recheck_kernel<<<(unsigned)(2 * sms), TILE_NT, 0, st>>>(L.inst, L.X, L.norms, L.st, L.g, L.trec,
                                                                      L.trec_cap, L.cand, L.cap);
    CPPGB_LAUNCH_CHECK();
  }
  // candidate kernels are sized for the capacity and read the live count on the device
  const unsigned cb = (unsigned)((L.cap + 255) / 256);
  batch_recheck_kernel<<<cb, 256, 0, st>>>(L.inst, L.st, L.g, L.cand, L.cap, L.d2buf, L.keep, L.pair_counts);
  CPPGB_LAUNCH_CHECK();
  batch_argmin_kernel<<<cb, 256, 0, st>>>(L.st, L.g, L.cand, L.cap, L.d2buf);
  CPPGB_LAUNCH_CHECK();
  int rc = launch_exclusive_scan_i32(L.pair_counts, count, L.pair_offs, L.tmp, st);
  if (rc) return rc;
  batch_fill_kernel<<<cb, 256, 0, st>>>(L.g, L.cand, L.cap, L.keep, L.pair_offs, L.st, pairs, pairs_cap);
  CPPGB_LAUNCH_CHECK();
  batch_finish_kernel<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(L.st, ci, L.pair_offs, pairs, pairs_cap, L.g,
                                                                      L.res);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

}  // namespace
}  // namespace cppgb

using namespace cppgb;

extern "C" {

size_t cpp_batch_workspace_size(const cpp_instance* inst, int64_t count) {
  if (count < 0 || (count > 0 && !inst)) return 0;
  for (int64_t q = 0; q < count; ++q)
    if (inst[q].n < 0 || inst[q].d < 1 || inst[q].d > 256) return 0;
  return batch_layout(nullptr, count, totals_of(inst, count), 0).bytes;
}

int cpp_batch(const cpp_instance* inst, int64_t count, cpp_pair_result* out_cpp, int64_t* pair_counts, int32_t* pairs,
              int64_t pairs_cap, void* ws, size_t ws_bytes, void* stream) {
  if (count < 0 || count > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "count out of range");
  if (count == 0) return CPPGB_OK;
  if (!inst || !out_cpp || !pair_counts) return set_error(CPPGB_ERR_ARG, "inst, out_cpp and pair_counts are required");
  if (pairs_cap < 0 || (pairs_cap > 0 && !pairs)) return set_error(CPPGB_ERR_ARG, "bad pairs / pairs_cap");
  if (!ws || ((uintptr_t)ws & 255)) return set_error(CPPGB_ERR_ARG, "workspace must be non-NULL and 256-byte aligned");
  for (int64_t q = 0; q < count; ++q) {
    const cpp_instance& c = inst[q];
    if (c.n < 0 || c.n > (1 << 30)) return set_error(CPPGB_ERR_ARG, "instance %lld: n out of range", (long long)q);
    if (c.d < 1 || c.d > 256) return set_error(CPPGB_ERR_ARG, "instance %lld: d must be in [1, 256]", (long long)q);
    if (c.n > 0 && !c.pts) return set_error(CPPGB_ERR_ARG, "instance %lld: pts is NULL", (long long)q);
    if (!isfinite(c.R)) return set_error(CPPGB_ERR_ARG, "instance %lld: R must be finite", (long long)q);
  }
  const Totals t = totals_of(inst, count);
  const BatchLayout L = batch_layout(ws, count, t, ws_bytes);
  if (ws_bytes < L.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.bytes);
  cudaStream_t st = (cudaStream_t)stream;

  // instance table (host-built, copied before the graph runs)
  std::vector<BatchInst> hi((size_t)count);
  std::vector<int64_t> hro((size_t)count + 1), hto((size_t)count + 1);
  int64_t xo = 0, ro = 0, to = 0;
  for (int64_t q = 0; q < count; ++q) {
    const cpp_instance& c = inst[q];
    BatchInst b;
    b.pts = c.pts;
    b.n = (int32_t)c.n;
    b.d = c.d;
    b.Kp = (c.d + 15) / 16 * 16;
    b.has_r = c.R >= 0.0;
    b.x_off = xo;
    b.row_off = ro;
    b.tile_off = to;
    b.rr = c.R >= 0.0 ? c.R * c.R : -1.0;
    b.rr32 = c.R >= 0.0 ? (float)(c.R * c.R) * (1.f + 0x1p-20f) : 0.f;
    b.kappa = kappa_fp32(b.Kp);
    const int64_t npad = (c.n + TILE_BM - 1) / TILE_BM * TILE_BM, nb = npad / TILE_BM;
    hro[(size_t)q] = ro;
    hto[(size_t)q] = to;
    xo += npad * b.Kp;
    ro += npad;
    to += c.n >= 2 ? nb * (nb + 1) / 2 : 0;
    hi[(size_t)q] = b;
  }
  hro[(size_t)count] = ro;
  hto[(size_t)count] = to;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.inst, hi.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.row_offs, hro.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.tile_offs, hto.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));

  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    const GraphKey key{ws, ws_bytes, count, t.rows, t.tiles, L.cap, pairs, pairs_cap};
    if (!(g_exec && key == g_key && g_dev == dev)) {
      if (g_exec) {
        cudaGraphExecDestroy(g_exec);
        g_exec = nullptr;
      }
      cudaStream_t cap_st;
      CPPGB_CUDA_TRY(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
      cudaGraph_t graph;
      CPPGB_CUDA_TRY(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
      const long long before = (long long)cpp_launch_count();
      const int rc = enqueue_batch(L, count, t, pairs, pairs_cap, sms, cap_st);
      g_graph_kernels = (long long)cpp_launch_count() - before;
      note_launches(-g_graph_kernels);  // captured, not launched
      cudaError_t ce = cudaStreamEndCapture(cap_st, &graph);
      cudaStreamDestroy(cap_st);
      if (rc) return rc;
      if (ce != cudaSuccess) return set_error(CPPGB_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(ce));
      ce = cudaGraphInstantiate(&g_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        g_exec = nullptr;
        return set_error(CPPGB_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
      }
      g_key = key;
      g_dev = dev;
    }
    CPPGB_CUDA_TRY(cudaGraphLaunch(g_exec, st));
    note_launches(g_graph_kernels);
  }
  BatchGlobals hg;
  std::vector<int64_t> hoff((size_t)count + 1);
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out_cpp, L.res, sizeof(cpp_pair_result) * count, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(hoff.data(), L.pair_offs, sizeof(int64_t) * (count + 1), cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&hg, L.g, sizeof hg, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  for (int64_t q = 0; q < count; ++q) pair_counts[q] = hoff[(size_t)q + 1] - hoff[(size_t)q];
  if (hg.status & 1u) return set_error(CPPGB_ERR_NUMERIC, "non-finite coordinate");
  if ((int64_t)hg.n_cand > L.cap)
    return set_error(CPPGB_ERR_CAPACITY, "%llu candidate pairs exceed the workspace's %lld; pass %zu bytes",
                     (unsigned long long)hg.n_cand, (long long)L.cap,
                     L.bytes + (size_t)((int64_t)hg.n_cand - L.cap) * (sizeof(BatchCand) + sizeof(double) + 1) + 4096);
  if (hoff[(size_t)count] > pairs_cap)
    return set_error(CPPGB_ERR_CAPACITY, "pairs_cap %lld is smaller than the %lld pairs within R",
                     (long long)pairs_cap, (long long)hoff[(size_t)count]);
  return CPPGB_OK;
}

}  // extern "C"
