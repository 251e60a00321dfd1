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
//
// Each instance takes one of the tile paths (cpp_instance.path): FP32 CUDA-core tiles of 128 x 128,
// or BF16 tensor-core tiles of 128 x 256 (tcgen05 with TMA-staged operands, one tensor map per width
// class of d) whose accumulators are read by four epilogue groups (path 2) or two (path 3), two
// persistent kernels.  Every instance's rows are first shifted to a centre of its points.  Blocks
// recorded by any path are recomputed in FP32 by the same second pass.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "tile_simt.cuh"

namespace cppgb {
namespace {

struct BatchInst {
  const float* pts;  // caller's FP32 [n][d]
  int32_t n, d, Kp, has_r;
  int64_t x_off;     // floats before this instance's rows in the packed FP32 X
  int64_t c_off;     // columns before this instance in the bounding-box key arrays (Kp per instance)
  int64_t row_off;   // rows before this instance (FP32 norms)
  int64_t tile_off;  // FP32-path tiles before this instance
  double rr;         // R * R (FP64 decision value)
  float rr32;        // R^2 rounded up to FP32 (radius emission)
  float kappa;       // FP32 accumulation bound coefficient for Kp
  // tensor-core path
  int32_t tc, cls;        // tc = 1: BF16 tcgen05 tiles (epilogue of four or two groups: path 2 or 3); class of Kp16
  int32_t nbj16, nrow16;  // 256-column blocks; 128-row blocks that hold pairs
  int64_t row_off16;      // rows before this instance in its class matrix
  int64_t grow_off16;     // rows before this instance over all tensor-core instances (BF16 norms)
  int64_t tile_off16;     // tiles before this instance in its tensor-core kernel's tile list
  float kappa16;          // BF16 / tensor-core accumulation bound coefficient for Kp16
};

struct BatchState {
  BoundParams bp, bp16;
  unsigned int U_bits, n2_bits, status, ferr_bits;
  unsigned int n2_16_bits, eps16_bits;
  unsigned int eps32_bits;   // largest rounding distance of an FP32 row shifted to the centre
  unsigned int tmin16_bits;  // smallest recorded tensor-core tile minimum (clamped at 0)
  unsigned long long best_bits, best_ij;
  int32_t n_rech, cursor;
};

// Tensor-core classes by padded width Kp16 = 16, 32, 64, 128, 192, 256.  A tile's K runs in stages
// of `chunk` columns: one stage of 16, 32 or 64 columns (32-, 64- or 128-byte swizzle) up to
// Kp16 = 64, then stages of 64.
constexpr int NCLS = 6;
__host__ __device__ constexpr int cls_kp16(int c) { return c == 0 ? 16 : c == 1 ? 32 : 64 * (c - 1); }
__host__ __device__ constexpr int cls_chunk(int c) { return c == 0 ? 16 : c == 1 ? 32 : 64; }
__host__ __device__ constexpr int cls_nchunks(int c) { return c < 3 ? 1 : c - 1; }
inline int cls_of_d(int d) { return d <= 16 ? 0 : d <= 32 ? 1 : (d + 63) / 64 + 1; }
struct X16Set {
  __nv_bfloat16* p[NCLS];
};
struct BatchMaps {
  CUtensorMap m[NCLS];
  CUtensorMap h;  // [rows16][16] BF16: -|x~|^2 / 2 as three BF16 pieces, then zeros
};

// candidate pair; the top bit of qk marks a closest-pair candidate (else a radius candidate)
struct BatchCand {
  int32_t qk, i, j;
  float d2f;
};
constexpr int32_t CPP_FLAG = (int32_t)0x80000000;

// a 128 x 128 tile whose minimum may reach its instance's closest pair; the top bit of qf marks a
// minimum measured by the tensor-core path (its bound parameters apply)
struct TileRec {
  int32_t qf, bi, bj;
  float tmin;
};
constexpr int32_t TC_FLAG = (int32_t)0x80000000;

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
  s.bp16 = s.bp;
  s.n2_16_bits = 0u;
  s.eps16_bits = 0u;
  s.eps32_bits = 0u;
  s.tmin16_bits = 0x7f800000u;
  s.U_bits = 0x7f800000u;
  s.n2_bits = 0u;
  s.status = 0u;
  s.ferr_bits = 0u;
  s.best_bits = 0x7ff0000000000000ull;
  s.best_ij = ~0ull;
  s.n_rech = 0;
  s.cursor = 0;
  st[q] = s;
}

// Preparation kernels: each block takes rows of one instance only (blocks numbered per instance by
// a host-built offset table, so every row of a block has the same width), several rows per warp with
// each lane of a row's lane group handling 16 bytes of output; the row norms are summed in the lane
// group and the per-instance maxima flushed with one atomic per block.
constexpr int PREP_NT = 256;

// Lanes per row: a power of two that covers the row's 16-byte output chunks (at most 32).
__host__ __device__ constexpr int prep_lanes(int chunks) {
  return chunks <= 1 ? 1 : chunks <= 2 ? 2 : chunks <= 4 ? 4 : chunks <= 8 ? 8 : chunks <= 16 ? 16 : 32;
}
__host__ __device__ constexpr int prep_log2(int l) { return l >= 32 ? 5 : l >= 16 ? 4 : l >= 8 ? 3 : l >= 4 ? 2 : l >= 2 ? 1 : 0; }

// Loads columns c .. c + 3 of an input row (zeros past d).
__device__ __forceinline__ float4 load4(const float* __restrict__ row, int c, int d, bool vec) {
  if (vec && c + 3 < d) return *reinterpret_cast<const float4*>(row + c);
  float4 v;
  v.x = c < d ? row[c] : 0.f;
  v.y = c + 1 < d ? row[c + 1] : 0.f;
  v.z = c + 2 < d ? row[c + 2] : 0.f;
  v.w = c + 3 < d ? row[c + 3] : 0.f;
  return v;
}

// Block maximum of a non-negative value, flushed with one atomic (every thread calls it).
__device__ __forceinline__ void block_max_flush(float v, unsigned int* dst, float pad, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = red[0];
    for (int w = 1; w < PREP_NT / 32; ++w) m = fmaxf(m, red[w]);
    atomic_max_nonneg(dst, m * pad);
  }
  __syncthreads();
}

// FP32 rows of every instance, shifted to the instance's centre c (batch_center_kernel) and padded
// to Kp columns and to 128 rows, and their squared norms.  v = fl(x - c) differs from x - c by at
// most 2^-24 (1 + 2^-24) |v| per coordinate, so a row lies within 2^-23 |v| of its exact shifted
// position (eps32).  Block b serves instance q = the last with blk_offs[q] <= b, rows
// (b - blk_offs[q]) * rows_per_block ...
__global__ void __launch_bounds__(PREP_NT) batch_prep_kernel(const BatchInst* __restrict__ inst,
                                                             const int64_t* __restrict__ blk_offs, int count,
                                                             float* __restrict__ X, float* __restrict__ norms,
                                                             BatchState* st, BatchGlobals* g,
                                                             const float* __restrict__ center) {
  __shared__ float red[PREP_NT / 32];
  const int q = find_inst(blk_offs, count, blockIdx.x);
  const BatchInst in = inst[q];
  const int ch = in.Kp / 4, L = prep_lanes(ch), rpb = PREP_NT / L;  // float4 chunks, lanes per row, rows per block
  const int64_t npad = (int64_t)(in.n + TILE_BM - 1) / TILE_BM * TILE_BM;
  const int64_t r = (blockIdx.x - blk_offs[q]) * rpb + threadIdx.x / L;
  const int gl = threadIdx.x % L;
  const bool vec = (in.d % 4 == 0) && ((reinterpret_cast<uintptr_t>(in.pts) & 15) == 0);
  float n2 = 0.f;
  bool bad = false;
  if (r < npad) {
    const float* row = in.pts + r * in.d;
    float* out = X + in.x_off + r * in.Kp;
    for (int c = gl; c < ch; c += L) {
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (r < in.n) {
        v = load4(row, 4 * c, in.d, vec);
        bad |= !(isfinite(v.x) && isfinite(v.y) && isfinite(v.z) && isfinite(v.w));
        const float4 cc = load4(center + in.c_off, 4 * c, in.d, true);  // 16-byte aligned (c_off % 16 == 0); zeros past d
        v.x -= cc.x;
        v.y -= cc.y;
        v.z -= cc.z;
        v.w -= cc.w;
      }
      *reinterpret_cast<float4*>(out + 4 * c) = v;
      n2 = fmaf(v.x, v.x, n2);
      n2 = fmaf(v.y, v.y, n2);
      n2 = fmaf(v.z, v.z, n2);
      n2 = fmaf(v.w, v.w, n2);
    }
  }
  for (int o = L / 2; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  if (r < npad && gl == 0) norms[in.row_off + r] = n2;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&g->status, 1u);
  block_max_flush(r < npad ? n2 : 0.f, &st[q].n2_bits, 1.f + 0x1p-12f, red);
  block_max_flush(r < npad ? 0x1p-23f * sqrtf(n2) : 0.f, &st[q].eps32_bits, 1.f + 0x1p-10f, red);
}

// The centre each instance's FP32 and BF16 rows are shifted to: the midpoint of the bounding box
// of its first (at most) 256 points, per column.  Any centre leaves the distances unchanged; one
// near the middle of the points keeps their norms, and so the Gram error bound, small.  One block
// of 256 threads per instance, a thread per column.
__global__ void __launch_bounds__(256) batch_center_kernel(const BatchInst* __restrict__ inst,
                                                           float* __restrict__ center) {
  const BatchInst in = inst[blockIdx.x];
  if (threadIdx.x >= in.d) return;
  const int k = threadIdx.x;
  const int m = in.n < 256 ? (int)in.n : 256;
  if (m == 0) {
    center[in.c_off + k] = 0.f;
    return;
  }
  float lo = in.pts[k], hi = lo;
#pragma unroll 8
  for (int r = 1; r < m; ++r) {
    const float v = in.pts[(int64_t)r * in.d + k];
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  const float c = 0.5f * lo + 0.5f * hi;
  center[in.c_off + k] = isfinite(c) ? c : 0.f;
}

__global__ void batch_bounds_kernel(const BatchInst* __restrict__ inst, BatchState* st, int count) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  st[q].bp.eps_pair = 2.f * __uint_as_float(st[q].eps32_bits) * (1.f + 0x1p-20f);  // the shift's rounding
  st[q].bp.e_acc = inst[q].kappa * __uint_as_float(st[q].n2_bits) * (1.f + 0x1p-20f);
  st[q].bp16.eps_pair = 2.f * __uint_as_float(st[q].eps16_bits) * (1.f + 0x1p-20f);
  st[q].bp16.e_acc = inst[q].kappa16 * __uint_as_float(st[q].n2_16_bits) * (1.f + 0x1p-20f);
}

// BF16 rows of the tensor-core instances (padded to their class width and to 256 rows), their FP32
// squared norms, and the norm pieces of the norm MMA; each lane converts 8 values (one 16-byte
// store).  Every point is first shifted by its instance's centre c (batch_center_kernel; distances
// do not change, while the norms, and with them the Gram error bound, shrink: for points in
// [0, 1]^d from up to d to about d / 4, and far more for points far from the origin).  The row's distance from its exact shifted position is at most the residual
// |v - x~| (exact in FP32) plus the rounding of v = fl(x - c), |v - (x - c)| <= 2^-24 (1 + 2^-24) |v|
// per coordinate; eps bounds their sum with 2^-23 |v|.  Blocks as in batch_prep_kernel, over the
// tensor-core instances' 256-row blocks.
__global__ void __launch_bounds__(PREP_NT) batch_prep16_kernel(const BatchInst* __restrict__ inst,
                                                               const int64_t* __restrict__ blk_offs, int count,
                                                               X16Set X16, float* __restrict__ norms16,
                                                               __nv_bfloat16* __restrict__ H16, BatchState* st,
                                                               const float* __restrict__ center) {
  __shared__ float red[PREP_NT / 32];
  const int q = find_inst(blk_offs, count, blockIdx.x);
  const BatchInst in = inst[q];
  const int Kp16 = cls_kp16(in.cls), ch = Kp16 / 8, L = prep_lanes(ch), rpb = PREP_NT / L;
  const int64_t npad = (int64_t)(in.n + 255) / 256 * 256;
  const int64_t r = (blockIdx.x - blk_offs[q]) * rpb + threadIdx.x / L;
  const int gl = threadIdx.x % L;
  const bool vec = (in.d % 4 == 0) && ((reinterpret_cast<uintptr_t>(in.pts) & 15) == 0);
  float n2 = 0.f, dd = 0.f, vv = 0.f;
  if (r < npad) {
    const float* row = in.pts + r * in.d;
    // (a select chain: indexing the parameter array with a runtime class would copy it to local memory)
    __nv_bfloat16* base = X16.p[0];
#pragma unroll
    for (int k = 1; k < NCLS; ++k) base = in.cls == k ? X16.p[k] : base;
    __nv_bfloat16* out = base + (in.row_off16 + r) * Kp16;
    for (int c = gl; c < ch; c += L) {
      float v[8];
      if (r < in.n) {
        const float4 a = load4(row, 8 * c, in.d, vec), b = load4(row, 8 * c + 4, in.d, vec);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int col = 8 * c + k;
          if (col < in.d) {
            v[k] = v[k] - center[in.c_off + col];
            vv = fmaf(v[k], v[k], vv);
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = 0.f;
      }
      uint32_t w[4];
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v[k]), h1 = __float2bfloat16_rn(v[k + 1]);
        const float f0 = __bfloat162float(h0), f1 = __bfloat162float(h1);
        const float d0 = v[k] - f0, d1 = v[k + 1] - f1;  // exact in FP32
        n2 = fmaf(f0, f0, n2);
        n2 = fmaf(f1, f1, n2);
        dd = fmaf(d0, d0, dd);
        dd = fmaf(d1, d1, dd);
        w[k / 2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      }
      *reinterpret_cast<uint4*>(out + 8 * c) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  for (int o = L / 2; o > 0; o >>= 1) {
    n2 += __shfl_xor_sync(0xffffffffu, n2, o);
    dd += __shfl_xor_sync(0xffffffffu, dd, o);
    vv += __shfl_xor_sync(0xffffffffu, vv, o);
  }
  if (r < npad) {
    const int64_t gr = in.grow_off16 + r;
    if (gl == 0) norms16[gr] = n2;
    if (gl < 2) {  // -n2 / 2 = -(h1 + h2 + h3) to 2^-27 relative; each residual is exact in FP32
      uint32_t w0 = 0u, w1 = 0u;
      if (gl == 0) {
        const float v = 0.5f * n2;
        const float h1 = __bfloat162float(__float2bfloat16_rn(v));
        const float r1 = v - h1;
        const float h2 = __bfloat162float(__float2bfloat16_rn(r1));
        const float h3 = r1 - h2;
        w0 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(-h1)) |
             ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(-h2)) << 16);
        w1 = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(-h3));
      }
      *reinterpret_cast<uint4*>(H16 + gr * 16 + 8 * gl) = make_uint4(w0, w1, 0u, 0u);
    }
  }
  block_max_flush(r < npad ? n2 : 0.f, &st[q].n2_16_bits, 1.f + 0x1p-12f, red);
  block_max_flush(r < npad ? sqrtf(dd) + 0x1p-23f * sqrtf(vv) : 0.f, &st[q].eps16_bits, 1.f + 0x1p-10f, red);
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
        if ((int64_t)k < trec_cap) trec[k] = TileRec{q, (int32_t)bi, (int32_t)bj, tmin};  // FP32-path record
      }
      if (ub < Ug) atomic_min_nonneg(&st[q].U_bits, ub);
    }
  }
}

// Pass 2: recompute the recorded tiles that can still reach their instance's final bound and emit
// their closest-pair candidates (D~ <= theta(U_final)).
__global__ void __launch_bounds__(TILE_NT, 2)
    batch_tile_recheck_kernel(const BatchInst* __restrict__ inst, const float* __restrict__ X,
                              const float* __restrict__ norms, BatchState* st, BatchGlobals* g,
                              const TileRec* __restrict__ trec, int64_t trec_cap, BatchCand* __restrict__ cand,
                              int64_t cap, int tighten) {
  __shared__ __align__(16) TileSmem sm;
  __shared__ int list[TILE_NT];
  __shared__ int nlist;
  __shared__ float red[TILE_NT / 32];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t nrec = (int64_t)g->n_trec < trec_cap ? (int64_t)g->n_trec : trec_cap;
  // tighten = 1: a tensor-core bound U comes from BF16 tile minima and cannot get below about
  //   (sqrt(e_acc16) + eps16)^2; the tile(s) of each instance with the smallest recorded minimum
  //   are recomputed in FP32 and U is lowered to the FP32 bound of their minimum.
  // tighten = 0: every record whose minimum may still reach the final U is recomputed in FP32 and
  //   its closest-pair candidates are emitted.
  // Most records were written before their instance's bound settled: the block tests TILE_NT of
  // them at once and recomputes only the survivors.
  for (int64_t base = (int64_t)blockIdx.x * TILE_NT; base < nrec; base += (int64_t)gridDim.x * TILE_NT) {
    if (tid == 0) nlist = 0;
    __syncthreads();
    if (base + tid < nrec) {
      const TileRec tr = trec[base + tid];
      const int q = tr.qf & ~TC_FLAG;
      bool keep;
      if (tighten) {
        keep = (tr.qf & TC_FLAG) && fmaxf(tr.tmin, 0.f) <= __uint_as_float(st[q].tmin16_bits);
      } else {
        // the record's minimum was measured by its own path: test it with that path's bound parameters
        keep = tr.tmin <= theta_of(__uint_as_float(st[q].U_bits), (tr.qf & TC_FLAG) ? st[q].bp16 : st[q].bp);
      }
      if (keep) list[atomicAdd(&nlist, 1)] = tid;
    }
    __syncthreads();
    const int m = nlist;
    for (int e = 0; e < m; ++e) {
      const TileRec tr = trec[base + list[e]];
      const int q = tr.qf & ~TC_FLAG;
      const BoundParams bp = st[q].bp;
      const float th = theta_of(__uint_as_float(st[q].U_bits), bp);
      const BatchInst in = inst[q];
      const int64_t row0 = (int64_t)tr.bi * TILE_BM, col0 = (int64_t)tr.bj * TILE_BM;
      float acc[8][8];
      simt_tile_mainloop(X + in.x_off, in.Kp, row0, col0, sm, acc);
      const float* nr = norms + in.row_off;
      float tmin = __int_as_float(0x7f800000);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int64_t i = row0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
        const float nx = nr[i];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int64_t j = col0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4);
          const float D = fmaf(-2.f, acc[r][c], nx + nr[j]);
          if (i < in.n && j < in.n && j > i) {
            tmin = fminf(tmin, D);
            if (!tighten && D <= th) {
              const unsigned long long k = atomicAdd(&g->n_cand, 1ull);
              if ((int64_t)k < cap) {
                BatchCand cd;
                cd.qk = q | CPP_FLAG;
                cd.i = (int32_t)i;
                cd.j = (int32_t)j;
                cd.d2f = D;
                cand[k] = cd;
              }
            }
          }
        }
      }
      if (tighten) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tmin = fminf(tmin, __shfl_xor_sync(0xffffffffu, tmin, o));
        if ((tid & 31) == 0) red[tid >> 5] = tmin;
        __syncthreads();
        if (tid == 0) {
          for (int w = 1; w < TILE_NT / 32; ++w) tmin = fminf(tmin, red[w]);
          if (tmin < __int_as_float(0x7f800000)) atomic_min_nonneg(&st[q].U_bits, upper_d2(tmin, bp));
        }
      }
    }
    __syncthreads();  // the list and the tile buffers are reused
  }
}


// ---------------------------------------------------------------- tensor-core tiles
namespace btc {
using namespace tc;
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
// A stage holds one K chunk (16, 32 or 64 columns) of the tile's A rows and B rows at fixed offsets
// sized for 64 columns, and on the first chunk the B rows' norm pieces H.  Every region starts on a
// 1024-byte boundary, and the B rows 128..255 start 128 rows (a multiple of the swizzle atom) after
// row 0, so the same offsets serve all three swizzle widths.
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, H_BYTES = BN * 16 * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES + H_BYTES;
constexpr int ONES_BYTES = 256;                           // 8 x 32-byte rows of the constant operand
// Epilogue shape G (the kernel's template parameter): G groups of four warps.  With G = 2 group a
// reads the whole accumulator a of the CTA's tiles a, a + 2, ...; with G = 4 group 2 h + a reads half
// h of it (TMEM columns 256 a + 128 h .. + 127), so twice the warps share each tile.  Either way every
// 128-column half of a tile is a block of its own for the minimum, the record and the bound update.
// Four groups pay off where the MMAs are short (small d: the epilogue paces the kernel), two where
// they are long (fewer warps pay the per-tile bookkeeping); the tuning policy picks per class.
template <int G>
struct Shape {
  static_assert(G == 2 || G == 4, "two or four epilogue groups");
  static constexpr int HALVES = 4 / G;                // 128-column halves per group and tile
  static constexpr int NTHREADS = 64 + G * 128 + 32;  // producer, MMA, the epilogue warps, tile decoder
  static constexpr int DECODER = NTHREADS / 32 - 1;   // the decoder's warp
  static constexpr int RING_READERS = 1 + 4 * (G / 2);  // producer and the warps of the tile's groups
};
constexpr uint32_t TMEM_COLS = 512;

// What the decoder warp publishes about each of the CTA's tiles (ring slot = tile iteration % RING).
struct TileInfo {
  int32_t q, bi, bj, n;
  int64_t grow;      // first BF16 row of the instance (norms, norm pieces)
  int64_t row16;     // first row of the instance in its class matrix
  int32_t cls;       // width class (cls_kp16, cls_chunk, cls_nchunks)
  float th_r;        // radius emission threshold on D~ (-inf: no radius output)
  BoundParams bp;    // the instance's tensor-core bound parameters
};
constexpr int RING = 16;         // tile records in flight
constexpr int TILE_RUN = 16;     // consecutive tiles a CTA takes at a time

// Shared-memory descriptor of a K-major operand region whose rows hold `chunk` 16-bit values.
__device__ __forceinline__ uint64_t op_desc(uint32_t saddr, int chunk) {
  return chunk == 64 ? sw128_desc(saddr) : chunk == 32 ? sw64_desc(saddr) : sw32_desc(saddr, 256);
}

// Fault injection for the tests of the bounded waits (cpp_set_fault_injection): when non-zero the TMA
// producer issues no copy (and consumes no tile record), so the MMA issuer's, the epilogue's and the
// decoder's waits run out and the batch reports CPPGB_ERR_TIMEOUT.  Zero unless a test sets it.
__device__ int g_fault_skip_tma = 0;

template <int G>
struct Ctl {
  uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], drain;  // tfull / tempty per accumulator
  uint32_t shdr[STAGES];  // what the stage holds: chunk width | chunk index << 8 | chunks of the tile << 16
  uint64_t info_full[RING], info_empty[RING];
  TileInfo info[RING];
  unsigned int wmin[G][2][Shape<G>::HALVES][4];  // per group, parity of its tile count and half: each warp's minimum
  unsigned int arrived[G][2];                    // warps that have stored their minima
  uint32_t tmem_base;
  int abort_flag;
};
template <int G>
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + ONES_BYTES + sizeof(Ctl<G>) + 1024;  // + alignment slack
static_assert(SMEM_BYTES<2> <= 232448 && SMEM_BYTES<4> <= 232448, "dynamic shared memory above the 227 KB opt-in limit");

// Tiles (bi, bj) of one instance: 128-row blocks bi < nrow16, 256-column blocks bj with
// bj >= bi / 2 (every such tile holds a pair i < j).  Rows 2k and 2k + 1 have nbj - k tiles, so
// the tiles before row 2k number 2k nbj - k (k - 1); k is found by bisection.
__device__ __forceinline__ void decode16(int64_t t, int64_t nbj, int64_t nrow, int64_t* bi, int64_t* bj) {
  auto P = [&](int64_t k) { return 2 * k * nbj - k * (k - 1); };
  int64_t lo = 0, hi = (nrow + 1) / 2;  // largest k with P(k) <= t
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) >> 1;
    if (P(mid) <= t) lo = mid;
    else hi = mid - 1;
  }
  const int64_t k = lo, r = t - P(k), c = nbj - k;
  if (r < c) {
    *bi = 2 * k;
    *bj = k + r;
  } else {
    *bi = 2 * k + 1;
    *bj = k + (r - c);
  }
}

// Follows one role's increasing tile sequence: the instance by a forward cursor over the tile
// offsets (binary search after a long jump), (bi, bj) by stepping along the rows of the instance
// (bisection on entering an instance or after a long step).
struct TileWalker {
  const int64_t* offs;
  const BatchInst* insts;
  int count, q;
  int64_t lo, hi, cur, bi, bj;
  BatchInst in;

  __device__ __forceinline__ void init(const int64_t* o, const BatchInst* is, int c) {
    offs = o;
    insts = is;
    count = c;
    q = -1;
    lo = hi = 0;
  }
  __device__ __forceinline__ void go(int64_t t) {
    if (t >= hi) {
      int qq = q + 1, steps = 0;
      while (qq < count - 1 && offs[qq + 1] <= t && steps < 8) {
        ++qq;
        ++steps;
      }
      if (qq < count - 1 && offs[qq + 1] <= t) qq = find_inst(offs, count, t);
      q = qq;
      in = insts[q];
      lo = offs[q];
      hi = offs[q + 1];
      cur = t - lo;
      decode16(cur, in.nbj16, in.nrow16, &bi, &bj);
      return;
    }
    int64_t r = t - lo - cur;
    cur += r;
    if (r > 4 * (in.nbj16 - (bi >> 1))) {
      decode16(cur, in.nbj16, in.nrow16, &bi, &bj);
      return;
    }
    while (r > 0) {
      const int64_t rem = in.nbj16 - bj;
      if (r < rem) {
        bj += r;
        break;
      }
      r -= rem;
      ++bi;
      bj = bi >> 1;
    }
  }
};


// One 32-column chunk of a row.  The accumulator holds a_ij = x~_i.x~_j - |x~_j|^2 / 2 (the norm
// pieces ride along in the MMA), so D~_ij = |x~_i|^2 - 2 a_ij is decreasing in a_ij and the chunk's
// smallest D~ comes from its largest a (a depth-5 tree).  EDGE tiles mask entries off the triangle
// and past n to -inf.
template <bool EDGE>
// Indices are 32-bit (n < 2^31): entry k (column j0 + k) is kept iff i < n and i < j0 + k < n.
__device__ __forceinline__ float chunk_max(uint32_t (&r)[32], int32_t i, int32_t j0, int32_t n) {
  if (EDGE) {
    const int32_t klo = i - j0, khi = i < n ? n - j0 : -1;  // keep klo < k < khi
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (!(k > klo && k < khi)) r[k] = __float_as_uint(__int_as_float(0xff800000));
  }
  float m[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) m[k] = fmaxf(__uint_as_float(r[k]), __uint_as_float(r[k + 16]));
#pragma unroll
  for (int k = 0; k < 8; ++k) m[k] = fmaxf(m[k], m[k + 8]);
#pragma unroll
  for (int k = 0; k < 4; ++k) m[k] = fmaxf(m[k], m[k + 4]);
  return fmaxf(fmaxf(m[0], m[2]), fmaxf(m[1], m[3]));
}

// 64-column TMEM loads, split into issue and wait (the wait names the destination registers, so no
// use of them is scheduled before it).
__device__ __forceinline__ void tmem_ld64_nowait(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,"
      "%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld64(uint32_t (&r)[64]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]),
                 "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]),
                 "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31]), "+r"(r[32]), "+r"(r[33]), "+r"(r[34]), "+r"(r[35]), "+r"(r[36]),
                 "+r"(r[37]), "+r"(r[38]), "+r"(r[39]), "+r"(r[40]), "+r"(r[41]), "+r"(r[42]), "+r"(r[43]),
                 "+r"(r[44]), "+r"(r[45]), "+r"(r[46]), "+r"(r[47]), "+r"(r[48]), "+r"(r[49]), "+r"(r[50]),
                 "+r"(r[51]), "+r"(r[52]), "+r"(r[53]), "+r"(r[54]), "+r"(r[55]), "+r"(r[56]), "+r"(r[57]),
                 "+r"(r[58]), "+r"(r[59]), "+r"(r[60]), "+r"(r[61]), "+r"(r[62]), "+r"(r[63])
               :
               : "memory");
}
// Two 32-column chunks of one 64-column load: the rows' largest a so far, and bit c / c + 1 of
// `hits` when some entry of that chunk may lie within the radius (D~ <= th_r).
template <bool EDGE>
__device__ __forceinline__ void reduce64(uint32_t (&r)[64], int32_t i, int32_t j0, int32_t n, float nx, float th_r,
                                         int c, uint32_t& hits, float& rmax) {
  uint32_t (&lo)[32] = *reinterpret_cast<uint32_t(*)[32]>(&r[0]);
  uint32_t (&hi)[32] = *reinterpret_cast<uint32_t(*)[32]>(&r[32]);
  float m = chunk_max<EDGE>(lo, i, j0, n);
  hits |= (fmaf(-2.f, m, nx) <= th_r ? 1u : 0u) << c;
  rmax = fmaxf(rmax, m);
  m = chunk_max<EDGE>(hi, i, j0 + 32, n);
  hits |= (fmaf(-2.f, m, nx) <= th_r ? 1u : 0u) << (c + 1);
  rmax = fmaxf(rmax, m);
}

// 32-column TMEM load into `r` that also names `keep` (the chunk being reduced meanwhile) as
// read-write, so the reduction of `keep` cannot be moved above the load's issue.
__device__ __forceinline__ void tmem_ld32_after(uint32_t taddr, uint32_t (&r)[32], uint32_t (&keep)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
      "[%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "+r"(keep[0]), "+r"(keep[1]), "+r"(keep[2]), "+r"(keep[3]), "+r"(keep[4]), "+r"(keep[5]), "+r"(keep[6]), "+r"(keep[7]), "+r"(keep[8]), "+r"(keep[9]), "+r"(keep[10]), "+r"(keep[11]), "+r"(keep[12]), "+r"(keep[13]), "+r"(keep[14]), "+r"(keep[15]), "+r"(keep[16]), "+r"(keep[17]), "+r"(keep[18]), "+r"(keep[19]), "+r"(keep[20]), "+r"(keep[21]), "+r"(keep[22]), "+r"(keep[23]), "+r"(keep[24]), "+r"(keep[25]), "+r"(keep[26]), "+r"(keep[27]), "+r"(keep[28]), "+r"(keep[29]), "+r"(keep[30]), "+r"(keep[31])
      : "r"(taddr)
      : "memory");
}
// Wait for the loads in flight; `after` (computed from the previous chunk) is an input, so that
// computation stays before the wait.
__device__ __forceinline__ void tmem_wait_ld32_after(uint32_t (&r)[32], float after) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
               : "f"(after)
               : "memory");
}

// A warp's 32 rows x (64 NLD) columns from TMEM.  Returns the rows' largest a; `hits` gets bit c for
// the 32-column chunks c that may hold radius pairs, for the rare second look.  Interior tiles issue
// each 32-column load before the previous chunk is reduced (the asm operands pin that order), so the
// load latency overlaps the max trees; EDGE tiles (masked entries, a small share of the work) load,
// wait and reduce 64 columns at a time.
template <bool EDGE, int NLD>
__device__ __forceinline__ float tile_rows(uint32_t tbase, int32_t i, int32_t col0, int32_t n, float nx, float th_r,
                                           uint32_t& hits) {
  float rmax = __int_as_float(0xff800000);
  if (EDGE) {
    uint32_t ra[64];
#pragma unroll 1
    for (int c = 0; c < NLD; ++c) {
      __syncwarp();
      tmem_ld64_nowait(tbase + (uint32_t)(c * 64), ra);
      tmem_wait_ld64(ra);
      reduce64<true>(ra, i, col0 + c * 64, n, nx, th_r, 2 * c, hits, rmax);
    }
    return rmax;
  }
  uint32_t ra[32], rb[32];
  __syncwarp();
  tmem_ld32_nowait(tbase, ra);
  tmem_wait_ld(ra);
#pragma unroll
  for (int c = 0; c < 2 * NLD; c += 2) {
    tmem_ld32_after(tbase + (uint32_t)((c + 1) * 32), rb, ra);
    float m = chunk_max<false>(ra, i, col0 + c * 32, n);
    hits |= (fmaf(-2.f, m, nx) <= th_r ? 1u : 0u) << c;
    rmax = fmaxf(rmax, m);
    tmem_wait_ld32_after(rb, rmax);
    if (c + 2 < 2 * NLD) tmem_ld32_after(tbase + (uint32_t)((c + 2) * 32), ra, rb);
    m = chunk_max<false>(rb, i, col0 + (c + 1) * 32, n);
    hits |= (fmaf(-2.f, m, nx) <= th_r ? 1u : 0u) << (c + 1);
    rmax = fmaxf(rmax, m);
    if (c + 2 < 2 * NLD) tmem_wait_ld32_after(ra, rmax);
  }
  return rmax;
}

// Rare: emit this lane's radius candidates of the flagged chunks (re-read from TMEM; the accumulator
// is still held).  Warp-collective: every lane of the warp calls it with the warp's union of flags.
__device__ __noinline__ void emit_radius(uint32_t tbase, uint32_t flags, int64_t i, int64_t col0, int64_t n, float nx,
                                         float th_r, int q, BatchGlobals* g, BatchCand* __restrict__ cand,
                                         int64_t cap) {
  for (int c = 0; c < BN / 32; ++c) {
    if (!((flags >> c) & 1u)) continue;  // warp-uniform
    uint32_t r[32];
    tmem_ld32_nowait(tbase + (uint32_t)(c * 32), r);
    tmem_wait_ld(r);
    uint32_t bits = 0u;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int64_t j = col0 + c * 32 + k;
      const float a = __uint_as_float(r[k]);
      bits |= (i < n && j < n && j > i && fmaf(-2.f, a, nx) <= th_r ? 1u : 0u) << k;
    }
    while (bits) {
      const int k = __ffs(bits) - 1;
      bits &= bits - 1u;
      const unsigned long long slot = atomicAdd(&g->n_cand, 1ull);
      if ((int64_t)slot < cap) {
        BatchCand cd;
        cd.qk = q;  // radius candidate: decided by the FP64 test alone, its FP32 value is not used
        cd.i = (int32_t)i;
        cd.j = (int32_t)(col0 + c * 32 + k);
        cd.d2f = 0.f;
        cand[slot] = cd;
      }
    }
  }
}

// 19 warps (four groups): five of them share an SM sub-partition's 16,384 registers, so at most 96
// each; 11 warps (two groups): three per sub-partition, at most 168.
template <int G>
__global__ void __maxnreg__(G == 4 ? 96 : 168)
    batch_tc_kernel(const __grid_constant__ BatchMaps maps, const BatchInst* __restrict__ inst,
                    const int64_t* __restrict__ tile_offs16, int count, int64_t total, const float* __restrict__ norms16,
                    BatchState* st, BatchGlobals* g, BatchCand* __restrict__ cand, int64_t cap,
                    TileRec* __restrict__ trec, int64_t trec_cap) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* ones = smem + STAGES * STAGE_BYTES;  // 1024-aligned
  using S = Shape<G>;
  Ctl<G>* ctl = (Ctl<G>*)(ones + ONES_BYTES);
  volatile int* abort_flag = &ctl->abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // This CTA's tiles: runs r = blockIdx.x, blockIdx.x + gridDim.x, ... of TILE_RUN consecutive tile
  // indices (tile_at below), so consecutive tiles of a CTA mostly share their row block.
  int64_t ntl = 0;
  {
    const int64_t nruns = (total + TILE_RUN - 1) / TILE_RUN;
    const int64_t mine = nruns > blockIdx.x ? (nruns - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    ntl = mine * TILE_RUN;
    if (mine > 0 && blockIdx.x + (mine - 1) * gridDim.x == nruns - 1) ntl -= nruns * TILE_RUN - total;
  }

  if (threadIdx.x < 64) {
    // Constant A operand of the norm MMA: every row is (1, 1, 1, 0, ..., 0) in BF16.  In the
    // 32-byte swizzle the two 16-byte halves of rows 4..7 (of every 8) trade places.
    const int row = threadIdx.x >> 3, word = threadIdx.x & 7;  // 8 rows x 8 words of 4 bytes
    const int half = (word >> 2) ^ ((row >> 2) & 1), w4 = word & 3;
    uint32_t v = 0u;
    if (half == 0 && w4 == 0) v = 0x3f803f80u;  // elements 0, 1
    if (half == 0 && w4 == 1) v = 0x00003f80u;  // element 2
    reinterpret_cast<uint32_t*>(ones)[threadIdx.x] = v;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&ctl->full[s], 1);
      mbar_init(&ctl->empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&ctl->tfull[a], 1);
      mbar_init(&ctl->tempty[a], 4 * (G / 2));  // the warps of the accumulator's epilogue groups
    }
    for (int r = 0; r < RING; ++r) {
      mbar_init(&ctl->info_full[r], 1);
      mbar_init(&ctl->info_empty[r], S::RING_READERS);
    }
    mbar_init(&ctl->drain, 1);
    for (int a = 0; a < G; ++a)
      for (int b = 0; b < 2; ++b) ctl->arrived[a][b] = 0u;
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

  if (warp == S::DECODER) {
    if (lane == 0) {  // ---------------------------------------------- tile decoder
      TileWalker w;
      w.init(tile_offs16, inst, count);
      int bq = -1;
      TileInfo ti;
      bool ok = true;
      for (int64_t it = 0; it < ntl; ++it) {
        const uint32_t slot = (uint32_t)(it % RING);
        if (it >= RING && !mbar_wait(&ctl->info_empty[slot], (uint32_t)((it / RING - 1) & 1), abort_flag)) {
          ok = false;
          break;
        }
        w.go((blockIdx.x + (it / TILE_RUN) * gridDim.x) * TILE_RUN + it % TILE_RUN);
        if (w.q != bq) {
          bq = w.q;
          ti.q = w.q;
          ti.n = w.in.n;
          ti.grow = w.in.grow_off16;
          ti.row16 = w.in.row_off16;
          ti.cls = w.in.cls;
          ti.bp = st[w.q].bp16;
          ti.th_r = w.in.has_r ? theta_of(w.in.rr32, ti.bp) : __int_as_float(0xff800000);
        }
        ti.bi = (int32_t)w.bi;
        ti.bj = (int32_t)w.bj;
        ctl->info[slot] = ti;
        mbar_arrive(&ctl->info_full[slot]);  // release: the record is visible to its waiters
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&g->status, 4u);
      }
    }
  } else if (warp == 0) {
    if (lane == 0) {  // ---------------------------------------------- TMA producer
      for (int c = 0; c < NCLS; ++c) asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.m[c]) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&maps.h) : "memory");
      uint32_t stage = 0, phase = 0;
      int64_t issued = 0;
      bool ok = true;
      const bool skip = *reinterpret_cast<volatile int*>(&g_fault_skip_tma) != 0;
      for (int64_t it = 0; it < ntl && ok && !skip; ++it) {
        const uint32_t slot = (uint32_t)(it % RING);
        if (!mbar_wait(&ctl->info_full[slot], (uint32_t)((it / RING) & 1), abort_flag)) { ok = false; break; }
        const TileInfo ti = ctl->info[slot];
        mbar_arrive(&ctl->info_empty[slot]);
        const CUtensorMap* map = &maps.m[ti.cls];
        const int ya = (int)(ti.row16 + (int64_t)ti.bi * BM), yb = (int)(ti.row16 + (int64_t)ti.bj * BN);
        const int yh = (int)(ti.grow + (int64_t)ti.bj * BN);
        const int kch = cls_nchunks(ti.cls), kcw = cls_chunk(ti.cls);
        const uint32_t rows128 = (uint32_t)(BM * kcw * 2);  // bytes of 128 rows of one chunk
        for (int kc = 0; kc < kch; ++kc) {
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1u, abort_flag)) { ok = false; break; }
          uint8_t* sa = smem + stage * STAGE_BYTES;
          ctl->shdr[stage] = (uint32_t)kcw | ((uint32_t)kc << 8) | ((uint32_t)kch << 16);  // released by the arrive
          mbar_arrive_expect_tx(&ctl->full[stage], 3u * rows128 + (kc == 0 ? H_BYTES : 0));
          tma_load_2d(sa, map, &ctl->full[stage], kc * kcw, ya);
          tma_load_2d(sa + A_BYTES, map, &ctl->full[stage], kc * kcw, yb);
          tma_load_2d(sa + A_BYTES + rows128, map, &ctl->full[stage], kc * kcw, yb + BM);
          if (kc == 0) tma_load_2d(sa + A_BYTES + B_BYTES, &maps.h, &ctl->full[stage], 0, yh);
          ++issued;
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&g->status, 4u);
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
      // Driven by the stages alone: each stage's header (written by the producer before the stage's
      // arrive, read after the full wait) gives the chunk's width, its index and the tile's chunk
      // count, so between two tiles this thread only waits for the next stage and, on a tile's first
      // chunk, for the accumulator.  Tile it goes to accumulator it & 1 (columns 256 (it & 1) ..);
      // one N = 256 MMA per K = 16 step, then one more that adds the B rows' norm pieces.
      const uint32_t idesc = make_idesc(1u, BM, BN);
      const uint64_t ones_d = sw32_desc(smem_u32(ones), 0);
      uint32_t stage = 0, phase = 0;
      bool ok = true;
      for (int64_t it = 0; it < ntl && ok; ++it) {
        const uint32_t acc = (uint32_t)(it & 1), use = (uint32_t)((it >> 1) & 1);
        const uint32_t dtmem = tmem_base + acc * (uint32_t)BN;
        int kc = 0, kch = 1;
        do {
          if (!mbar_wait(&ctl->full[stage], phase, abort_flag)) { ok = false; break; }
          const uint32_t hdr = ctl->shdr[stage];
          const int kcw = (int)(hdr & 0xffu);
          kc = (int)((hdr >> 8) & 0xffu);
          kch = (int)(hdr >> 16);
          if (kc == 0 && !mbar_wait(&ctl->tempty[acc], use ^ 1u, abort_flag)) { ok = false; break; }
          tc_fence_after();
          const uint32_t sa = smem_u32(smem + stage * STAGE_BYTES);
          const uint64_t ad = op_desc(sa, kcw), bd = op_desc(sa + A_BYTES, kcw);
          mma_f16(dtmem, ad, bd, idesc, kc != 0);
          if (kcw >= 32) mma_f16(dtmem, ad + 2, bd + 2, idesc, 1u);
          if (kcw == 64) {
            mma_f16(dtmem, ad + 4, bd + 4, idesc, 1u);
            mma_f16(dtmem, ad + 6, bd + 6, idesc, 1u);
          }
          if (kc == 0)  // + ones x (B rows' norm pieces): a_ij = x~_i.x~_j - |x~_j|^2 / 2
            mma_f16(dtmem, ones_d, sw32_desc(sa + A_BYTES + B_BYTES, 256), idesc, 1u);
          mma_commit(&ctl->empty[stage]);
          if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        } while (kc + 1 < kch);
        if (!ok) break;
        mma_commit(&ctl->tfull[acc]);
      }
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&g->status, 4u);
      }
      mma_commit(&ctl->drain);
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < WAIT_NS) {
      }
    }
  } else {  // -------------------------------------------------------- epilogue groups
    // Group grp takes the CTA's tiles it = a, a + 2, ... in accumulator a and, of each, the 128-column
    // halves h0 .. h0 + HALVES - 1; warp (warp & 3) reads TMEM lanes 32 (warp & 3) .. + 31 (the rows
    // it may access).  Each half is a 128 x 128 block of its own: its minimum, its record for the FP32
    // second pass and its bound update.  The groups never wait for one another, nor do the warps of
    // a group: each stores its minima, and the last to arrive takes the halves' record decisions.
    constexpr int HALVES = S::HALVES;
    const int grp = (warp - 2) >> 2, par_a = grp % 2, h0 = (grp / 2) * HALVES;
    const uint32_t quarter = (uint32_t)(warp & 3);
    const float INF = __int_as_float(0x7f800000);
    // A warp keeps its tile's ring slot until the tile is done and reads the record's fields from
    // shared memory where it needs them (few registers stay live across the TMEM reads); the row
    // norm of the group's next tile is loaded one tile ahead.
    // The norms are reloaded only when the row block changes (consecutive tiles mostly share it).
    float nx_n = 0.f;
    int32_t f_q = -1, f_bi = -1;
    bool ok = true;
    auto fetch = [&](int64_t it) -> bool {
      const uint32_t slot = (uint32_t)(it % RING);
      const bool got = __all_sync(0xffffffffu, mbar_wait(&ctl->info_full[slot], (uint32_t)((it / RING) & 1), abort_flag));
      if (!got) return false;
      const TileInfo* ti = &ctl->info[slot];
      const int32_t q = ti->q, bi = ti->bi;
      if (q != f_q || bi != f_bi) {
        nx_n = norms16[ti->grow + (int64_t)bi * BM + quarter * 32 + lane];
        f_q = q;
        f_bi = bi;
      }
      return true;
    };
    if (par_a < ntl) ok = fetch(par_a);
    int64_t k = 0;
    const uint32_t tb = tmem_base + ((quarter * 32u) << 16) + (uint32_t)par_a * (uint32_t)BN + (uint32_t)h0 * (BN / 2);
    for (int64_t it = par_a; it < ntl && ok; it += 2, ++k) {
      const TileInfo* cur = &ctl->info[it % RING];
      const float nx = nx_n;
      const float Ug = __uint_as_float(*reinterpret_cast<volatile unsigned int*>(&st[cur->q].U_bits));  // early load
      if (it + 2 < ntl && !fetch(it + 2)) { ok = false; break; }
      const uint32_t par = (uint32_t)(k & 1);
      if (!__all_sync(0xffffffffu, mbar_wait(&ctl->tfull[par_a], par, abort_flag))) { ok = false; break; }
      tc_fence_after();
      float rmax[HALVES];
#pragma unroll
      for (int hh = 0; hh < HALVES; ++hh) {
        const int32_t n = cur->n, row0 = cur->bi * BM, c0 = cur->bj * BN + (h0 + hh) * (BN / 2);
        const int32_t i = row0 + (int32_t)quarter * 32 + lane;
        const bool edge = (row0 + BM - 1 >= n) || (c0 + BN / 2 - 1 >= n) || (c0 < row0 + BM);
        const float th_r = cur->th_r;
        const uint32_t t = tb + (uint32_t)hh * (BN / 2);
        uint32_t hits = 0u;
        rmax[hh] = edge ? tile_rows<true, 2>(t, i, c0, n, nx, th_r, hits) : tile_rows<false, 2>(t, i, c0, n, nx, th_r, hits);
        const uint32_t flags = __reduce_or_sync(0xffffffffu, hits);
        if (flags) emit_radius(t, flags, i, c0, n, nx, th_r, cur->q, g, cand, cap);
      }
      // The accumulator has been read for the last time: release it now, so that the MMA of the
      // group's next tile overlaps the reductions and the record decision below.
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->tempty[par_a]);
      // this warp's smallest D~ per half (+inf for masked rows), clamped at 0 (a looser but valid
      // bound), so the float bits order like the values
      unsigned int wm[HALVES];
#pragma unroll
      for (int hh = 0; hh < HALVES; ++hh)
        wm[hh] = __reduce_min_sync(0xffffffffu, __float_as_uint(fmaxf(fmaf(-2.f, rmax[hh], nx), 0.f)));
      // The minimum slots [grp][par] are reused two of the group's tiles later.  That tile's MMA needs
      // every warp's release of the group's tile in between, which each warp gives only after this
      // publication (and the last warp after its reset below), so no warp can overwrite a slot still
      // being read.
      bool last = false;
      float tmin[HALVES];
      if (lane == 0) {
#pragma unroll
        for (int hh = 0; hh < HALVES; ++hh) ctl->wmin[grp][par][hh][quarter] = wm[hh];
        __threadfence_block();
        last = atomicAdd(&ctl->arrived[grp][par], 1u) == 3u;
        if (last) {
          __threadfence_block();
#pragma unroll
          for (int hh = 0; hh < HALVES; ++hh) {
            const volatile unsigned int* v = ctl->wmin[grp][par][hh];
            tmin[hh] = __uint_as_float(min(min(v[0], v[1]), min(v[2], v[3])));
          }
          ctl->arrived[grp][par] = 0u;
        }
      }
      if (last) {  // each half's record and the bound update
        const int q = cur->q;
        const int32_t bi = cur->bi;
        const BoundParams bp = cur->bp;
        float ub = INF;
#pragma unroll
        for (int hh = 0; hh < HALVES; ++hh) {
          if (!(tmin[hh] < INF)) continue;
          // record the half for the FP32 second pass when its minimum can reach the bound (a half
          // with a finite minimum holds a pair i < j < n, so its FP32 rows exist)
          if (tmin[hh] <= theta_of(Ug, bp)) {
            atomic_min_nonneg(&st[q].tmin16_bits, tmin[hh]);
            const unsigned long long kr = atomicAdd(&g->n_trec, 1ull);
            if ((int64_t)kr < trec_cap) trec[kr] = TileRec{q | TC_FLAG, bi, 2 * cur->bj + h0 + hh, tmin[hh]};
          }
          ub = fminf(ub, upper_d2(tmin[hh], bp));
        }
        if (ub < Ug) atomic_min_nonneg(&st[q].U_bits, ub);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->info_empty[it % RING]);  // the record is no longer read
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      atomicOr(&g->status, 4u);
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
}  // namespace btc

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
                                    int64_t cap, cpp_pair_result* __restrict__ res,
                                    int64_t* __restrict__ counts64) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  const int64_t b = pair_offs[q], e = pair_offs[q + 1];
  counts64[q] = e - b;
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
  r.filter_e_acc = s.bp.e_acc;   // the bound of the FP32 pass whose candidates are rechecked
  r.filter_eps = s.bp.eps_pair;
  r.tiles_kept = r.tiles_total = -1;
  const unsigned int gs = g->status;
  r.status = (gs & 1u) ? CPPGB_ERR_NUMERIC : (gs & 4u) ? CPPGB_ERR_TIMEOUT
             : ((int64_t)g->n_cand > cap || pair_offs[count] > pairs_cap) ? CPPGB_ERR_CAPACITY : CPPGB_OK;
  r.reserved = 0;
  res[q] = r;
}

// ---------------------------------------------------------------- host side
struct BatchLayout {
  BatchInst* inst;
  int64_t *tile_offs, *tile_offs16[2];  // FP32-path tiles; tensor-core tile lists (four-group, two-group kernel)
  int64_t *pblk32, *pblk16;  // preparation blocks before each instance (FP32 rows; BF16 rows)
  float* center;  // per instance and column: the centre its FP32 and BF16 rows are shifted to
  BatchState* st;
  BatchGlobals* g;
  int32_t* pair_counts;
  int64_t* pair_offs;
  int64_t* tmp;
  float* X;
  float* norms;
  __nv_bfloat16* X16[NCLS];
  float* norms16;
  __nv_bfloat16* H16;  // [max(rows16, 256)][16]
  BatchCand* cand;
  double* d2buf;
  uint8_t* keep;
  TileRec* trec;
  cpp_pair_result* res;
  int64_t* counts64;  // pairs within R per instance, copied to the caller's pair_counts
  int64_t cap, trec_cap;
  size_t bytes;
};

// Path of one instance: 1 = FP32 CUDA-core tiles, 2 = BF16 tensor-core tiles read by four epilogue
// groups, 3 = the same tiles read by two; 0 takes the tuning policy's entry for the instance's
// n-bucket and d-class.
int path_of(const cpp_instance& c) {
  if (c.path >= 1 && c.path <= 3) return c.path;
  return tuned_batch_path(c.n, c.d);
}

struct Totals {
  int64_t rows = 0, xfloats = 0, tiles = 0;         // FP32 layout (all instances) and FP32-path tiles
  int64_t rows16 = 0, tiles16 = 0, crow16[NCLS] = {0, 0, 0, 0, 0, 0};
  int64_t tiles16s[2] = {0, 0};  // tensor-core tiles of path 2 (four-group kernel) and path 3 (two-group)
  int64_t blk32 = 0, blk16 = 0;  // preparation blocks (FP32 rows of every instance, BF16 rows of the tensor-core ones)
  int64_t cols = 0;              // padded columns of all instances (the centres)
};

int64_t nrow16_of(int64_t n) { return n >= 2 ? (n - 2) / 128 + 1 : 0; }
int64_t prep_blocks32(int64_t npad, int64_t Kp) {
  const int64_t rpb = PREP_NT / prep_lanes((int)(Kp / 4));
  return (npad + rpb - 1) / rpb;
}
int64_t prep_blocks16(int64_t npad16, int64_t Kp16) {
  const int64_t rpb = PREP_NT / prep_lanes((int)(Kp16 / 8));
  return (npad16 + rpb - 1) / rpb;
}
int64_t tiles16_of(int64_t n) {
  const int64_t nbj = (n + 255) / 256, nr = nrow16_of(n);
  int64_t t = 0;
  for (int64_t bi = 0; bi < nr; ++bi) t += nbj - (bi >> 1);
  return t;
}

Totals totals_of(const cpp_instance* inst, int64_t count) {
  Totals t;
  for (int64_t q = 0; q < count; ++q) {
    const int64_t n = inst[q].n, Kp = (inst[q].d + 15) / 16 * 16;
    const int64_t npad = (n + TILE_BM - 1) / TILE_BM * TILE_BM;
    const int64_t nb = npad / TILE_BM;
    t.rows += npad;
    t.xfloats += npad * Kp;
    t.blk32 += prep_blocks32(npad, Kp);
    t.cols += Kp;
    if (path_of(inst[q]) >= 2) {
      const int64_t npad16 = (n + 255) / 256 * 256;
      t.rows16 += npad16;
      t.crow16[cls_of_d(inst[q].d)] += npad16;
      t.tiles16 += tiles16_of(n);
      t.tiles16s[path_of(inst[q]) - 2] += tiles16_of(n);
      t.blk16 += prep_blocks16(npad16, cls_kp16(cls_of_d(inst[q].d)));
    } else {
      t.tiles += n >= 2 ? nb * (nb + 1) / 2 : 0;
    }
  }
  return t;
}

BatchLayout batch_layout(void* ws, int64_t count, const Totals& t, size_t ws_bytes) {
  BatchLayout L;
  Carver c(ws);
  L.inst = c.take<BatchInst>(count);
  L.tile_offs = c.take<int64_t>(count + 1);
  L.pblk32 = c.take<int64_t>(count + 1);
  L.center = c.take<float>(t.cols + 1);
  L.pblk16 = c.take<int64_t>(count + 1);
  L.tile_offs16[0] = c.take<int64_t>(count + 1);
  L.tile_offs16[1] = c.take<int64_t>(count + 1);
  L.st = c.take<BatchState>(count);
  L.g = c.take<BatchGlobals>(1);
  L.pair_counts = c.take<int32_t>(count + 1);
  L.pair_offs = c.take<int64_t>(count + 1);
  L.tmp = c.take<int64_t>(scan_temp_elems(count + 1));
  L.res = c.take<cpp_pair_result>(count);
  L.counts64 = c.take<int64_t>(count);
  L.X = c.take<float>(t.xfloats + 16);
  L.norms = c.take<float>(t.rows + 1);
  for (int k = 0; k < NCLS; ++k)  // at least 256 rows each, so every class has a valid tensor map
    L.X16[k] = c.take<__nv_bfloat16>((size_t)(t.crow16[k] > 256 ? t.crow16[k] : 256) * cls_kp16(k));
  L.norms16 = c.take<float>(t.rows16 + 1);
  L.H16 = c.take<__nv_bfloat16>((size_t)(t.rows16 > 256 ? t.rows16 : 256) * 16);
  L.trec_cap = 2 * (t.tiles + t.tiles16) + 2;  // at most one record per 128 x 128 tile
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

// Tensor-core tiles compute a_ij = x~_i.x~_j - h_j (h_j: three BF16 pieces of |x~_j|^2 / 2, within
// 2^-27 relative) with K' = Kp + 16 exact products whose magnitudes sum to at most
// |x~_i||x~_j| + 1.01 |x~_j|^2 / 2 <= 1.51 m (m = max |x~|^2); the accumulation error is padded to
// 2 K' 2^-22 of that sum.  D~ = fma(-2, a, |x~_i|^2) adds the FP32 norm error of both rows (each norm
// is eight fused products per lane, then a tree over the row's L lanes: at most 8 + log2 L
// roundings), the split error and one rounding of |D~| <= 4.03 m.
float kappa_tc(int64_t Kp) {
  const double K = (double)Kp, K2 = K + 16.0, u = 0x1p-24;
  const double nrm = 8.0 + prep_log2(prep_lanes((int)(Kp / 8)));
  return (float)((2.0 * 1.51 * 2.0 * K2 * 0x1p-22 + 2.0 * nrm * 1.01 * u + 0x1p-27 + 4.03 * u) * 1.01);
}

EncodeTiledFn encode_fn() {
  EncodeTiledFn fn = tensor_map_encoder();
  if (!fn) set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  return fn;
}

// norm pieces: [rows][16] BF16 (32-byte rows), box 16 x 256 (the B rows of one tile), 32-byte swizzle
int encode_h_map(CUtensorMap* m, void* base, int64_t rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return CPPGB_ERR_CUDA;
  const cuuint64_t gdim[2] = {16, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {32};
  const cuuint32_t box[2] = {16, 256};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult cr = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return CPPGB_OK;
}

// rows of class cls: [rows][Kp16] BF16, box chunk x 128 with the swizzle of the chunk's row length
int encode_class_map(CUtensorMap* m, void* base, int64_t rows, int cls) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return CPPGB_ERR_CUDA;
  const int Kp = cls_kp16(cls), chunk = cls_chunk(cls);
  const cuuint64_t gdim[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)Kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)chunk, 128};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw = chunk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : chunk == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  const CUresult cr = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (cr != CUDA_SUCCESS) return set_error(CPPGB_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)cr);
  return CPPGB_OK;
}

// Graph cache: one instantiated graph per argument set (all kernel arguments are baked in).
struct GraphKey {
  void* ws;
  size_t ws_bytes;
  int64_t count, rows, tiles, cap, rows16, tiles16, t2, t3, c[NCLS];
  int32_t* pairs;
  int64_t pairs_cap;
  bool timing;
  bool operator==(const GraphKey& o) const {
    return timing == o.timing && ws == o.ws && ws_bytes == o.ws_bytes && count == o.count && rows == o.rows && tiles == o.tiles &&
           cap == o.cap && rows16 == o.rows16 && tiles16 == o.tiles16 && t2 == o.t2 && t3 == o.t3 &&
           std::equal(c, c + NCLS, o.c) &&
           pairs == o.pairs && pairs_cap == o.pairs_cap;
  }
};
std::mutex g_graph_mu;
GraphKey g_key{};
cudaGraphExec_t g_exec = nullptr;
int g_dev = -1;
long long g_graph_kernels = 0;  // kernels in the instantiated graph

// events around the batch's stages, recorded inside the captured graph while stage timing is on
cudaEvent_t g_bev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

int enqueue_batch(const BatchLayout& L, int64_t count, const Totals& t, int32_t* pairs, int64_t pairs_cap, int sms,
                  const BatchMaps& maps, bool timing, cudaStream_t st) {
  const int ci = (int)count;
  if (timing) CPPGB_CUDA_TRY(cudaEventRecordWithFlags(g_bev[0], st, cudaEventRecordExternal));
  batch_init_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(L.st, ci, L.g);
  CPPGB_LAUNCH_CHECK();
  CPPGB_CUDA_TRY(cudaMemsetAsync(L.pair_counts, 0, sizeof(int32_t) * (count + 1), st));
  batch_center_kernel<<<(unsigned)count, 256, 0, st>>>(L.inst, L.center);
  CPPGB_LAUNCH_CHECK();
  if (t.blk32 > 0) {
    batch_prep_kernel<<<(unsigned)t.blk32, PREP_NT, 0, st>>>(L.inst, L.pblk32, ci, L.X, L.norms, L.st, L.g, L.center);
    CPPGB_LAUNCH_CHECK();
  }
  if (t.rows16 > 0) {
    X16Set xs;
    for (int k = 0; k < NCLS; ++k) xs.p[k] = L.X16[k];
    batch_prep16_kernel<<<(unsigned)t.blk16, PREP_NT, 0, st>>>(L.inst, L.pblk16, ci, xs, L.norms16, L.H16, L.st,
                                                               L.center);
    CPPGB_LAUNCH_CHECK();
  }
  batch_bounds_kernel<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(L.inst, L.st, ci);
  CPPGB_LAUNCH_CHECK();
  if (timing) CPPGB_CUDA_TRY(cudaEventRecordWithFlags(g_bev[1], st, cudaEventRecordExternal));
  if (t.tiles16s[0] > 0) {  // path 2: four epilogue groups
    const int64_t runs = (t.tiles16s[0] + btc::TILE_RUN - 1) / btc::TILE_RUN, grid = runs < sms ? runs : sms;
    btc::batch_tc_kernel<4><<<(unsigned)grid, btc::Shape<4>::NTHREADS, btc::SMEM_BYTES<4>, st>>>(
        maps, L.inst, L.tile_offs16[0], ci, t.tiles16s[0], L.norms16, L.st, L.g, L.cand, L.cap, L.trec, L.trec_cap);
    CPPGB_LAUNCH_CHECK();
  }
  if (t.tiles16s[1] > 0) {  // path 3: two epilogue groups
    const int64_t runs = (t.tiles16s[1] + btc::TILE_RUN - 1) / btc::TILE_RUN, grid = runs < sms ? runs : sms;
    btc::batch_tc_kernel<2><<<(unsigned)grid, btc::Shape<2>::NTHREADS, btc::SMEM_BYTES<2>, st>>>(
        maps, L.inst, L.tile_offs16[1], ci, t.tiles16s[1], L.norms16, L.st, L.g, L.cand, L.cap, L.trec, L.trec_cap);
    CPPGB_LAUNCH_CHECK();
  }
  if (timing) CPPGB_CUDA_TRY(cudaEventRecordWithFlags(g_bev[2], st, cudaEventRecordExternal));
  if (t.tiles > 0) {
    const int64_t grid = t.tiles < 2 * sms ? t.tiles : 2 * sms;
    batch_dense_kernel<<<(unsigned)grid, TILE_NT, 0, st>>>(L.inst, L.tile_offs, ci, t.tiles, L.X, L.norms, L.st, L.g,
                                                           L.cand, L.cap, L.trec, L.trec_cap);
    CPPGB_LAUNCH_CHECK();
  }
  if (timing) CPPGB_CUDA_TRY(cudaEventRecordWithFlags(g_bev[3], st, cudaEventRecordExternal));
  if (t.tiles16 > 0) {
    batch_tile_recheck_kernel<<<(unsigned)(2 * sms), TILE_NT, 0, st>>>(L.inst, L.X, L.norms, L.st, L.g, L.trec,
                                                                      L.trec_cap, L.cand, L.cap, 1);
    CPPGB_LAUNCH_CHECK();
  }
  if (t.tiles + t.tiles16 > 0) {
    batch_tile_recheck_kernel<<<(unsigned)(2 * sms), TILE_NT, 0, st>>>(L.inst, L.X, L.norms, L.st, L.g, L.trec,
                                                                      L.trec_cap, L.cand, L.cap, 0);
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
                                                                      L.cap, L.res, L.counts64);
  CPPGB_LAUNCH_CHECK();
  if (timing) CPPGB_CUDA_TRY(cudaEventRecordWithFlags(g_bev[4], st, cudaEventRecordExternal));
  return CPPGB_OK;
}

}  // namespace

int set_fault_batch(int on) {
  CPPGB_CUDA_TRY(cudaMemcpyToSymbol(btc::g_fault_skip_tma, &on, sizeof on));
  return CPPGB_OK;
}
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
    if (c.path < 0 || c.path > 3) return set_error(CPPGB_ERR_ARG, "instance %lld: path must be 0, 1, 2 or 3", (long long)q);
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
  std::vector<int64_t> hto((size_t)count + 1), hb32((size_t)count + 1), hb16((size_t)count + 1);
  std::vector<int64_t> hto16[2] = {std::vector<int64_t>((size_t)count + 1), std::vector<int64_t>((size_t)count + 1)};
  int64_t xo = 0, ro = 0, to = 0, go = 0, to16[2] = {0, 0}, co[NCLS] = {0, 0, 0, 0, 0, 0}, pb32 = 0, pb16 = 0,
          cofs = 0;
  for (int64_t q = 0; q < count; ++q) {
    const cpp_instance& c = inst[q];
    BatchInst b;
    b.pts = c.pts;
    b.n = (int32_t)c.n;
    b.d = c.d;
    b.Kp = (c.d + 15) / 16 * 16;
    b.has_r = c.R >= 0.0;
    b.x_off = xo;
    b.c_off = cofs;
    b.row_off = ro;
    b.tile_off = to;
    b.rr = c.R >= 0.0 ? c.R * c.R : -1.0;
    b.rr32 = c.R >= 0.0 ? (float)(c.R * c.R) * (1.f + 0x1p-20f) : 0.f;
    b.kappa = kappa_fp32(b.Kp);
    const int64_t npad = (c.n + TILE_BM - 1) / TILE_BM * TILE_BM, nb = npad / TILE_BM;
    const int path = path_of(c);
    const int kl = path == 3 ? 1 : 0;  // tensor-core tile list (kernel) of the instance
    b.tc = path >= 2;
    b.cls = cls_of_d(c.d);
    b.nbj16 = (int32_t)((c.n + 255) / 256);
    b.nrow16 = (int32_t)nrow16_of(c.n);
    b.row_off16 = b.tc ? co[b.cls] : 0;
    b.grow_off16 = go;
    b.tile_off16 = to16[kl];
    b.kappa16 = kappa_tc(cls_kp16(b.cls));
    if (b.tc) b.tile_off = to;  // no FP32-path tiles
    hb32[(size_t)q] = pb32;
    hb16[(size_t)q] = pb16;
    hto[(size_t)q] = to;
    hto16[0][(size_t)q] = to16[0];
    hto16[1][(size_t)q] = to16[1];
    xo += npad * b.Kp;
    cofs += b.Kp;
    ro += npad;
    pb32 += prep_blocks32(npad, b.Kp);
    if (b.tc) {
      const int64_t npad16 = (c.n + 255) / 256 * 256;
      co[b.cls] += npad16;
      go += npad16;
      pb16 += prep_blocks16(npad16, cls_kp16(b.cls));
      to16[kl] += tiles16_of(c.n);
    } else {
      to += c.n >= 2 ? nb * (nb + 1) / 2 : 0;
    }
    hi[(size_t)q] = b;
  }
  hb32[(size_t)count] = pb32;
  hb16[(size_t)count] = pb16;
  hto[(size_t)count] = to;
  hto16[0][(size_t)count] = to16[0];
  hto16[1][(size_t)count] = to16[1];
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.inst, hi.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.pblk32, hb32.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.pblk16, hb16.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(L.tile_offs, hto.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
  for (int k = 0; k < 2; ++k)
    CPPGB_CUDA_TRY(
        cudaMemcpyAsync(L.tile_offs16[k], hto16[k].data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, st));
  BatchMaps maps;
  for (int k = 0; k < NCLS; ++k) {
    const int rc = encode_class_map(&maps.m[k], L.X16[k], t.crow16[k] > 256 ? t.crow16[k] : 256, k);
    if (rc) return rc;
  }
  {
    const int rc = encode_h_map(&maps.h, L.H16, t.rows16 > 256 ? t.rows16 : 256);
    if (rc) return rc;
  }

  int dev = 0, sms = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (t.tiles16s[0] > 0)
    CPPGB_CUDA_TRY(cudaFuncSetAttribute(btc::batch_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)btc::SMEM_BYTES<4>));
  if (t.tiles16s[1] > 0)
    CPPGB_CUDA_TRY(cudaFuncSetAttribute(btc::batch_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)btc::SMEM_BYTES<2>));
  bool timing = stage_timing_on();
  if (timing && !g_bev[0])
    for (auto& e : g_bev)
      if (cudaEventCreate(&e) != cudaSuccess) timing = false;
  {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    GraphKey key{ws,        ws_bytes,     count, t.rows, t.tiles,   L.cap, t.rows16, t.tiles16,
                 t.tiles16s[0], t.tiles16s[1], {},    pairs,  pairs_cap, timing};
    std::copy(t.crow16, t.crow16 + NCLS, key.c);
    if (!(g_exec && key == g_key && g_dev == dev)) {
      if (g_exec) {
        cudaGraphExecDestroy(g_exec);
        g_exec = nullptr;
      }
      cudaStream_t cap_st;
      CPPGB_CUDA_TRY(cudaStreamCreateWithFlags(&cap_st, cudaStreamNonBlocking));
      cudaGraph_t graph = nullptr;
      CPPGB_CUDA_TRY(cudaStreamBeginCapture(cap_st, cudaStreamCaptureModeThreadLocal));
      const long long before = (long long)cpp_launch_count();
      const int rc = enqueue_batch(L, count, t, pairs, pairs_cap, sms, maps, timing, cap_st);
      g_graph_kernels = (long long)cpp_launch_count() - before;
      note_launches(-g_graph_kernels);  // captured, not launched
      cudaError_t ce = cudaStreamEndCapture(cap_st, &graph);
      cudaStreamDestroy(cap_st);
      if (rc) {  // a failed enqueue: drop whatever the capture recorded
        if (ce == cudaSuccess && graph) cudaGraphDestroy(graph);
        return rc;
      }
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
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out_cpp, L.res, sizeof(cpp_pair_result) * count, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaMemcpyAsync(pair_counts, L.counts64, sizeof(int64_t) * count, cudaMemcpyDeviceToHost, st));
  // [preparation, tensor-core tiles, FP32 tiles, second pass + recheck + output]
  if (timing) set_stage_events(g_bev, 4);
  return CPPGB_OK;
}

}  // extern "C"
