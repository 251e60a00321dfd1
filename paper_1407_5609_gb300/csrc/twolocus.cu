// Two-locus association scan (Sec. 6): argmax over SNP pairs i < j of |P_A(i,j) - P_B(i,j)|.
//
// P_Q(i,j) is the correlation of Sec. 5.3: the fraction of the subjects of group Q whose genotypes
// at SNPs i and j match (the number of matches of Sec. 2 divided by the group size).  With the
// group sizes m1 (cases) and m2 (controls), |P_A - P_B| * m1 * m2 = |u_A * m2 - u_B * m1|, so the
// scan compares exact int64 scores.
//
// Input: per SNP and group, the one-hot code of Sec. 5.3 as bitplanes (plane 0 = [g == 1],
// plane 1 = [g == 2]; [g == 0] is implied).  Subject t matches at (i, j) iff both planes agree:
//   eq = ~(P1_i ^ P1_j) & ~(P2_i ^ P2_j),   u = popcount(eq) - (pad bits, which are 0 in both).
// The hot loop is thus two LOP3 and one POPC per 32 subjects and pair.  The full 3x3 contingency
// tables of the winning pair are then counted with AND + POPC of the planes and the marginals.
#include <mutex>

#include "common.cuh"

namespace cppgb {
namespace {

constexpr int TI = 64, TJ = 128, WC = 8, NT = 256;

struct Partial {
  long long score;  // -1: no pair in this block
  int32_t i, j;
};

__device__ __forceinline__ bool better(long long s, int i, int j, long long bs, int bi, int bj) {
  if (s != bs) return s > bs;
  if (i != bi) return i < bi;
  return j < bj;
}

__global__ void __launch_bounds__(NT, 2)
    twolocus_scan_kernel(const uint64_t* __restrict__ planes, int64_t S, int64_t W, int64_t m1, int64_t m2,
                         Partial* __restrict__ partials, int64_t shard, int64_t nshards) {
  __shared__ __align__(16) uint32_t Si[2 * WC][2][TI];
  __shared__ __align__(16) uint32_t Sj[2 * WC][2][TJ];
  __shared__ Partial red[NT / 32];

  const int64_t i0 = (int64_t)blockIdx.y * TI, j0 = (int64_t)blockIdx.x * TJ;
  const int64_t pid = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  // no pair i < j in this tile, or the tile belongs to another shard (uniform exit)
  if (j0 + TJ - 1 <= i0 || i0 >= S || pid % nshards != shard) {
    if (tid == 0) partials[pid] = Partial{-1, -1, -1};
    return;
  }

  int uA[4][8], acc[4][8];
  for (int g = 0; g < 2; ++g) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = 0;
    for (int64_t w0 = 0; w0 < W; w0 += WC) {
      const int wc = (int)(W - w0 < WC ? W - w0 : WC);
      __syncthreads();
      // stage rows: TI SNPs x 2 planes x WC words, split into 32-bit halves
#pragma unroll
      for (int q = 0; q < (TI * 2 * WC) / NT; ++q) {
        const int e = tid + q * NT, s = e / (2 * WC), p = (e / WC) & 1, w = e % WC;
        uint64_t v = 0;
        if (i0 + s < S && w < wc) v = planes[(((i0 + s) * 2 + g) * 2 + p) * W + w0 + w];
        Si[2 * w][p][s] = (uint32_t)v;
        Si[2 * w + 1][p][s] = (uint32_t)(v >> 32);
      }
#pragma unroll
      for (int q = 0; q < (TJ * 2 * WC) / NT; ++q) {
        const int e = tid + q * NT, s = e / (2 * WC), p = (e / WC) & 1, w = e % WC;
        uint64_t v = 0;
        if (j0 + s < S && w < wc) v = planes[(((j0 + s) * 2 + g) * 2 + p) * W + w0 + w];
        Sj[2 * w][p][s] = (uint32_t)v;
        Sj[2 * w + 1][p][s] = (uint32_t)(v >> 32);
      }
      __syncthreads();
      for (int h = 0; h < 2 * wc; ++h) {
        uint4 a1 = *reinterpret_cast<const uint4*>(&Si[h][0][ty * 4]);
        uint4 a2 = *reinterpret_cast<const uint4*>(&Si[h][1][ty * 4]);
        uint4 b1l = *reinterpret_cast<const uint4*>(&Sj[h][0][tx * 4]);
        uint4 b1h = *reinterpret_cast<const uint4*>(&Sj[h][0][64 + tx * 4]);
        uint4 b2l = *reinterpret_cast<const uint4*>(&Sj[h][1][tx * 4]);
        uint4 b2h = *reinterpret_cast<const uint4*>(&Sj[h][1][64 + tx * 4]);
        const uint32_t x1[4] = {a1.x, a1.y, a1.z, a1.w}, x2[4] = {a2.x, a2.y, a2.z, a2.w};
        const uint32_t y1[8] = {b1l.x, b1l.y, b1l.z, b1l.w, b1h.x, b1h.y, b1h.z, b1h.w};
        const uint32_t y2[8] = {b2l.x, b2l.y, b2l.z, b2l.w, b2h.x, b2h.y, b2h.z, b2h.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] += __popc(~((x1[r] ^ y1[c]) | (x2[r] ^ y2[c])));
      }
    }
    if (g == 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) uA[r][c] = acc[r][c];
    }
  }

  // scores: u_g = popcount - pad bits of the group (pad bits are 0 in every plane)
  const long long padA = 64 * W - m1, padB = 64 * W - m2;
  long long bs = -1;
  int bi = -1, bj = -1;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t i = i0 + ty * 4 + r;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t j = j0 + (c < 4 ? tx * 4 + c : 64 + tx * 4 + c - 4);
      if (i < j && j < S) {
        long long ua = (long long)uA[r][c] - padA, ub = (long long)acc[r][c] - padB;
        long long s = ua * m2 - ub * m1;
        s = s < 0 ? -s : s;
        if (bi < 0 || better(s, (int)i, (int)j, bs, bi, bj)) { bs = s; bi = (int)i; bj = (int)j; }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long os = __shfl_xor_sync(0xffffffffu, bs, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o), oj = __shfl_xor_sync(0xffffffffu, bj, o);
    if (oi >= 0 && (bi < 0 || better(os, oi, oj, bs, bi, bj))) { bs = os; bi = oi; bj = oj; }
  }
  if ((tid & 31) == 0) red[tid >> 5] = Partial{bs, bi, bj};
  __syncthreads();
  if (tid == 0) {
    Partial b = red[0];
    for (int w = 1; w < NT / 32; ++w) {
      Partial o = red[w];
      if (o.i >= 0 && (b.i < 0 || better(o.score, o.i, o.j, b.score, b.i, b.j))) b = o;
    }
    partials[pid] = b;
  }
}

// One block: reduce the partials, then the winner's 3x3 tables by AND + POPC and marginals.
__global__ void __launch_bounds__(NT)
    twolocus_finish_kernel(const uint64_t* __restrict__ planes, int64_t W, int64_t m1, int64_t m2,
                           const Partial* __restrict__ partials, int64_t np, twolocus_result* out) {
  __shared__ Partial red[NT];
  __shared__ unsigned long long cnt[2][8];
  const int tid = threadIdx.x;
  Partial b{-1, -1, -1};
  for (int64_t q = tid; q < np; q += NT) {
    Partial o = partials[q];
    if (o.i >= 0 && (b.i < 0 || better(o.score, o.i, o.j, b.score, b.i, b.j))) b = o;
  }
  red[tid] = b;
  if (tid < 16) cnt[tid >> 3][tid & 7] = 0;
  __syncthreads();
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (tid < s) {
      Partial o = red[tid + s], c = red[tid];
      if (o.i >= 0 && (c.i < 0 || better(o.score, o.i, o.j, c.score, c.i, c.j))) red[tid] = o;
    }
    __syncthreads();
  }
  b = red[0];
  if (b.i < 0) {
    if (tid == 0) {
      out->i = -1; out->j = -1; out->score = -1;
      for (int q = 0; q < 9; ++q) { out->countsA[q] = 0; out->countsB[q] = 0; }
      out->score_real = -1.0;
      out->status = CPPGB_OK;
      out->reserved = 0;
    }
    return;
  }
  // counts per group g: n11, n12, n21, n22, c1_i, c2_i, c1_j, c2_j  (n_ab: g_i = a, g_j = b)
  for (int g = 0; g < 2; ++g) {
    unsigned long long loc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const uint64_t* pi = planes + ((int64_t)b.i * 2 + g) * 2 * W;
    const uint64_t* pj = planes + ((int64_t)b.j * 2 + g) * 2 * W;
    for (int64_t w = tid; w < W; w += NT) {
      uint64_t i1 = pi[w], i2 = pi[W + w], j1 = pj[w], j2 = pj[W + w];
      loc[0] += __popcll(i1 & j1); loc[1] += __popcll(i1 & j2);
      loc[2] += __popcll(i2 & j1); loc[3] += __popcll(i2 & j2);
      loc[4] += __popcll(i1); loc[5] += __popcll(i2);
      loc[6] += __popcll(j1); loc[7] += __popcll(j2);
    }
    for (int q = 0; q < 8; ++q) atomicAdd(&cnt[g][q], loc[q]);
  }
  __syncthreads();
  if (tid == 0) {
    out->i = b.i; out->j = b.j; out->score = b.score;
    out->score_real = (double)b.score / ((double)m1 * (double)m2);  // |P_A - P_B| of the match measure
    out->status = CPPGB_OK;
    out->reserved = 0;
    for (int g = 0; g < 2; ++g) {
      const long long m = g == 0 ? m1 : m2;
      const long long n11 = cnt[g][0], n12 = cnt[g][1], n21 = cnt[g][2], n22 = cnt[g][3];
      const long long n10 = (long long)cnt[g][4] - n11 - n12, n20 = (long long)cnt[g][5] - n21 - n22;
      const long long n01 = (long long)cnt[g][6] - n11 - n21, n02 = (long long)cnt[g][7] - n12 - n22;
      const long long n00 = m - (n11 + n12 + n21 + n22 + n10 + n20 + n01 + n02);
      int32_t* t = g == 0 ? out->countsA : out->countsB;
      t[0] = (int32_t)n00; t[1] = (int32_t)n01; t[2] = (int32_t)n02;
      t[3] = (int32_t)n10; t[4] = (int32_t)n11; t[5] = (int32_t)n12;
      t[6] = (int32_t)n20; t[7] = (int32_t)n21; t[8] = (int32_t)n22;
    }
  }
}

}  // namespace

// Reduce per-block partials {score, i, j} (largest score, then smallest (i, j)) and count the
// winner's tables; the tensor-core scan writes the same partials.
int launch_twolocus_finish(const uint64_t* planes, int64_t W, int64_t m1, int64_t m2, const void* partials,
                           int64_t np, twolocus_result* dev_out, cudaStream_t st) {
  twolocus_finish_kernel<<<1, NT, 0, st>>>(planes, W, m1, m2, (const Partial*)partials, np, dev_out);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

int64_t twolocus_num_partials(int64_t S) {
  const int64_t gx = (S + TJ - 1) / TJ, gy = (S + TI - 1) / TI;
  return gx * gy;
}

int launch_twolocus(const uint64_t* planes, int64_t S, int64_t W, int64_t m1, int64_t m2, void* partials,
                    int64_t n_partials, twolocus_result* dev_out, cudaStream_t st, int64_t shard, int64_t nshards) {
  const int64_t gx = (S + TJ - 1) / TJ, gy = (S + TI - 1) / TI;
  if (gx * gy > n_partials) return set_error(CPPGB_ERR_CAPACITY, "internal: partials too small");
  if (gx > 0 && gy > 0) {
    if (gy > 65535) return set_error(CPPGB_ERR_ARG, "S too large for the tile grid");
    twolocus_scan_kernel<<<dim3((unsigned)gx, (unsigned)gy), NT, 0, st>>>(planes, S, W, m1, m2, (Partial*)partials,
                                                                       shard, nshards);
    CPPGB_LAUNCH_CHECK();
  }
  twolocus_finish_kernel<<<1, NT, 0, st>>>(planes, W, m1, m2, (const Partial*)partials, gx * gy, dev_out);
  CPPGB_LAUNCH_CHECK();
  return CPPGB_OK;
}

// ------------------------------------------------------------------ allocation-free variant
// twolocus_scan_noalloc keeps its scratch (the per-block partials and the device copy of the
// result) in this fixed array instead of a caller workspace.  Every device that loads the library
// holds the array until the process exits.  Layout: [0, 256) the result, [256, end) the partials.
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char twolocus_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static void* g_noalloc_ptr[kMaxDevices];
static std::mutex g_noalloc_mu;

// Device address of the array on the current device, looked up once per device.  In host code the
// array's name is only a host-side stand-in, so the kernels get this address instead.
static int noalloc_scratch_address(void** out) {
  int dev = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(CPPGB_ERR_ARG, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, twolocus_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return set_error(CPPGB_ERR_CUDA, "cudaGetSymbolAddress of the two-locus scratch failed: %s",
                       cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return CPPGB_OK;
}

static bool noalloc_fits(int64_t S) {
  return 256 + (size_t)16 * (size_t)twolocus_num_partials(S) <= kNoAllocScratchBytes;
}

// Largest S whose partials fit the array.
static int64_t noalloc_max_snps() {
  int64_t s = 0;
  while (noalloc_fits(s + 1)) ++s;
  return s;
}

}  // namespace cppgb

extern "C" int twolocus_scan_noalloc(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases,
                                     int64_t m_controls, twolocus_result* out, void* stream) {
  using namespace cppgb;
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (S < 0 || S > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "S out of range");
  if (m_cases < 1 || m_controls < 1) return set_error(CPPGB_ERR_ARG, "group sizes must be >= 1");
  if (W < (m_cases + 63) / 64 || W < (m_controls + 63) / 64)
    return set_error(CPPGB_ERR_ARG, "W = %lld words cannot hold the groups", (long long)W);
  if ((double)m_cases * (double)m_controls >= 1099511627776.0)
    return set_error(CPPGB_ERR_ARG, "m_cases * m_controls must be < 2^40");
  if (S > 0 && !planes) return set_error(CPPGB_ERR_ARG, "planes is NULL");
  if (!noalloc_fits(S))
    return set_error(CPPGB_ERR_CAPACITY,
                     "S = %lld SNPs needs more than the %zu-byte fixed scratch of twolocus_scan_noalloc "
                     "(at most %lld SNPs); use twolocus_scan with a workspace",
                     (long long)S, kNoAllocScratchBytes, (long long)noalloc_max_snps());
  void* base = nullptr;
  int rc = noalloc_scratch_address(&base);
  if (rc) return rc;
  // Nothing in the array has to start at zero: the scan writes every partial slot it later reads
  // (empty tiles write a sentinel) and the finishing kernel writes the whole result.
  cudaStream_t st = (cudaStream_t)stream;
  twolocus_result* dres = (twolocus_result*)base;
  void* partials = (char*)base + 256;
  if ((rc = launch_twolocus(planes, S, W, m_cases, m_controls, partials, twolocus_num_partials(S), dres, st)))
    return rc;
  twolocus_result h;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&h, dres, sizeof h, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  h.score_real = h.i >= 0 ? (double)h.score / ((double)m_cases * (double)m_controls) : -1.0;
  *out = h;
  return CPPGB_OK;
}
