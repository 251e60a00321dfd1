// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/cppgb.h"

namespace cppgb {

// ------------------------------------------------------------------ errors
int set_error(int code, const char* fmt, ...);

#define CPPGB_CUDA_TRY(expr)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return ::cppgb::set_error(CPPGB_ERR_CUDA, "%s failed: %s (%s:%d)", #expr,            \
                                cudaGetErrorString(e_), __FILE__, __LINE__);              \
  } while (0)

// Every kernel launch is followed by this check, which also counts the launch.
void note_launch();
void note_launches(long long k);  // adjusts the count (kernels captured into or replayed from a graph)
#define CPPGB_LAUNCH_CHECK()     \
  do {                           \
    ::cppgb::note_launch();      \
    CPPGB_CUDA_TRY(cudaGetLastError()); \
  } while (0)

// ------------------------------------------------------------------ workspace
// Carves a caller-provided device buffer into 256-byte aligned pieces.  With base == nullptr it
// only measures (used by the *_workspace_size queries), so both paths share one layout.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
  size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// ------------------------------------------------------------------ dense stage state
// One emitted candidate pair of the dense all-pairs stage.
struct Candidate {
  int32_t i, j;  // global row indices, i < j
  float d2f;     // filtered squared distance D~ (FP32 Gram value)
  float pad;
};

// Bound parameters of the dense stage for one problem (all in squared-distance units unless noted).
struct BoundParams {
  float eps_pair;  // eps_i + eps_j upper bound, in distance units
  float e_acc;     // bound on |D~ - |x~_i - x~_j|^2| from the Gram arithmetic
};

// Scalars of one dense all-pairs search, living in the workspace.
struct DenseScalars {
  BoundParams bp;               // written on the device once the row errors are known
  unsigned int U_bits;          // running upper bound on the best true d^2 (non-negative float bits)
  unsigned int eps_bits;        // max over rows of eps_i (distance from the exact row, float bits)
  unsigned int n2_bits;         // max over rows of |x~_i|^2 (float bits)
  unsigned int status;          // device-side flags: 1 = non-finite input, 2 = zero-variance l-mer,
                                // 4 = a bounded wait of the tensor-core stage gave up (CPPGB_ERR_TIMEOUT)
  unsigned long long n_cand;    // candidates emitted (may exceed capacity -> overflow)
  unsigned long long n_rech;    // candidates rechecked in FP64
  unsigned long long best_bits; // FP64 bits of the best rechecked d^2
  unsigned long long best_ij;   // (i << 32) | j of the best pair among equal d^2
  unsigned int ferr_bits;       // max |d2_fp64 - D~| over rechecked candidates (float bits)
  unsigned int n_surv;          // l-mer recheck: candidates that pass the final screen (listed)
  unsigned int redo;            // 1: the first pass overflowed the candidate buffer, run the second
  unsigned int pad;
};

// True distance d of a pair with filtered value D~ satisfies
//   sqrt(max(D~ - e_acc, 0)) - eps_pair  <=  d  <=  sqrt(D~ + e_acc) + eps_pair.
// upper_d2(D~) bounds d^2 from above; theta(U) is the largest D~ whose lower bound on d^2 is
// still <= U.  Both are rounded outwards by a relative pad that covers the FP32 evaluation and
// the FP64 rounding of the reference distances.
__device__ __forceinline__ float upper_d2(float D, BoundParams bp) {
  float s = sqrtf(fmaxf(D + bp.e_acc, 0.f)) + bp.eps_pair;
  return s * s * (1.f + 0x1p-19f) + 1e-30f;
}
__device__ __forceinline__ float theta_of(float U, BoundParams bp) {
  float s = sqrtf(U * (1.f + 0x1p-19f)) + bp.eps_pair;
  return (s * s + bp.e_acc) * (1.f + 0x1p-19f) + 1e-30f;
}

// atomic min/max on non-negative floats through their bit patterns (monotone for x >= 0)
__device__ __forceinline__ void atomic_min_nonneg(unsigned int* addr, float v) {
  atomicMin(addr, __float_as_uint(fmaxf(v, 0.f)));
}
__device__ __forceinline__ void atomic_max_nonneg(unsigned int* addr, float v) {
  atomicMax(addr, __float_as_uint(fmaxf(v, 0.f)));
}

// Upper-triangular tile list: tiles (bi, bj) with bj - bi >= delta among nb x nb blocks, in the
// order t -> (r, c) of a lower-triangular walk of an m x m triangle, m = nb - delta,
// bi = c, bj = r + delta.  Consecutive t share the column block bj (its tile stays in L2).
__host__ __device__ __forceinline__ int64_t tri_count(int64_t m) { return m > 0 ? m * (m + 1) / 2 : 0; }
__device__ __forceinline__ void tri_decode(int64_t t, int64_t delta, int64_t* bi, int64_t* bj) {
  int64_t r = (int64_t)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while (r > 0 && r * (r + 1) / 2 > t) --r;
  while ((r + 1) * (r + 2) / 2 <= t) ++r;
  int64_t c = t - r * (r + 1) / 2;
  *bi = c;
  *bj = r + delta;
}

// ------------------------------------------------------------------ launchers (host side)
// Point / l-mer preparation: writes X [n_pad][Kp] (FP32, FP16 or BF16 by `mode`), row norms
// |x~_i|^2 (FP32), row errors eps_i, and their maxima into the scalars.
int launch_prep_points(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, void* X,
                       int64_t n_pad, int64_t Kp, float* norms, float* eps, DenseScalars* sc,
                       cudaStream_t st);
int launch_prep_lmers(const float* series, int64_t n, int64_t l, int mode, void* X, int64_t n_pad,
                      int64_t Kp, float* norms, float* eps, DenseScalars* sc, cudaStream_t st);

// Dense all-pairs stage on FP32 CUDA cores.
// shard / nshards: only the tiles t with t % nshards == shard are evaluated (a slice of the pair space).
// gate (optional, device): the kernel returns at once unless *gate is non-zero (the second pass).
int launch_gram_simt(const float* X, int64_t n, int64_t Kp, int64_t excl, const float* norms,
                     DenseScalars* sc, Candidate* cand, int64_t cap, cudaStream_t st, int64_t shard = 0,
                     int64_t nshards = 1, const unsigned int* gate = nullptr);
// Fixed-radius variant: emits every pair i < j with D~ <= theta(rr) (rr = R^2 rounded up to FP32).
int launch_gram_simt_radius(const float* X, int64_t n, int64_t Kp, const float* norms, DenseScalars* sc,
                            Candidate* cand, int64_t cap, float rr, cudaStream_t st);
// Dense all-pairs stage on tcgen05 tensor cores (FP16 or BF16 operands).
int launch_gram_tc(const void* X, int mode, int64_t n, int64_t n_pad, int64_t Kp, int64_t excl,
                   const float* norms, DenseScalars* sc, Candidate* cand, int64_t cap, cudaStream_t st,
                   int64_t shard = 0, int64_t nshards = 1,
                   const int32_t* tlist = nullptr, const int64_t* tcount = nullptr,
                   const int32_t* perm = nullptr, int64_t excl_orig = 1, float* dump = nullptr,
                   int64_t dump_tiles = 0, const unsigned int* gate = nullptr);
// (dump != nullptr: tlist holds dump_tiles (bi, bj) pairs and each tile's raw accumulator is written
// to dump[t][128][256]; nothing else is computed.)
bool gram_tc_available();

// cuTensorMapEncodeTiled from the driver, looked up once (thread-safe); nullptr when unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn tensor_map_encoder();

// Test-only fault injection (cpp_set_fault_injection): the TMA producers of the tensor-core kernels
// of each translation unit issue no copy while `on` is non-zero (current device).
int set_fault_gram_tc(int on);
int set_fault_batch(int on);
int set_fault_match(int on);

// Tuning policy, process-wide (set through cpp_set_tuning, normally from the autotuner's cache).
// batch n-buckets (n < 1024, 4096, 16384, rest) x d-classes (the tensor-core widths d <= 16, 32, 64,
// 128, 192, 256)
constexpr int TUNE_NB = 4, TUNE_DC = 6;
int tuned_batch_path(int64_t n, int d);  // 1 (FP32 tiles), 2 or 3 (tensor-core tiles, 4- or 2-group epilogue)
int tuned_dense_band();                   // column blocks per band of the tensor-core dense stage
int tuned_dense_shape();                  // 1: 128 x 256 tiles on one CTA, 2: 256 x 256 tiles on CTA pairs

// Stage timing (cpp_set_stage_timing): whether it is on, and the last call's stage durations --
// given directly, or as intervals + 1 events recorded on the call's stream (read when asked for).
bool stage_timing_on();
void set_stage_times(const double* ms, int n);
void set_stage_events(const cudaEvent_t* ev, int intervals);

// FP64 recheck of the surviving candidates and the lexicographic (d^2, i, j) minimum.
// Source of the exact coordinates: points (dtype F32/F64, [n][ld]) or a series with l-mers.  The
// kernels read the live candidate count, min(emitted, cap), on the device (grid-stride loops).
int launch_recheck_points(const void* pts, int dtype, int64_t d, int64_t ld, DenseScalars* sc, const Candidate* cand,
                          int64_t cap, double* d2buf, cudaStream_t st);
int launch_recheck_lmers(const float* series, int64_t l, DenseScalars* sc, int32_t* surv,
                         const Candidate* cand, int64_t cap, double* d2buf, cudaStream_t st);
// Between the two passes of the dense stage: sc->redo = 1 (and the candidate count reset) when the
// first pass overflowed the buffer and found no error, else 0.
int launch_pass2_gate(DenseScalars* sc, int64_t cap, cudaStream_t st);
// The search's result from the scalars (status, pair, distances, bound terms, counts); tcount
// (optional, device) is the number of tiles a pruned search kept, of tiles_total.
int launch_dense_result(const DenseScalars* sc, int64_t cap, const int64_t* tcount, int64_t tiles_total,
                        cpp_pair_result* res, cudaStream_t st);

// Scalars reset and the bound parameters: e_acc = kappa * max_i |x~_i|^2, eps_pair = 2 max_i eps_i.
int launch_init_scalars(DenseScalars* sc, cudaStream_t st);
int launch_bounds(DenseScalars* sc, float kappa, cudaStream_t st);

// Exclusive prefix sums; out has n + 1 entries (out[n] = total); tmp holds scan_temp_elems(n) int64.
size_t scan_temp_elems(int64_t n);
int launch_exclusive_scan_i32(const int32_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t st);
int launch_exclusive_scan_i64(const int64_t* in, int64_t n, int64_t* out, int64_t* tmp, cudaStream_t st);

// Reference pruning of the tensor-core dense stage's tiles (prune.cu, gram_tc.cu).
constexpr int PRUNE_REFS = 10;  // reference rows
constexpr int PRUNE_SEEDS = 3;  // partners per row in the reference order that seed U0
struct PruneRefs {
  int64_t row[PRUNE_REFS];
};
// lo / hi [PRUNE_REFS][n_pad]: intervals of each row's exact distance to each reference;
// blo / bhi [PRUNE_REFS][n_pad / 128]: their hulls per 128-row block.
int launch_prune_intervals(const void* X, int mode, int64_t n, int64_t n_pad, int64_t Kp, const float* norms,
                           const float* eps, const DenseScalars* sc, float* lo, float* hi, float* blo, float* bhi,
                           cudaStream_t st);
// Rows (16-bit), norms and block intervals in the order `perm` (sorted position -> original row);
// rows past n are zero.
int launch_prune_permute(const void* X, int64_t n, int64_t n_pad, int64_t Kp, const float* norms,
                         const int32_t* perm, const float* lo, const float* hi, void* Xs, float* norms_s, float* blo,
                         float* bhi, cudaStream_t st);
// Sort by reference 0 and lower U with the seed pairs' bounded distances (U0).
int launch_prune_seeds(const void* X, int mode, int64_t Kp, const float* norms, const float* eps, const float* lo,
                       const float* hi, int64_t n, int64_t excl, DenseScalars* sc, int32_t* hist, int32_t* cursor,
                       int64_t* start, int64_t* tmp, int32_t* perm, cudaStream_t st);
// Tiles of the tensor-core schedule (this shard's) that the block intervals cannot exclude at the
// current bound U: flags, compacted list (increasing) and its count at list_count[0].
int64_t gram_tc_tile_count(int64_t n, int64_t n_pad, int64_t excl, int64_t shard, int64_t nshards);
int launch_gram_tc_prune_list(int64_t n, int64_t n_pad, int64_t excl, const float* blo, const float* bhi,
                              const DenseScalars* sc, int32_t* flags, int64_t* pos, int64_t* tmp, int32_t* list,
                              cudaStream_t st, int64_t shard, int64_t nshards);

// Two-locus scan.
int launch_twolocus(const uint64_t* planes, int64_t S, int64_t W, int64_t m1, int64_t m2, void* partials,
                    int64_t n_partials, twolocus_result* dev_out, cudaStream_t st, int64_t shard = 0, int64_t nshards = 1);
int64_t twolocus_num_partials(int64_t S);
int launch_twolocus_finish(const uint64_t* planes, int64_t W, int64_t m1, int64_t m2, const void* partials,
                           int64_t np, twolocus_result* dev_out, cudaStream_t st);

// Tensor-core match engine (match_tc.cu): exact integer GEMMs of 0/1/2-valued BF16 rows.
enum MatchMode { MATCH_TL_COUNT = 0, MATCH_TL_PEARSON = 1, MATCH_HAMMING_MIN = 2, MATCH_HAMMING_MAX = 3 };
struct MatchPartial {  // one per CTA: the best key (larger wins) and its pair (smaller (i, j) on ties)
  long long key;
  int32_t i, j;
};

}  // namespace cppgb
