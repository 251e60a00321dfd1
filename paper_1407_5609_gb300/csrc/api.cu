// C-ABI entry points: argument checks, workspace layout, stage sequencing, result read-back.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include "common.cuh"

#include <atomic>

namespace cppgb {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_timing{0};

// tuning policy: batch path per (n-bucket, d-class), tensor-core dense band (0: the launcher's default)
static std::atomic<int> g_batch_path[TUNE_NB * TUNE_DC];
static std::atomic<int> g_dense_band{0};
static std::atomic<int> g_dense_shape{1};
static std::atomic<int> g_tuning_init{0};

static void init_tuning() {
  int expect = 0;
  if (g_tuning_init.load() == 2 || !g_tuning_init.compare_exchange_strong(expect, 1)) {
    while (g_tuning_init.load() != 2) {
    }
    return;
  }
  // measured default: the tensor-core tiles win at every class and size this library runs; their
  // epilogue of four groups for d <= 16, of two groups from d = 17 on
  const bool tc = gram_tc_available();
  for (int k = 0; k < TUNE_NB * TUNE_DC; ++k) g_batch_path[k].store(!tc ? 1 : k % TUNE_DC == 0 ? 2 : 3);
  g_tuning_init.store(2);
}

int tuned_batch_path(int64_t n, int d) {
  init_tuning();
  const int nb = n < 1024 ? 0 : n < 4096 ? 1 : n < 16384 ? 2 : 3;
  const int dc = d <= 16 ? 0 : d <= 32 ? 1 : d <= 64 ? 2 : d <= 128 ? 3 : d <= 192 ? 4 : 5;
  const int p = g_batch_path[nb * TUNE_DC + dc].load();
  return (p >= 2 && !gram_tc_available()) ? 1 : p;
}

int tuned_dense_band() { return g_dense_band.load(); }
int tuned_dense_shape() { return g_dense_shape.load(); }

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Per-thread CUDA events for the optional stage timing of the dense searches.  A call records its
// events and leaves them pending; cpp_stage_times waits for the last one and turns them into
// stage durations.
struct StageTimer {
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  double ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int n = 0;
  const cudaEvent_t* pend = nullptr;  // events of the last call, not yet read (n + 1 of them)
  bool ready = false;
  bool init() {
    if (!ready) {
      for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) return false;
      ready = true;
    }
    return true;
  }
};
static thread_local StageTimer g_timer;

bool stage_timing_on() { return g_timing.load() != 0; }

void set_stage_times(const double* ms, int n) {
  g_timer.pend = nullptr;
  g_timer.n = n < 8 ? n : 8;
  for (int k = 0; k < g_timer.n; ++k) g_timer.ms[k] = ms[k];
}

void set_stage_events(const cudaEvent_t* ev, int intervals) {
  g_timer.pend = ev;
  g_timer.n = intervals < 8 ? intervals : 8;
}

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

namespace {

constexpr double kU32 = 5.9604644775390625e-08;  // 2^-24

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

int check_device() {
  int dev = 0, major = 0, minor = 0;
  CPPGB_CUDA_TRY(cudaGetDevice(&dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  CPPGB_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  if (major != 10 || minor != 3)
    return set_error(CPPGB_ERR_CUDA, "this library is built for sm_103a only; device %d is sm_%d%d", dev, major, minor);
  return CPPGB_OK;
}

// mode = one base mode, optionally | CPPGB_MODE_PRUNE (tensor-core filter modes only)
int base_mode(int mode) { return mode & ~CPPGB_MODE_PRUNE; }
bool is_prune(int mode) { return (mode & CPPGB_MODE_PRUNE) != 0; }
bool is_filter(int mode) {
  const int b = base_mode(mode);
  return b == CPPGB_MODE_FILTER_BF16 || b == CPPGB_MODE_FILTER_FP16;
}
bool mode_ok(int mode) { return base_mode(mode) == CPPGB_MODE_PLAIN_FP32 ? !is_prune(mode) : is_filter(mode); }

// ---------------------------------------------------------------- dense search layout
struct DenseLayout {
  int64_t n, n_pad, Kp, cap;
  size_t elem;
  DenseScalars* sc;
  float* norms;
  float* eps;
  void* X;
  // reference pruning (CPPGB_MODE_PRUNE): intervals, sort, and the rows in the sorted order
  float *plo, *phi, *pblo, *pbhi, *norms_s;
  void* Xs;
  int32_t *hist, *cursor, *perm, *flags, *list;
  int64_t *start, *pos, *ptmp;
  Candidate* cand;
  double* d2buf;
  int32_t* surv;  // the candidates that pass the final screen (l-mer recheck)
  cpp_pair_result* res;  // the result, copied to the caller's host struct
  size_t bytes;
};

// The candidate buffer takes whatever the caller's workspace holds beyond the fixed part, at
// least the default capacity that *_workspace_size() reports.
DenseLayout dense_layout(void* ws, int64_t n, int64_t d, int mode, size_t ws_bytes = 0) {
  DenseLayout L;
  L.n = n;
  L.n_pad = round_up(n > 0 ? n : 1, 256);
  L.Kp = round_up(d, is_filter(mode) ? 64 : 16);
  L.elem = is_filter(mode) ? 2 : 4;
  int64_t cap = 4 * n;
  cap = cap < (1 << 16) ? (1 << 16) : (cap > (1 << 22) ? (1 << 22) : cap);
  Carver c(ws);
  L.sc = c.take<DenseScalars>(1);
  L.norms = c.take<float>(L.n_pad);
  L.eps = c.take<float>(L.n_pad);
  L.X = c.take<char>((size_t)L.n_pad * L.Kp * L.elem);
  if (is_prune(mode)) {
    const int64_t nbi = L.n_pad / 128, tiles = nbi * (L.n_pad / 256);  // all tiles: an upper bound
    L.plo = c.take<float>((size_t)PRUNE_REFS * L.n_pad);
    L.phi = c.take<float>((size_t)PRUNE_REFS * L.n_pad);
    L.pblo = c.take<float>((size_t)PRUNE_REFS * nbi);
    L.pbhi = c.take<float>((size_t)PRUNE_REFS * nbi);
    L.hist = c.take<int32_t>(65536);
    L.cursor = c.take<int32_t>(65536);
    L.start = c.take<int64_t>(65537);
    L.perm = c.take<int32_t>(L.n_pad);
    L.flags = c.take<int32_t>(tiles);
    L.pos = c.take<int64_t>(tiles + 1);
    L.list = c.take<int32_t>(tiles);
    L.ptmp = c.take<int64_t>(scan_temp_elems(tiles > 65536 ? tiles : 65536));
    L.Xs = c.take<char>((size_t)L.n_pad * L.Kp * L.elem);
    L.norms_s = c.take<float>(L.n_pad);
  }
  const size_t fixed = c.bytes() + 1536;  // the result slot and the 256-byte rounding of the arrays below
  if (ws_bytes > fixed) {
    int64_t fit = (int64_t)((ws_bytes - fixed) / (sizeof(Candidate) + sizeof(double) + sizeof(int32_t)));
    if (fit > cap) cap = fit;
  }
  L.cap = cap;
  L.res = c.take<cpp_pair_result>(1);
  L.cand = c.take<Candidate>(L.cap);
  L.d2buf = c.take<double>(L.cap);
  L.surv = c.take<int32_t>(L.cap);
  L.bytes = c.bytes();
  return L;
}

// e_acc = kappa * max |x~|^2 bounds the Gram-form error |D~ - |x~_i - x~_j|^2|:
//   FP32 FFMA:  2 gamma_K |x||y| (dot) + gamma_K (|x|^2 + |y|^2) (norms) + 3 roundings of the
//               epilogue on magnitudes <= 2 (|x|^2 + |y|^2)  ->  (4 gamma_K + 8u) max|x|^2
//   tensor cores (exact 16-bit products, FP32 accumulation whose internal rounding is not
//               specified to be round-to-nearest): the dot term padded to 2 * K * 2^-22 |x||y|,
//               norms from the prep's two-level sums (22u each) and the same epilogue terms.
float kappa_for(int mode, int64_t Kp) {
  mode = base_mode(mode);
  double K = (double)Kp;
  if (!is_filter(mode)) {
    double g = K * kU32 / (1.0 - K * kU32);
    return (float)((4.0 * g + 8.0 * kU32) * 1.01);
  }
  return (float)((2.0 * 2.0 * K * 0x1p-22 + 2.0 * 22.0 * kU32 + 8.0 * kU32) * 1.01);
}

struct Source {
  bool lmers;
  const void* pts;
  int dtype;
  int64_t d, ld;
  const float* series;
  int64_t l;
};

int dense_search(const Source& src, int64_t n, int64_t d, int64_t excl, int mode, cpp_pair_result* out, void* ws,
                 size_t ws_bytes, cudaStream_t st, int64_t shard = 0, int64_t nshards = 1) {
  DenseLayout L = dense_layout(ws, n, d, mode, ws_bytes);
  if (ws_bytes < L.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.bytes);
  if (((uintptr_t)ws & 255) != 0) return set_error(CPPGB_ERR_ARG, "workspace must be 256-byte aligned");
  if (is_filter(mode) && !gram_tc_available())
    return set_error(CPPGB_ERR_ARG, "tensor-core filter modes are not available in this build");

  const bool timing = g_timing.load() != 0 && g_timer.init();
  const bool prune = is_prune(mode);
  mode = base_mode(mode);
  g_timer.n = 0;
  g_timer.pend = nullptr;
  if (timing) CPPGB_CUDA_TRY(cudaEventRecord(g_timer.ev[0], st));
  int rc;
  if ((rc = launch_init_scalars(L.sc, st))) return rc;
  if (src.lmers)
    rc = launch_prep_lmers(src.series, n, src.l, mode, L.X, L.n_pad, L.Kp, L.norms, L.eps, L.sc, st);
  else
    rc = launch_prep_points(src.pts, src.dtype, n, d, src.ld, mode, L.X, L.n_pad, L.Kp, L.norms, L.eps, L.sc, st);
  if (rc) return rc;
  if ((rc = launch_bounds(L.sc, kappa_for(mode, L.Kp), st))) return rc;

  // Reference pruning: distance intervals to the references, a seed bound U0 from pairs that are
  // neighbours in the order of reference 0, then the list of tiles the intervals cannot exclude
  // (its length stays on the device).
  const int32_t* tlist = nullptr;
  const int64_t* tcount = nullptr;
  int64_t tiles_total = -1;
  const void* Xd = L.X;          // the dense stage's rows, norms, original-index map and schedule exclusion
  const float* normsd = L.norms;
  const int32_t* permd = nullptr;
  int64_t excl_sched = excl;
  if (prune && n >= 2) {
    if ((rc = launch_prune_intervals(L.X, mode, n, L.n_pad, L.Kp, L.norms, L.eps, L.sc, L.plo, L.phi, L.pblo, L.pbhi,
                                     st)))
      return rc;
    if ((rc = launch_prune_seeds(L.X, mode, L.Kp, L.norms, L.eps, L.plo, L.phi, n, excl, L.sc, L.hist, L.cursor,
                                 L.start, L.ptmp, L.perm, st)))
      return rc;
    // One search: the rows go into the order of their distance to reference 0 (as in Algorithm MK),
    // which makes the blocks' intervals narrow.  The counting sort's order inside a bucket is not
    // reproducible, so shards of a search (which must partition the same pairs) keep the original order.
    if (nshards == 1) {
      if ((rc = launch_prune_permute(L.X, n, L.n_pad, L.Kp, L.norms, L.perm, L.plo, L.phi, L.Xs, L.norms_s, L.pblo,
                                     L.pbhi, st)))
        return rc;
      Xd = L.Xs;
      normsd = L.norms_s;
      permd = L.perm;
      excl_sched = 1;
    }
    tiles_total = gram_tc_tile_count(n, L.n_pad, excl_sched, shard, nshards);
    if ((rc = launch_gram_tc_prune_list(n, L.n_pad, excl_sched, L.pblo, L.pbhi, L.sc, L.flags, L.pos, L.ptmp, L.list,
                                        st, shard, nshards)))
      return rc;
    tlist = L.list;
    tcount = L.pos + tiles_total;
  }
  if (timing) CPPGB_CUDA_TRY(cudaEventRecord(g_timer.ev[1], st));

  // Two passes of the dense stage; the second runs (on the device's decision) only when the first
  // overflowed the candidate buffer, and then emits against the final bound U.
  for (int pass = 0; pass < 2; ++pass) {
    const unsigned int* gate = pass == 0 ? nullptr : &L.sc->redo;
    if (pass == 1 && (rc = launch_pass2_gate(L.sc, L.cap, st))) return rc;
    if (is_filter(mode))
      rc = launch_gram_tc(Xd, mode, n, L.n_pad, L.Kp, excl_sched, normsd, L.sc, L.cand, L.cap, st, shard, nshards,
                          tlist, tcount, permd, excl, nullptr, 0, gate);
    else
      rc = launch_gram_simt((const float*)L.X, n, L.Kp, excl, L.norms, L.sc, L.cand, L.cap, st, shard, nshards, gate);
    if (rc) return rc;
  }
  if (timing) CPPGB_CUDA_TRY(cudaEventRecord(g_timer.ev[2], st));
  if (src.lmers)
    rc = launch_recheck_lmers(src.series, src.l, L.sc, L.surv, L.cand, L.cap, L.d2buf, st);
  else
    rc = launch_recheck_points(src.pts, src.dtype, d, src.ld, L.sc, L.cand, L.cap, L.d2buf, st);
  if (rc) return rc;
  if (timing) CPPGB_CUDA_TRY(cudaEventRecord(g_timer.ev[3], st));
  if ((rc = launch_dense_result(L.sc, L.cap, tcount, tiles_total, L.res, st))) return rc;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out, L.res, sizeof *out, cudaMemcpyDeviceToHost, st));
  if (timing) set_stage_events(g_timer.ev, 3);  // [prep (+ pruning set-up), dense stage, FP64 recheck]
  return CPPGB_OK;
}

}  // namespace
}  // namespace cppgb

using namespace cppgb;

extern "C" {

const char* cpp_last_error(void) { return g_err; }

int cpp_filter_available(void) { return gram_tc_available() ? 1 : 0; }

int cpp_set_fault_injection(int kind) {
  g_err[0] = 0;
  if (kind != CPPGB_FAULT_NONE && kind != CPPGB_FAULT_SKIP_TMA)
    return set_error(CPPGB_ERR_ARG, "unknown fault kind %d", kind);
  const int on = kind == CPPGB_FAULT_SKIP_TMA ? 1 : 0;
  int rc;
  if ((rc = set_fault_gram_tc(on)) || (rc = set_fault_batch(on)) || (rc = set_fault_match(on))) return rc;
  return CPPGB_OK;
}

int cpp_set_tuning(int kind, const int32_t* values, int count) {
  init_tuning();
  if (kind == CPPGB_TUNE_BATCH_PATH) {
    if (!values || count != TUNE_NB * TUNE_DC) return set_error(CPPGB_ERR_ARG, "batch path table needs %d entries", TUNE_NB * TUNE_DC);
    for (int k = 0; k < count; ++k)
      if (values[k] < 1 || values[k] > 3) return set_error(CPPGB_ERR_ARG, "batch path entries must be 1, 2 or 3");
    for (int k = 0; k < count; ++k) g_batch_path[k].store(values[k]);
    return CPPGB_OK;
  }
  if (kind == CPPGB_TUNE_DENSE_BAND) {
    if (!values || count != 1 || values[0] < 1 || values[0] > 4096) return set_error(CPPGB_ERR_ARG, "dense band must be one value in [1, 4096]");
    g_dense_band.store(values[0]);
    return CPPGB_OK;
  }
  if (kind == CPPGB_TUNE_DENSE_SHAPE) {
    if (!values || count != 1 || (values[0] != 1 && values[0] != 2))
      return set_error(CPPGB_ERR_ARG, "dense tile shape must be one value, 1 or 2");
    g_dense_shape.store(values[0]);
    return CPPGB_OK;
  }
  return set_error(CPPGB_ERR_ARG, "unknown tuning kind %d", kind);
}

int cpp_get_tuning(int kind, int32_t* values, int count) {
  init_tuning();
  if (kind == CPPGB_TUNE_BATCH_PATH) {
    if (!values || count < TUNE_NB * TUNE_DC) return set_error(CPPGB_ERR_ARG, "batch path table needs %d entries", TUNE_NB * TUNE_DC);
    for (int k = 0; k < TUNE_NB * TUNE_DC; ++k) values[k] = g_batch_path[k].load();
    return CPPGB_OK;
  }
  if (kind == CPPGB_TUNE_DENSE_BAND) {
    if (!values || count < 1) return set_error(CPPGB_ERR_ARG, "dense band needs one entry");
    values[0] = g_dense_band.load();
    return CPPGB_OK;
  }
  if (kind == CPPGB_TUNE_DENSE_SHAPE) {
    if (!values || count < 1) return set_error(CPPGB_ERR_ARG, "dense tile shape needs one entry");
    values[0] = g_dense_shape.load();
    return CPPGB_OK;
  }
  return set_error(CPPGB_ERR_ARG, "unknown tuning kind %d", kind);
}

void cpp_set_stage_timing(int on) { g_timing.store(on ? 1 : 0); }

int cpp_stage_times(double* ms, int cap) {
  if (g_timer.pend) {  // the last call's events: wait for them, then take the intervals
    const cudaEvent_t* ev = g_timer.pend;
    g_timer.pend = nullptr;
    if (cudaEventSynchronize(ev[g_timer.n]) != cudaSuccess) {
      g_timer.n = 0;
      return 0;
    }
    for (int k = 0; k < g_timer.n; ++k) {
      float v = 0.f;
      if (cudaEventElapsedTime(&v, ev[k], ev[k + 1]) != cudaSuccess) v = 0.f;
      g_timer.ms[k] = v;
    }
  }
  int k = 0;
  for (; k < g_timer.n && k < cap; ++k) ms[k] = g_timer.ms[k];
  return k;
}

int64_t cpp_launch_count(void) { return (int64_t)g_launches.load(); }


// ------------------------------------------------------------------ closest pair
size_t cpp_closest_pair_workspace_size(int64_t n, int64_t d, int mode) {
  if (n < 0 || d < 1 || !mode_ok(mode)) return 0;
  return dense_layout(nullptr, n, d, mode).bytes;
}

int cpp_closest_pair(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, cpp_pair_result* out,
                     void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (n < 0 || n > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "n out of range (%lld)", (long long)n);
  if (d < 1 || d > 4096 || ld < d) return set_error(CPPGB_ERR_ARG, "need 1 <= d <= 4096 and ld >= d");
  if (dtype != CPPGB_F32 && dtype != CPPGB_F64) return set_error(CPPGB_ERR_ARG, "dtype must be CPPGB_F32 or CPPGB_F64");
  if (!mode_ok(mode)) return set_error(CPPGB_ERR_ARG, "unknown mode %d", mode);
  if (n > 0 && !pts) return set_error(CPPGB_ERR_ARG, "pts is NULL");
  if (!ws) return set_error(CPPGB_ERR_ARG, "workspace is NULL");
  int rc = check_device();
  if (rc) return rc;
  Source src{false, pts, dtype, d, ld, nullptr, 0};
  return dense_search(src, n, d, 1, mode, out, ws, ws_bytes, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ tensor-core Gram dump (diagnostics)
int cpp_gram_tile_dump(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, const int32_t* tiles,
                       int64_t ntiles, float* S, void* rows, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (n < 1 || n > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "n out of range (%lld)", (long long)n);
  if (d < 1 || d > 4096 || ld < d) return set_error(CPPGB_ERR_ARG, "need 1 <= d <= 4096 and ld >= d");
  if (dtype != CPPGB_F32 && dtype != CPPGB_F64) return set_error(CPPGB_ERR_ARG, "dtype must be CPPGB_F32 or CPPGB_F64");
  if (mode != CPPGB_MODE_FILTER_BF16 && mode != CPPGB_MODE_FILTER_FP16)
    return set_error(CPPGB_ERR_ARG, "mode must be CPPGB_MODE_FILTER_BF16 or CPPGB_MODE_FILTER_FP16");
  if (!pts || !S || !ws || (ntiles > 0 && !tiles)) return set_error(CPPGB_ERR_ARG, "NULL argument");
  if (!gram_tc_available()) return set_error(CPPGB_ERR_ARG, "tensor-core kernels are not available in this build");
  DenseLayout L = dense_layout(ws, n, d, mode, ws_bytes);
  if (ws_bytes < L.bytes)
    return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu bytes given, %zu needed", ws_bytes, L.bytes);
  if (((uintptr_t)ws & 255) != 0) return set_error(CPPGB_ERR_ARG, "workspace must be 256-byte aligned");
  if (ntiles < 0 || ntiles * 2 * (int64_t)sizeof(int32_t) > L.cap * (int64_t)sizeof(Candidate))
    return set_error(CPPGB_ERR_ARG, "ntiles out of range");
  const int64_t nbi = L.n_pad / 128, nbj = L.n_pad / 256;
  for (int64_t t = 0; t < ntiles; ++t)
    if (tiles[2 * t] < 0 || tiles[2 * t] >= nbi || tiles[2 * t + 1] < 0 || tiles[2 * t + 1] >= nbj)
      return set_error(CPPGB_ERR_ARG, "tile %lld = (%d, %d) outside the %lld x %lld blocks", (long long)t,
                       tiles[2 * t], tiles[2 * t + 1], (long long)nbi, (long long)nbj);
  int rc = check_device();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t* dlist = reinterpret_cast<int32_t*>(L.cand);  // the candidate buffer is unused by a dump
  if (ntiles > 0)
    CPPGB_CUDA_TRY(cudaMemcpyAsync(dlist, tiles, (size_t)ntiles * 2 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if ((rc = launch_init_scalars(L.sc, st))) return rc;
  if ((rc = launch_prep_points(pts, dtype, n, d, ld, mode, L.X, L.n_pad, L.Kp, L.norms, L.eps, L.sc, st))) return rc;
  if ((rc = launch_bounds(L.sc, kappa_for(mode, L.Kp), st))) return rc;
  if ((rc = launch_gram_tc(L.X, mode, n, L.n_pad, L.Kp, 1, L.norms, L.sc, L.cand, L.cap, st, 0, 1, dlist, nullptr,
                           nullptr, 1, S, ntiles)))
    return rc;
  if (rows) CPPGB_CUDA_TRY(cudaMemcpyAsync(rows, L.X, (size_t)L.n_pad * L.Kp * L.elem, cudaMemcpyDeviceToDevice, st));
  DenseScalars h;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(&h, L.sc, sizeof h, cudaMemcpyDeviceToHost, st));
  CPPGB_CUDA_TRY(cudaStreamSynchronize(st));
  if (h.status & 1u) return set_error(CPPGB_ERR_NUMERIC, "non-finite input value");
  if (h.status & 4u) return set_error(CPPGB_ERR_TIMEOUT, "a tensor-core pipeline wait timed out");
  return CPPGB_OK;
}

// ------------------------------------------------------------------ motif pair
size_t tsmm_motif_workspace_size(int64_t N, int64_t l, int mode) {
  if (l < 2 || N < l || !mode_ok(mode)) return 0;
  return dense_layout(nullptr, N - l + 1, l, mode).bytes;
}

int tsmm_motif(const float* series, int64_t N, int64_t l, int64_t excl, int mode, cpp_pair_result* out, void* ws,
               size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (!series) return set_error(CPPGB_ERR_ARG, "series is NULL");
  if (l < 2 || l > 4096 || N < l) return set_error(CPPGB_ERR_ARG, "need 2 <= l <= 4096 and N >= l");
  if (N - l + 1 > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "too many l-mers");
  if (excl < 1) return set_error(CPPGB_ERR_ARG, "excl must be >= 1");
  if (!mode_ok(mode)) return set_error(CPPGB_ERR_ARG, "unknown mode %d", mode);
  if (!ws) return set_error(CPPGB_ERR_ARG, "workspace is NULL");
  int rc = check_device();
  if (rc) return rc;
  Source src{true, nullptr, CPPGB_F32, l, l, series, l};
  return dense_search(src, N - l + 1, l, excl, mode, out, ws, ws_bytes, (cudaStream_t)stream);
}

// ------------------------------------------------------------------ shards of the pair space
static int shard_ok(int64_t shard, int64_t nshards) {
  if (nshards < 1 || shard < 0 || shard >= nshards)
    return set_error(CPPGB_ERR_ARG, "need 0 <= shard < nshards (got %lld of %lld)", (long long)shard,
                     (long long)nshards);
  return CPPGB_OK;
}

int cpp_closest_pair_shard(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, int64_t shard,
                           int64_t nshards, cpp_pair_result* out, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  int rc = shard_ok(shard, nshards);
  if (rc) return rc;
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (n < 0 || n > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "n out of range (%lld)", (long long)n);
  if (d < 1 || d > 4096 || ld < d) return set_error(CPPGB_ERR_ARG, "need 1 <= d <= 4096 and ld >= d");
  if (dtype != CPPGB_F32 && dtype != CPPGB_F64) return set_error(CPPGB_ERR_ARG, "dtype must be CPPGB_F32 or CPPGB_F64");
  if (!mode_ok(mode)) return set_error(CPPGB_ERR_ARG, "unknown mode %d", mode);
  if (n > 0 && !pts) return set_error(CPPGB_ERR_ARG, "pts is NULL");
  if (!ws) return set_error(CPPGB_ERR_ARG, "workspace is NULL");
  if ((rc = check_device())) return rc;
  Source src{false, pts, dtype, d, ld, nullptr, 0};
  return dense_search(src, n, d, 1, mode, out, ws, ws_bytes, (cudaStream_t)stream, shard, nshards);
}

int tsmm_motif_shard(const float* series, int64_t N, int64_t l, int64_t excl, int mode, int64_t shard,
                     int64_t nshards, cpp_pair_result* out, void* ws, size_t ws_bytes, void* stream) {
  g_err[0] = 0;
  int rc = shard_ok(shard, nshards);
  if (rc) return rc;
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (!series) return set_error(CPPGB_ERR_ARG, "series is NULL");
  if (l < 2 || l > 4096 || N < l) return set_error(CPPGB_ERR_ARG, "need 2 <= l <= 4096 and N >= l");
  if (N - l + 1 > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "too many l-mers");
  if (excl < 1) return set_error(CPPGB_ERR_ARG, "excl must be >= 1");
  if (!mode_ok(mode)) return set_error(CPPGB_ERR_ARG, "unknown mode %d", mode);
  if (!ws) return set_error(CPPGB_ERR_ARG, "workspace is NULL");
  if ((rc = check_device())) return rc;
  Source src{true, nullptr, CPPGB_F32, l, l, series, l};
  return dense_search(src, N - l + 1, l, excl, mode, out, ws, ws_bytes, (cudaStream_t)stream, shard, nshards);
}

// ------------------------------------------------------------------ two-locus
size_t twolocus_scan_workspace_size(int64_t S, int64_t W) {
  if (S < 0 || W < 1) return 0;
  Carver c(nullptr);
  c.take<twolocus_result>(1);
  c.take<char>((size_t)16 * (size_t)(twolocus_num_partials(S) > 0 ? twolocus_num_partials(S) : 1));
  return c.bytes();
}

static int twolocus_common(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                           int64_t shard, int64_t nshards, twolocus_result* out, void* ws, size_t ws_bytes,
                           void* stream) {
  g_err[0] = 0;
  if (!out) return set_error(CPPGB_ERR_ARG, "out is NULL");
  if (S < 0 || S > 0x7fffffffLL) return set_error(CPPGB_ERR_ARG, "S out of range");
  if (m_cases < 1 || m_controls < 1) return set_error(CPPGB_ERR_ARG, "group sizes must be >= 1");
  if (W < (m_cases + 63) / 64 || W < (m_controls + 63) / 64)
    return set_error(CPPGB_ERR_ARG, "W = %lld words cannot hold the groups", (long long)W);
  if ((double)m_cases * (double)m_controls >= 1099511627776.0)
    return set_error(CPPGB_ERR_ARG, "m_cases * m_controls must be < 2^40");
  if (S > 0 && !planes) return set_error(CPPGB_ERR_ARG, "planes is NULL");
  if (!ws) return set_error(CPPGB_ERR_ARG, "workspace is NULL");
  size_t need = twolocus_scan_workspace_size(S, W);
  if (ws_bytes < need) return set_error(CPPGB_ERR_CAPACITY, "workspace too small: %zu given, %zu needed", ws_bytes, need);
  if (((uintptr_t)ws & 255) != 0) return set_error(CPPGB_ERR_ARG, "workspace must be 256-byte aligned");
  int rc = check_device();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Carver c(ws);
  twolocus_result* dres = c.take<twolocus_result>(1);
  const int64_t np = twolocus_num_partials(S);
  void* partials = c.take<char>((size_t)16 * (size_t)(np > 0 ? np : 1));
  if ((rc = launch_twolocus(planes, S, W, m_cases, m_controls, partials, np, dres, st, shard, nshards))) return rc;
  CPPGB_CUDA_TRY(cudaMemcpyAsync(out, dres, sizeof *out, cudaMemcpyDeviceToHost, st));
  return CPPGB_OK;
}

int twolocus_scan(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                  twolocus_result* out, void* ws, size_t ws_bytes, void* stream) {
  return twolocus_common(planes, S, W, m_cases, m_controls, 0, 1, out, ws, ws_bytes, stream);
}

int twolocus_scan_shard(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                        int64_t shard, int64_t nshards, twolocus_result* out, void* ws, size_t ws_bytes,
                        void* stream) {
  if (nshards < 1 || nshards > 65536 || shard < 0 || shard >= nshards) {
    g_err[0] = 0;
    return set_error(CPPGB_ERR_ARG, "need 0 <= shard < nshards <= 65536");
  }
  return twolocus_common(planes, S, W, m_cases, m_controls, shard, nshards, out, ws, ws_bytes, stream);
}

}  // extern "C"
