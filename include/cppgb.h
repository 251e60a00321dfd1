/*
 * cppgb.h -- exact closest-pair family on GB300 (sm_103a): C ABI.
 *
 * Implements the exact (brute-force-equivalent) search of Rajasekaran & Pathak,
 * "Efficient Algorithms for the Closest Pair Problem and Applications":
 *   - closest pair (CPP) of n points in R^d           (Sec. 3 problem statement; distance of Sec. 2)
 *   - motif pair of a time series: closest pair of its z-normalised l-mers  (Sec. 2, Sec. 3)
 *   - fixed-radius near neighbours N(i) for all i     (Sec. 3.5)
 *   - two-locus association: argmax_{i,j} |P_A(i,j) - P_B(i,j)|  (Sec. 6, correlation of Sec. 5.3)
 *
 * Conventions shared by every entry point
 *   - Data pointers (points, series, planes, outputs named as device) are DEVICE pointers
 *     owned by the caller.  Result structs (`out`) and scalar out-params are HOST pointers.
 *   - `ws` is a caller-provided DEVICE workspace of at least the matching *_workspace_size()
 *     bytes, 256-byte aligned.  The library allocates nothing on these paths.  For the dense
 *     searches (cpp_closest_pair, tsmm_motif) any workspace beyond that size enlarges the
 *     candidate buffer of the filter stage.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls are asynchronous:
 *     each enqueues its kernels on `stream` and returns; the result struct is written to the
 *     caller's host memory by a copy on the same stream and is valid after the stream has been
 *     synchronised (pass pinned host memory for the call to return before the work is done;
 *     with pageable memory the copy itself waits).  Exceptions, which wait for the stream before
 *     returning: twolocus_scan_noalloc, mlba_pair, cpp_gram_tile_dump, cpp_measure_alu_peaks.
 *     Calls on one stream are serialised; a workspace must not be shared by calls that may run
 *     at the same time, and the inputs, workspace and result memory must stay valid until the
 *     stream reaches the call's end.
 *   - Errors found before any work is enqueued (arguments, workspace size, launch failures)
 *     are the return value.  Errors that only the device can see (a non-finite input, a
 *     timed-out wait, more candidates or pairs than the buffers hold) are reported in the
 *     result's `status` field (CPPGB_OK otherwise), valid after the stream sync.
 *   - Indices are 0-based (the paper counts from 1).  Pairs are reported with i < j.
 *   - Ties are broken towards the lexicographically smallest (i, j).
 *   - Return value: CPPGB_OK or one of the error codes below; cpp_last_error() then
 *     returns a message (per calling thread).  No exception crosses this boundary.
 */
#ifndef CPPGB_H
#define CPPGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define CPPGB_OK 0
#define CPPGB_ERR_ARG 1      /* bad size, pointer, alignment or mode */
#define CPPGB_ERR_CAPACITY 2 /* workspace or output buffer too small; required size reported */
#define CPPGB_ERR_TIMEOUT 3  /* a bounded device-side wait gave up */
#define CPPGB_ERR_CUDA 4     /* a CUDA runtime call failed */
#define CPPGB_ERR_NUMERIC 5  /* e.g. an l-mer with zero variance, or a non-finite input */

/* element type of a point array */
#define CPPGB_F32 0
#define CPPGB_F64 1

/* how the dense all-pairs stage evaluates distances; every mode returns the exact answer */
#define CPPGB_MODE_PLAIN_FP32 0  /* FP32 CUDA-core Gram tiles, rigorous bound, FP64 recheck */
#define CPPGB_MODE_FILTER_BF16 1 /* BF16 tensor-core Gram tiles (tcgen05), bound, FP64 recheck */
#define CPPGB_MODE_FILTER_FP16 2 /* FP16 tensor-core Gram tiles (tcgen05), bound, FP64 recheck */
/* OR'd into a FILTER mode: reference pruning of whole tiles (the reference-point bound of
 * Algorithms MK / MPR, Sec. 3.1-3.3).  Ten reference rows give every row an interval holding its
 * exact distance to each reference; a 128 x 256 tile whose row and column intervals are, for some
 * reference, further apart than sqrt(U0) is skipped, U0 being the exact best d^2 of seed pairs
 * (rows adjacent in the order of their distance to the first reference, as in Algorithm MK).  The
 * answer is the same as without pruning. */
#define CPPGB_MODE_PRUNE 0x100

/* Result of a closest-pair style search. */
typedef struct {
  int64_t i, j;          /* the pair, i < j; both -1 when no pair is valid */
  double dist;           /* FP64 Euclidean distance of the pair (Sec. 2) */
  double dist2;          /* its square, summed in coordinate order in FP64 */
  double filter_err;     /* max |dist2_fp64 - D~| over the rechecked candidates (D~: the filter's value) */
  double filter_bound;   /* final upper bound U on dist2 reached by the dense stage */
  int64_t n_emitted;     /* candidate pairs the dense stage emitted (on CPPGB_ERR_CAPACITY: the number
                            a workspace would have to hold, 28 bytes each) */
  int64_t n_rechecked;   /* candidates whose lower bound met the final upper bound (FP64-rechecked) */
  double filter_e_acc;   /* e_acc: bound on |D~ - |x~_i - x~_j|^2| from the Gram arithmetic (x~: stored rows) */
  double filter_eps;     /* eps_pair: bound on | |x_i - x_j| - |x~_i - x~_j| | from the rows' rounding, so
                            |dist2 - D~| <= e_acc + 2 eps sqrt(D~ + e_acc) + eps^2 for every rechecked pair */
  int64_t tiles_kept;    /* CPPGB_MODE_PRUNE: tiles of the dense stage evaluated; -1 otherwise */
  int64_t tiles_total;   /* CPPGB_MODE_PRUNE: tiles of the schedule; -1 otherwise */
  int32_t status;        /* CPPGB_OK, or the error the device found (valid after the stream sync) */
  int32_t reserved;
} cpp_pair_result;

/*
 * cpp_closest_pair -- closest pair of n points in R^d: the general form of the problem stated at
 * the start of Sec. 3, with the Euclidean distance of Sec. 2.
 *   pts    device, row-major [n][ld] of `dtype` (CPPGB_F32 or CPPGB_F64); d <= ld.
 *   n      number of points (0 and 1 give i = j = -1).   d in [1, 4096].
 *   mode   CPPGB_MODE_*.
 *   out    host (pinned for an asynchronous call); valid after the stream sync.
 * Errors (return value): CPPGB_ERR_ARG (sizes, null pointers, mode), CPPGB_ERR_CAPACITY (ws too
 *         small), CPPGB_ERR_CUDA.
 * Errors (out->status): CPPGB_ERR_CAPACITY (more candidate pairs tie within the filter's error
 *         bound than the workspace holds: out->n_emitted holds the number needed, 28 bytes each),
 *         CPPGB_ERR_NUMERIC (non-finite coordinates), CPPGB_ERR_TIMEOUT (a bounded wait of the
 *         tensor-core stage gave up).
 */
size_t cpp_closest_pair_workspace_size(int64_t n, int64_t d, int mode);
int cpp_closest_pair(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode,
                     cpp_pair_result* out, void* ws, size_t ws_bytes, void* stream);

/*
 * tsmm_motif -- time-series motif pair: of all pairs of l-mers of the series, the pair at least
 * distance (Sec. 3; l-mers T_i = a_i..a_{i+l-1} as defined in Sec. 2).  Each l-mer is z-normalised with its own
 * mean and population standard deviation before the Euclidean distance is taken; a pair (i, j)
 * is eligible when j - i >= excl (trivial-match exclusion).
 *   series device FP32 [N].   l in [2, 4096], N >= l.   excl >= 1.
 *   out    host; dist2 is the FP64 squared distance of the z-normalised l-mers.
 * Errors as for cpp_closest_pair; out->status = CPPGB_ERR_NUMERIC also for an l-mer of zero
 *         variance.
 */
size_t tsmm_motif_workspace_size(int64_t N, int64_t l, int mode);
int tsmm_motif(const float* series, int64_t N, int64_t l, int64_t excl, int mode,
               cpp_pair_result* out, void* ws, size_t ws_bytes, void* stream);

/*
 * Shards of the pair space (for running one search across several GPUs or calls).  The dense stage
 * evaluates the pairs tile by tile; shard s of nshards (0 <= s < nshards) evaluates only the tiles
 * t with t mod nshards == s and returns the exact best pair among them (i = j = -1 when it has
 * none), with the same conventions as the unsharded call.  The lexicographically smallest
 * (dist2, i, j) over the results of all nshards shards is exactly the result of the unsharded
 * call; combining them is the caller's one exchange step.  Workspace sizes are those of the
 * unsharded calls.  Errors as for the unsharded calls, plus CPPGB_ERR_ARG for a bad shard.
 */
int cpp_closest_pair_shard(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, int64_t shard,
                           int64_t nshards, cpp_pair_result* out, void* ws, size_t ws_bytes, void* stream);
int tsmm_motif_shard(const float* series, int64_t N, int64_t l, int64_t excl, int mode, int64_t shard,
                     int64_t nshards, cpp_pair_result* out, void* ws, size_t ws_bytes, void* stream);

/* Result of a two-locus scan. */
typedef struct {
  int64_t i, j;        /* best SNP pair, i < j; -1 when S < 2 */
  int64_t score;       /* |u_A * m_controls - u_B * m_cases| = |P_A - P_B| * m_cases * m_controls */
  int32_t countsA[9];  /* cases: countsA[3a+b] = #subjects with g_i = a, g_j = b */
  int32_t countsB[9];  /* controls, same layout */
  double score_real;   /* the score as a real number: |P_A - P_B| (matches), |r_A - r_B| (Pearson) */
  int32_t status;      /* CPPGB_OK, or the error the device found (valid after the stream sync) */
  int32_t reserved;
} twolocus_result;

/*
 * twolocus_scan -- two-locus association (Sec. 6): the SNP pair maximising |P_A(i,j) - P_B(i,j)|,
 * where P_Q(i,j) is the fraction of subjects of group Q whose genotypes at SNPs i and j match
 * (the correlation of Sec. 5.3; matches as in Sec. 2).  Exact integer arithmetic.
 *   planes device uint64 [S][2 groups][2 planes][W]: group 0 = cases (m_cases subjects),
 *          group 1 = controls; plane 0 has bit [g == 1], plane 1 bit [g == 2] (the one-hot code
 *          of Sec. 5.3 with the g == 0 plane implied); bit b of word w is subject 64w+b; bits
 *          at or beyond the group size must be 0.
 *   W      words per plane, W >= ceil(max(m_cases, m_controls) / 64).
 *   out    host; counts are the full 3x3 tables of the winning pair.
 * Errors: CPPGB_ERR_ARG (sizes: S < 2^31, m_cases * m_controls < 2^40), CPPGB_ERR_CAPACITY, CPPGB_ERR_CUDA.
 */
size_t twolocus_scan_workspace_size(int64_t S, int64_t W);
int twolocus_scan(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                  twolocus_result* out, void* ws, size_t ws_bytes, void* stream);

/*
 * twolocus_scan_noalloc -- the same scan and result as twolocus_scan, without a workspace.  The
 * paper has no counterpart; this exists for callers that cannot allocate device memory: code
 * embedded in a host framework that owns all device memory and offers no allocation hook, and
 * latency-critical loops that cannot afford cudaMalloc/cudaFree, which may synchronise the whole
 * device.  Its scratch is a fixed 1 MiB array inside the library, so S is limited to 23,104 SNPs
 * (larger S returns CPPGB_ERR_CAPACITY with a message); every device that loads the library keeps
 * that 1 MiB until the process exits.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call outside any stream capture.  Every call
 * waits for the stream before it returns (it reads the result back through the shared array), so
 * no call may be made while the stream is being captured.  All calls on a device share the array:
 * calls whose work may overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  Planes and out are as for twolocus_scan; out is valid on return.
 */
int twolocus_scan_noalloc(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                          twolocus_result* out, void* stream);

/*
 * twolocus_scan_shard -- shard s of nshards of the two-locus scan: evaluates only the SNP-pair tiles
 * (64 x 128 SNPs) whose index is s mod nshards and returns the best pair among them with its tables
 * (i = j = -1, score = -1 when the shard has none).  The answer of the whole scan is the shard
 * result with the largest score, then the smallest (i, j): one max-reduce across the shards.
 * Arguments and workspace as for twolocus_scan; CPPGB_ERR_ARG also for a bad shard.
 */
int twolocus_scan_shard(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                        int64_t shard, int64_t nshards, twolocus_result* out, void* ws, size_t ws_bytes,
                        void* stream);

/*
 * twolocus_scan_tc -- the two-locus scan of Sec. 6 on the tensor cores, with either measure:
 *   CPPGB_TL_MATCHES  the match fraction of Sec. 5.3 (the result equals twolocus_scan's);
 *   CPPGB_TL_PEARSON  Pearson's correlation of the genotype values 0, 1, 2 within each group (the
 *                     measure Sec. 5 and Sec. 6 attribute to the method they compare with):
 *                     r = (m Sxy - Sx Sy) / sqrt(vx vy), vx = m Sxx - Sx^2 (0 when vx or vy is 0),
 *                     score |r_A - r_B| in score_real (score = -1), ties to the smallest (i, j).
 * The per-pair counts are exact integer GEMMs: one-hot planes a = [g = 1], b = [g = 2] become FP8
 * (E4M3) rows [a, b] (left) and [2c + d, c + 2d] or [c + 2d, 2c + 4d] (right) -- every value is
 * 0, 1, 2 or 4, exact in E4M3 -- and every partial sum is an integer below 2^24, so the FP32
 * tensor-core accumulation is exact.  Arguments as for twolocus_scan (W <= 4096, groups < 2^20
 * subjects); the workspace holds the four FP8 matrices, 4 S W 128 bytes (128 MB at 4096 SNPs x
 * 4096 + 4096 subjects).
 * Errors (return value): CPPGB_ERR_ARG, CPPGB_ERR_CAPACITY (ws), CPPGB_ERR_CUDA; (out->status):
 * CPPGB_ERR_TIMEOUT.
 */
#define CPPGB_TL_MATCHES 0
#define CPPGB_TL_PEARSON 1
size_t twolocus_scan_tc_workspace_size(int64_t S, int64_t W);
int twolocus_scan_tc(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls, int measure,
                     twolocus_result* out, void* ws, size_t ws_bytes, void* stream);
/* Shard `shard` of `nshards` of twolocus_scan_tc: the 128 x 128 tiles t (in the scan's order of the
 * SNP-pair triangle) with t mod nshards == shard; the best pair of those tiles (i = j = -1 when they
 * hold none).  The answer of the whole scan is the shard result with the largest score (score_real
 * for Pearson), ties to the smallest (i, j).  Same workspace as twolocus_scan_tc. */
int twolocus_scan_tc_shard(const uint64_t* planes, int64_t S, int64_t W, int64_t m_cases, int64_t m_controls,
                           int measure, int64_t shard, int64_t nshards, twolocus_result* out, void* ws, size_t ws_bytes,
                           void* stream);

/* Result of a string-pair search. */
typedef struct {
  int64_t i, j;        /* the pair, i < j; -1 when n < 2 */
  int64_t mismatches;  /* its Hamming distance */
  int32_t status;      /* CPPGB_OK, or the error the device found (valid after the stream sync) */
  int32_t reserved;
} hamming_result;

/*
 * hamming_pair -- closest pair (least = 0: fewest mismatches, the CPP of Sec. 4) or least
 * correlated pair (least = 1: most mismatches, Sec. 5) of n strings of t symbols from
 * {0, .., sigma - 1}, ties to the smallest (i, j).  Each string becomes a one-hot FP8 (E4M3) row
 * of t sigma entries (the mapping of Sec. 5.5, one 1 per position); the dot product of two rows,
 * accumulated exactly in FP32 on the tensor cores, is the number of agreeing positions.
 *   strs  device uint8 [n][ld], ld >= t.   2 <= sigma <= 256, t <= 2^23.
 * Errors (return value): CPPGB_ERR_ARG, CPPGB_ERR_CAPACITY (ws), CPPGB_ERR_CUDA; (out->status):
 * CPPGB_ERR_ARG for a symbol >= sigma, CPPGB_ERR_TIMEOUT.
 */
size_t hamming_pair_workspace_size(int64_t n, int64_t t, int sigma);
int hamming_pair(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, hamming_result* out,
                 void* ws, size_t ws_bytes, void* stream);
/* Shard `shard` of `nshards` of hamming_pair: the 128 x 128 tiles t with t mod nshards == shard; the
 * answer of the whole search is the shard result with the fewest (least = 0) or most (least = 1)
 * mismatches, ties to the smallest (i, j).  Same workspace as hamming_pair. */
int hamming_pair_shard(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, int64_t shard,
                       int64_t nshards, hamming_result* out, void* ws, size_t ws_bytes, void* stream);

/* Result of a light-bulb candidate search. */
typedef struct {
  int64_t i, j;        /* the best candidate pair, i < j; -1 when no pair shared a bucket */
  int64_t mismatches;  /* its Hamming distance; -1 when there is no candidate */
  int64_t candidates;  /* candidate pairs verified, each counted once per iteration it was found in */
  int32_t status;      /* CPPGB_OK, or the error the device found */
  int32_t reserved;
} mlba_result;

/*
 * mlba_pair -- the modified light-bulb algorithm (MLBA) of Sec. 4: a randomised search for the
 * closest pair of strings (least = 0) that looks only at the pairs sharing a bucket in some
 * iteration, and its least correlated form (least = 1) over the one-hot strings and their
 * complements of Sec. 5.4-5.5.  The random choice of columns is the caller's: cols holds, for each
 * of the iters iterations, L sampled columns (the paper samples c log n of them), which are
 *   least = 0: symbol positions 0 .. t-1;
 *   least = 1: one-hot columns 0 .. sigma*t - 1, column c being the bit [s_{c / sigma} = c % sigma]
 *              of a string and its negation for a complement.
 * In each iteration the rows are grouped by their characters in the sampled columns (a radix sort);
 * every two strings in a group are a candidate (least = 1: a string and the complement of another;
 * each unordered pair at most once per iteration), and every candidate is verified by its Hamming
 * distance.  The answer is the candidate with the fewest (least = 0) or most (least = 1)
 * mismatches, ties to the smallest (i, j); it is the exact answer when the best pair met in some
 * iteration (L = 0 makes every pair a candidate: the brute force).
 *   strs  device uint8 [n][ld], ld >= t, symbols < sigma, 2 <= sigma <= 256.
 *   cols  device int32 [iters][L] (not read when L = 0).  The sampled characters fill one 64-bit
 *         key: L * ceil(log2 sigma) <= 64 (least = 0), 1 <= L <= 64 (least = 1); iters x rows
 *         (n, or 2n for least = 1) below 2^31.
 * The call synchronises the stream before it returns.  Its kernels are captured once into a CUDA
 * graph per argument set (pointers and sizes) and replayed while the arguments stay the same; calls
 * from several threads are serialised by a library-wide lock (so the call cannot itself be captured
 * into a caller's graph).
 * Errors: CPPGB_ERR_ARG (also for a symbol >= sigma or a column out of range), CPPGB_ERR_CAPACITY
 * (ws), CPPGB_ERR_CUDA.
 */
size_t mlba_pair_workspace_size(int64_t n, int64_t t, int sigma, int least, int64_t iters, int64_t L);
int mlba_pair(const uint8_t* strs, int64_t n, int64_t t, int64_t ld, int sigma, int least, const int32_t* cols,
              int64_t iters, int64_t L, mlba_result* out, void* ws, size_t ws_bytes, void* stream);

/* Result of a fixed-radius query. */
typedef struct {
  int64_t n_pairs;     /* directed pairs (= row_ptr[n]), also when cols_cap was too small */
  int32_t status;      /* CPPGB_OK, or the error the device found (valid after the stream sync) */
  int32_t n_rows;      /* points whose rows the call wrote: n, or for frnn_query_shard its slab's */
} frnn_result;

/*
 * frnn_query -- fixed-radius near neighbours (Sec. 3.5): for every point p_i its R-neighbourhood
 * N(i) = { j != i : d(p_i, p_j) <= R }, with j in N(i) iff i in N(j).  The decision is the FP64
 * test sum_k (x_ik - x_jk)^2 <= R*R (coordinate order).
 *   pts      device FP32 row-major [n][ld], d in [1, 4] (uniform-grid cell hash) or
 *            d in [5, 4096] (tiled all-pairs with a radius test).
 *   R        radius, finite and >= 0.
 *   row_ptr  device int64 [n+1], CSR offsets (written).
 *   cols     device int32 [cols_cap], neighbour indices ascending within each row (written).
 *   out      host (pinned for an asynchronous call); valid after the stream sync.
 * Errors (return value): CPPGB_ERR_ARG, CPPGB_ERR_CAPACITY (ws), CPPGB_ERR_CUDA.
 * Errors (out->status): CPPGB_ERR_CAPACITY (cols_cap < out->n_pairs; cols is then untouched, or,
 *         on the high-d path, more candidate pairs than the workspace holds), CPPGB_ERR_NUMERIC
 *         (a non-finite coordinate).
 */
size_t frnn_query_workspace_size(int64_t n, int d);
int frnn_query(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t* row_ptr, int32_t* cols,
               int64_t cols_cap, frnn_result* out, void* ws, size_t ws_bytes, void* stream);

/*
 * frnn_query_shard -- shard s of nshards of frnn_query on the grid path (1 <= d <= 4): the points
 * are split into nshards slabs along x, each a range of whole x-cells (cells of side >= R over the
 * bounding box) holding an equal share of the points (up to one of 4096 equal-width bins of the
 * x-cells, so clustered data balances too), and only the points of slab s get their neighbour
 * lists; every other row is empty (row_ptr has n + 1 entries as usual); out->n_rows is the number of
 * points of slab s.  Each shard still builds the grid over all points, so the neighbours of
 * a slab's points in the adjacent slabs (the halo) are found.  Concatenating, point by point, the
 * rows of the point's own shard gives exactly the CSR of frnn_query.  Arguments, workspace and
 * errors as for frnn_query; CPPGB_ERR_ARG for d > 4 or a bad shard.
 */
int frnn_query_shard(const float* pts, int64_t n, int d, int64_t ld, double R, int64_t shard, int64_t nshards,
                     int64_t* row_ptr, int32_t* cols, int64_t cols_cap, frnn_result* out, void* ws,
                     size_t ws_bytes, void* stream);

/* One instance of a batch. */
typedef struct {
  const float* pts; /* device FP32 [n][d] row-major (ld = d) */
  int64_t n;
  int32_t d;        /* 1 .. 256 */
  int32_t path;     /* 0: the tuning policy's choice, 1: FP32 CUDA-core tiles, 2: BF16 tensor-core
                       tiles read by four epilogue groups (128 columns each), 3: the same tiles read
                       by two (256 columns each) -- the answer is exact either way */
  double R;         /* FRNN radius for this instance (< 0: no FRNN output) */
} cpp_instance;

/*
 * cpp_batch -- many independent CPP + FRNN instances of uneven n and d in one persistent launch
 * (the problems of Sec. 3 and Sec. 3.5, instance by instance).  Instances on the FP32 path share
 * one persistent CUDA-core tile kernel, those on the tensor-core path one persistent tcgen05
 * kernel (BF16 rows padded to 16, 32, 64, 128, 192 or 256 columns, one tensor map per width); both feed
 * the same FP32 second pass and FP64 recheck, so the answer does not depend on the path.
 *   inst        host array [count].
 *   out_cpp     host [count]: closest pair of each instance (identical to cpp_closest_pair; the
 *               prune fields are -1); valid after the stream sync.
 *   pair_counts host int64 [count]: number of undirected pairs (i < j) with d <= R per instance;
 *               valid after the stream sync.
 *   pairs       device int32 [pairs_cap][2]: the (i, j) pairs, instance after instance, ascending (i, j).
 * Errors (return value): CPPGB_ERR_ARG, CPPGB_ERR_CAPACITY (ws), CPPGB_ERR_CUDA.
 * Errors (status of every out_cpp entry): CPPGB_ERR_CAPACITY (pairs_cap smaller than the pairs
 *         within R -- pair_counts still holds the counts -- or more candidate pairs than the
 *         workspace holds), CPPGB_ERR_NUMERIC, CPPGB_ERR_TIMEOUT.
 */
size_t cpp_batch_workspace_size(const cpp_instance* inst, int64_t count);
int cpp_batch(const cpp_instance* inst, int64_t count, cpp_pair_result* out_cpp, int64_t* pair_counts,
              int32_t* pairs, int64_t pairs_cap, void* ws, size_t ws_bytes, void* stream);

/*
 * Diagnostics (no counterpart in the paper; used to measure the library).
 * cpp_set_stage_timing(1) makes the dense searches record CUDA events on their stream around
 * their stages; cpp_stage_times() then waits for the last call's events and copies its stage
 * durations in milliseconds (per calling thread) into ms[0..cap) and returns how many it wrote: [prep, dense all-pairs stage,
 * FP64 recheck] after cpp_closest_pair / tsmm_motif, [preparation, tensor-core tiles, FP32 tiles,
 * second pass + recheck + output] after cpp_batch (events captured in its graph), [pack + keys,
 * radix sort, buckets + pair offsets, verification] after mlba_pair.  cpp_launch_count() returns the number of kernels this library has launched
 * in the process so far.
 */
void cpp_set_stage_timing(int on);
/* Measures the CUDA-core rates the ALU rooflines are checked against (diagnostics): FP32 FFMA in
 * TFLOP/s (2 flop per FMA) and POPC in Tpopc/s, each from independent chains on a full grid of the
 * current device, timed with CUDA events on the legacy default stream (about 0.1 s; allocates and
 * frees 1.2 MB of device memory).  Errors: CPPGB_ERR_ARG, CPPGB_ERR_CUDA. */
int cpp_measure_alu_peaks(double* ffma_tflops, double* popc_tops);
int cpp_stage_times(double* ms, int cap);
int64_t cpp_launch_count(void);

/* 1 when this build carries the tensor-core filter modes (CPPGB_MODE_FILTER_*), else 0. */
int cpp_filter_available(void);

/*
 * cpp_gram_tile_dump -- diagnostics (no counterpart in the paper): the raw Gram values that the
 * tensor-core filter stage of cpp_closest_pair accumulates for chosen tiles, so that their error
 * can be compared with the accumulation term of the filter's error bound.  The points are prepared
 * exactly as by cpp_closest_pair in `mode`, and the tiles run through the same TMA / tcgen05.mma
 * pipeline; only the epilogue differs (it stores the accumulator instead of reducing it).
 *   pts, dtype, n (>= 1), d, ld  as for cpp_closest_pair.   mode  CPPGB_MODE_FILTER_BF16 or _FP16.
 *   tiles  host int32 [ntiles][2]: (bi, bj) = rows 128 bi .. 128 bi + 127 against rows
 *          256 bj .. 256 bj + 255, with 0 <= bi < n_pad / 128, 0 <= bj < n_pad / 256 (n_pad = n
 *          rounded up to a multiple of 256; rows past n are zero).
 *   S      device FP32 [ntiles][128][256]: S[t][r][c] = x~_(128 bi + r) . x~_(256 bj + c), the
 *          FP32 accumulator of the tensor cores (x~ = the stored 16-bit rows).
 *   rows   device, optional (NULL: not written): the stored 16-bit rows, [n_pad][Kp] with Kp = d
 *          rounded up to a multiple of 64, zero-padded (2 n_pad Kp bytes).
 *   ws     a workspace of cpp_closest_pair_workspace_size(n, d, mode) bytes.
 * The call synchronises the stream.  Errors: CPPGB_ERR_ARG (also a tile out of range, or more
 * than 131,072 tiles), CPPGB_ERR_CAPACITY (ws), CPPGB_ERR_NUMERIC, CPPGB_ERR_TIMEOUT, CPPGB_ERR_CUDA.
 */
int cpp_gram_tile_dump(const void* pts, int dtype, int64_t n, int64_t d, int64_t ld, int mode, const int32_t* tiles,
                       int64_t ntiles, float* S, void* rows, void* ws, size_t ws_bytes, void* stream);

/*
 * Fault injection for tests of the failure path (no counterpart in the paper).  Every wait of the
 * tensor-core kernels (TMA copies, MMA completion, accumulator hand-over, tile records) is bounded
 * by about 2 s; when one runs out the kernel stops issuing work, waits (bounded) for what it has in
 * flight, frees its tensor memory and returns, and the call reports CPPGB_ERR_TIMEOUT.
 *   CPPGB_FAULT_SKIP_TMA  the TMA producers of the tensor-core kernels (dense filter stage of
 *                         cpp_closest_pair / tsmm_motif, tensor-core tiles of cpp_batch,
 *                         twolocus_scan_tc, hamming_pair) issue no copy, so the consumers' waits
 *                         run out: each such call then takes about 2 s and returns
 *                         CPPGB_ERR_TIMEOUT; nothing is left in flight and the device stays usable.
 *   CPPGB_FAULT_NONE      normal operation (the default).
 * Process-wide, for the current device; a synchronous copy to device memory, so make no call
 * during stream capture.  Errors: CPPGB_ERR_ARG (unknown kind), CPPGB_ERR_CUDA.
 */
#define CPPGB_FAULT_NONE 0
#define CPPGB_FAULT_SKIP_TMA 1
int cpp_set_fault_injection(int kind);

/*
 * Tuning policy (process-wide; no counterpart in the paper).  The project's autotuner times the
 * candidates on the device, caches its choice as JSON and installs it here; every later call reads it.
 *   CPPGB_TUNE_BATCH_PATH  values = int32 [4 n-buckets][6 d-classes], count 24, each 1 (FP32 128 x 128
 *                          CUDA-core tiles), 2 (BF16 128 x 256 tensor-core tiles, four epilogue groups
 *                          of 128 columns) or 3 (the same tiles, two epilogue groups of 256 columns);
 *                          used by cpp_batch instances whose path is 0.
 *                          n-buckets: n < 1024, < 4096, < 16384, the rest; d-classes: d <= 16, <= 32,
 *                          <= 64, <= 128, <= 192, <= 256.  Default (when the tensor-core kernels exist):
 *                          2 for d <= 16, 3 above (measured on GB300).
 *   CPPGB_TUNE_DENSE_BAND  values = int32 [1]: column blocks per band of the tensor-core dense stage's
 *                          tile order (1 .. 4096; 0 from cpp_get_tuning means the built-in 16).
 *   CPPGB_TUNE_DENSE_SHAPE values = int32 [1]: tile of the tensor-core dense stage (unpruned searches):
 *                          1 = 128 x 256 on one SM (M = 128 MMAs), 2 = 256 x 256 on a cluster of two SMs
 *                          (tcgen05 cta_group::2, M = 256 MMAs; each SM loads half of the column
 *                          block).  Default 1 (measured faster on GB300: the single-SM tiles run at the
 *                          same tensor-pipe occupancy with less synchronisation).
 * Both return CPPGB_ERR_ARG for an unknown kind, a short array or an invalid entry; the choice only
 * changes speed, never a result.
 */
#define CPPGB_TUNE_BATCH_PATH 1
#define CPPGB_TUNE_DENSE_BAND 2
#define CPPGB_TUNE_DENSE_SHAPE 3
int cpp_set_tuning(int kind, const int32_t* values, int count);
int cpp_get_tuning(int kind, int32_t* values, int count);

/* Message for the last non-OK status returned on the calling thread ("" if none). */
const char* cpp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CPPGB_H */
