/*
 * Oracle for the exact closest-pair family -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU brute force of what the GPU library computes.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the library never calls it and shares no code with it.
 *
 * Every answer here is a plain definition written out (the method reaches the
 * brute-force answer exactly), so each function is a direct loop over all pairs:
 *
 *   oracle_cpp        closest pair, Sec. 3 (problem statement) with the
 *                     Euclidean distance of Sec. 2; optional index gap `excl`
 *   oracle_znorm      z-normalised l-mers (l-mers as defined in Sec. 2)
 *   oracle_tsmm       motif pair: closest pair of z-normalised l-mers, Sec. 3
 *   oracle_tsmm_pairs / oracle_tsmm_rows   the same distance for chosen pairs
 *                     or rows (sampled checks at full size)
 *   oracle_frnn       R-neighbourhoods N(i) for all i, Sec. 3.5 (d <= R,
 *                     symmetric insertion into N(i) and N(j))
 *   oracle_frnn_rows  N(i) for chosen rows
 *   oracle_radius_pairs  the same neighbourhoods as a list of pairs i < j, each
 *                     once, in increasing (i, j)
 *   oracle_twolocus   argmax |P_A(i,j) - P_B(i,j)|, Sec. 6, with the
 *                     match-count correlation of Sec. 2 / Sec. 5.3
 *   oracle_twolocus_tables / oracle_twolocus_rows   3x3 tables for chosen
 *                     pairs, best partner for chosen rows
 *   oracle_twolocus_pearson   the same argmax with Pearson's correlation of the
 *                     genotype values within each group (the measure Sec. 5 and
 *                     Sec. 6 attribute to the light-bulb/LSH method they compare
 *                     with)
 *   oracle_hamming    closest (or least correlated) pair of strings over an
 *                     alphabet of sigma symbols under the Hamming distance, Sec. 4
 *                     (and Sec. 5 for the least correlated pair)
 *   oracle_mlba       the modified light-bulb algorithm of Sec. 4 (sampled columns,
 *                     sort, buckets, candidate pairs, verification), and its least
 *                     correlated form over the one-hot strings and their complements
 *                     of Sec. 5.4-5.5; the columns each iteration samples are inputs
 *
 * Readings taken where the paper is silent (each also listed in the design
 * notes): ties go to the lexicographically smallest (d^2, i, j) with i < j;
 * z-normalisation uses the population standard deviation; a motif pair needs
 * j - i >= excl; FRNN uses "<= R" and excludes the point itself; two-locus
 * compares |u_A*m2 - u_B*m1| exactly in integers (u = matches); Pearson's r is
 * (m Sxy - Sx Sy) / sqrt(vx vy) with vx = m Sxx - Sx^2 (exact integers, one FP64
 * product, square root and division), 0 when a variance is 0, and the score
 * |r_A - r_B| is compared as a double (ties to the smallest (i, j)); Hamming
 * pairs are ranked by their number of mismatches (ties to the smallest (i, j)).
 *
 * Build: plain C99, -O2 -ffp-contract=off (no FMA contraction, so every sum is
 * a rounded add of a rounded product, in index order), OpenMP over the outer
 * loop only; the per-pair arithmetic is unchanged by the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_ERR_ARG 1
#define ORACLE_ERR_CAPACITY 2
#define ORACLE_ERR_NUMERIC 5

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following calls (for timing the oracle on one core); k < 1 is ignored. */
void oracle_set_num_threads(int k) {
#ifdef _OPENMP
  if (k >= 1) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

/* (d2, i, j) is lexicographically smaller than (bd2, bi, bj) */
static int lex_less(double d2, int64_t i, int64_t j, double bd2, int64_t bi, int64_t bj) {
  if (d2 < bd2) return 1;
  if (d2 > bd2) return 0;
  if (i < bi) return 1;
  if (i > bi) return 0;
  return j < bj;
}

/* Squared Euclidean distance, Sec. 2: sum over k = 0..d-1 of (x_k - y_k)^2, in k order. */
static double sqdist(const double* x, const double* y, int64_t d) {
  double s = 0.0;
  for (int64_t k = 0; k < d; ++k) {
    double t = x[k] - y[k];
    s = s + t * t;
  }
  return s;
}

double oracle_sqdist(const double* x, const double* y, int64_t d) { return sqdist(x, y, d); }

/*
 * Closest pair (Sec. 3): over all 0 <= i < j < n with j - i >= excl, the pair with the
 * least distance.  excl = 1 gives the plain CPP.  Returns (-1,-1,+inf) when no pair is valid.
 */
int oracle_cpp(const double* x, int64_t n, int64_t d, int64_t excl,
               int64_t* bi, int64_t* bj, double* bd2) {
  if (!x || n < 0 || d <= 0 || excl < 1 || !bi || !bj || !bd2) return ORACLE_ERR_ARG;
  double best = INFINITY;
  int64_t best_i = -1, best_j = -1;
#pragma omp parallel
  {
    double lb = INFINITY;
    int64_t li = -1, lj = -1;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = i + excl; j < n; ++j) {
        double s = sqdist(x + i * d, x + j * d, d);
        if (li < 0 || lex_less(s, i, j, lb, li, lj)) { lb = s; li = i; lj = j; }
      }
    }
#pragma omp critical
    {
      if (li >= 0 && (best_i < 0 || lex_less(lb, li, lj, best, best_i, best_j))) {
        best = lb; best_i = li; best_j = lj;
      }
    }
  }
  *bi = best_i; *bj = best_j; *bd2 = best;
  return ORACLE_OK;
}

/*
 * z-normalisation of the l-mers T_i = a_i .. a_{i+l-1} (Sec. 2), i = 0 .. N-l:
 *   mu_i = (sum_k a_{i+k}) / l,  sigma_i = sqrt((sum_k (a_{i+k} - mu_i)^2) / l),
 *   z_ik = (a_{i+k} - mu_i) / sigma_i.
 * Sums in k order.  z may be NULL (only mu, sigma wanted).  sigma = 0 -> ERR_NUMERIC.
 */
static int znorm_row(const double* a, int64_t l, double* mu_out, double* sd_out, double* z) {
  double s = 0.0;
  for (int64_t k = 0; k < l; ++k) s = s + a[k];
  double mu = s / (double)l;
  double v = 0.0;
  for (int64_t k = 0; k < l; ++k) {
    double t = a[k] - mu;
    v = v + t * t;
  }
  double sd = sqrt(v / (double)l);
  if (mu_out) *mu_out = mu;
  if (sd_out) *sd_out = sd;
  if (!(sd > 0.0)) return ORACLE_ERR_NUMERIC;
  if (z)
    for (int64_t k = 0; k < l; ++k) z[k] = (a[k] - mu) / sd;
  return ORACLE_OK;
}

int oracle_znorm(const double* a, int64_t N, int64_t l, double* z, double* mu, double* sigma) {
  if (!a || l < 1 || N < l) return ORACLE_ERR_ARG;
  int64_t n = N - l + 1;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < n; ++i) {
    double m, s;
    int rc = znorm_row(a + i, l, &m, &s, z ? z + i * l : NULL);
    if (mu) mu[i] = m;
    if (sigma) sigma[i] = s;
    bad |= (rc != ORACLE_OK);
  }
  return bad ? ORACLE_ERR_NUMERIC : ORACLE_OK;
}

/* Motif pair (Sec. 3): closest pair of z-normalised l-mers with j - i >= excl. */
int oracle_tsmm(const double* a, int64_t N, int64_t l, int64_t excl,
                int64_t* bi, int64_t* bj, double* bd2) {
  if (!a || l < 1 || N < l || excl < 1) return ORACLE_ERR_ARG;
  int64_t n = N - l + 1;
  double* z = (double*)malloc((size_t)n * (size_t)l * sizeof(double));
  if (!z) return ORACLE_ERR_ARG;
  int rc = oracle_znorm(a, N, l, z, NULL, NULL);
  if (rc == ORACLE_OK) rc = oracle_cpp(z, n, l, excl, bi, bj, bd2);
  free(z);
  return rc;
}

/* The motif distance of chosen pairs (I[p], J[p]), each l-mer normalised on its own. */
int oracle_tsmm_pairs(const double* a, int64_t N, int64_t l, const int64_t* I, const int64_t* J,
                      int64_t np, double* out_d2) {
  if (!a || l < 1 || N < l || np < 0 || !I || !J || !out_d2) return ORACLE_ERR_ARG;
  int64_t n = N - l + 1;
  int bad = 0;
#pragma omp parallel reduction(| : bad)
  {
    double* zi = (double*)malloc((size_t)l * sizeof(double));
    double* zj = (double*)malloc((size_t)l * sizeof(double));
#pragma omp for schedule(dynamic, 4)
    for (int64_t p = 0; p < np; ++p) {
      if (I[p] < 0 || I[p] >= n || J[p] < 0 || J[p] >= n) { bad |= 1; out_d2[p] = NAN; continue; }
      int r1 = znorm_row(a + I[p], l, NULL, NULL, zi);
      int r2 = znorm_row(a + J[p], l, NULL, NULL, zj);
      out_d2[p] = (r1 || r2) ? NAN : sqdist(zi, zj, l);
      bad |= (r1 || r2) ? 2 : 0;
    }
    free(zi);
    free(zj);
  }
  return bad ? ((bad & 1) ? ORACLE_ERR_ARG : ORACLE_ERR_NUMERIC) : ORACLE_OK;
}

/*
 * For each chosen row r = rows[p]: the lexicographically smallest (d2, min(r,j), max(r,j))
 * over all j with |r - j| >= excl (partners on both sides).  best_j = -1 if none.
 */
int oracle_tsmm_rows(const double* a, int64_t N, int64_t l, int64_t excl, const int64_t* rows,
                     int64_t nr, int64_t* best_j, double* best_d2) {
  if (!a || l < 1 || N < l || excl < 1 || nr < 0 || !rows || !best_j || !best_d2)
    return ORACLE_ERR_ARG;
  int64_t n = N - l + 1;
  for (int64_t p = 0; p < nr; ++p)
    if (rows[p] < 0 || rows[p] >= n) return ORACLE_ERR_ARG;
  double* z = (double*)malloc((size_t)n * (size_t)l * sizeof(double));
  if (!z) return ORACLE_ERR_ARG;
  int rc = oracle_znorm(a, N, l, z, NULL, NULL);
  if (rc == ORACLE_OK) {
    for (int64_t p = 0; p < nr; ++p) {
      int64_t r = rows[p];
      double bd = INFINITY;
      int64_t bjj = -1;
#pragma omp parallel
      {
        double lb = INFINITY;
        int64_t lj = -1;
#pragma omp for schedule(static)
        for (int64_t j = 0; j < n; ++j) {
          int64_t gap = j > r ? j - r : r - j;
          if (gap < excl) continue;
          double s = sqdist(z + r * l, z + j * l, l);
          int64_t lo = r < j ? r : j, hi = r < j ? j : r;
          int64_t llo = lj < 0 ? 0 : (r < lj ? r : lj), lhi = lj < 0 ? 0 : (r < lj ? lj : r);
          if (lj < 0 || lex_less(s, lo, hi, lb, llo, lhi)) { lb = s; lj = j; }
        }
#pragma omp critical
        {
          if (lj >= 0) {
            int64_t lo = r < lj ? r : lj, hi = r < lj ? lj : r;
            int64_t blo = bjj < 0 ? 0 : (r < bjj ? r : bjj), bhi = bjj < 0 ? 0 : (r < bjj ? bjj : r);
            if (bjj < 0 || lex_less(lb, lo, hi, bd, blo, bhi)) { bd = lb; bjj = lj; }
          }
        }
      }
      best_j[p] = bjj;
      best_d2[p] = bd;
    }
  }
  free(z);
  return rc;
}

/*
 * FRNN (Sec. 3.5): N(i) = { j != i : d(a_i, a_j) <= R }, decided as
 * sum_k (x_ik - x_jk)^2 <= R*R in FP64 (k order).  Output CSR: row_ptr[n+1], cols ascending
 * per row.  If cap < total pairs, returns ORACLE_ERR_CAPACITY with *total set.
 */
static int frnn_pred(const double* x, const double* y, int64_t d, double rr) {
  return sqdist(x, y, d) <= rr;
}

int oracle_frnn(const double* x, int64_t n, int64_t d, double R, int64_t* row_ptr, int32_t* cols,
                int64_t cap, int64_t* total) {
  if (!x || n < 0 || d <= 0 || !(R >= 0.0) || !row_ptr || !total || n > INT32_MAX) return ORACLE_ERR_ARG;
  double rr = R * R;
  row_ptr[0] = 0;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j)
      if (j != i && frnn_pred(x + i * d, x + j * d, d, rr)) ++c;
    row_ptr[i + 1] = c;
  }
  for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] += row_ptr[i];
  *total = row_ptr[n];
  if (!cols || cap < row_ptr[n]) return ORACLE_ERR_CAPACITY;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    int64_t o = row_ptr[i];
    for (int64_t j = 0; j < n; ++j)
      if (j != i && frnn_pred(x + i * d, x + j * d, d, rr)) cols[o++] = (int32_t)j;
  }
  return ORACLE_OK;
}

/* N(r) for chosen rows; neighbours of rows[p] land in cols[offs[p] .. offs[p+1]). */
int oracle_frnn_rows(const double* x, int64_t n, int64_t d, double R, const int64_t* rows,
                     int64_t nr, int64_t* offs, int32_t* cols, int64_t cap) {
  if (!x || n < 0 || d <= 0 || !(R >= 0.0) || !rows || !offs || nr < 0) return ORACLE_ERR_ARG;
  double rr = R * R;
  offs[0] = 0;
  for (int64_t p = 0; p < nr; ++p) {
    if (rows[p] < 0 || rows[p] >= n) return ORACLE_ERR_ARG;
    int64_t c = 0;
#pragma omp parallel for reduction(+ : c) schedule(static)
    for (int64_t j = 0; j < n; ++j)
      if (j != rows[p] && frnn_pred(x + rows[p] * d, x + j * d, d, rr)) ++c;
    offs[p + 1] = offs[p] + c;
  }
  if (!cols || cap < offs[nr]) return ORACLE_ERR_CAPACITY;
  for (int64_t p = 0; p < nr; ++p) {
    int64_t o = offs[p];
    for (int64_t j = 0; j < n; ++j)
      if (j != rows[p] && frnn_pred(x + rows[p] * d, x + j * d, d, rr)) cols[o++] = (int32_t)j;
  }
  return ORACLE_OK;
}

/*
 * The pairs of an R-neighbourhood query (Sec. 3.5) counted once each: every i < j with
 * sum_k (x_ik - x_jk)^2 <= R*R in FP64 (k order), listed in increasing (i, j) as int32
 * pairs[2p], pairs[2p+1].  One pass over the pairs; each thread collects its rows' pairs, and the
 * collected list is sorted at the end.  *total = number of pairs; ERR_CAPACITY when cap < total.
 */
static int pair_cmp(const void* a, const void* b) {
  const int32_t* p = (const int32_t*)a;
  const int32_t* q = (const int32_t*)b;
  if (p[0] != q[0]) return p[0] < q[0] ? -1 : 1;
  if (p[1] != q[1]) return p[1] < q[1] ? -1 : 1;
  return 0;
}

int oracle_radius_pairs(const double* x, int64_t n, int64_t d, double R, int32_t* pairs, int64_t cap,
                        int64_t* total) {
  if (!x || n < 0 || d <= 0 || !(R >= 0.0) || !total || n > INT32_MAX) return ORACLE_ERR_ARG;
  double rr = R * R;
  int32_t* all = NULL;
  int64_t nall = 0;
  int bad = 0;
#pragma omp parallel reduction(| : bad)
  {
    int32_t* mine = NULL;
    int64_t nm = 0, capm = 0;
#pragma omp for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = i + 1; j < n; ++j) {
        if (!frnn_pred(x + i * d, x + j * d, d, rr)) continue;
        if (nm == capm) {
          int64_t nc = capm ? 2 * capm : 64;
          int32_t* grown = (int32_t*)realloc(mine, (size_t)nc * 2 * sizeof(int32_t));
          if (!grown) { bad = 1; continue; }
          mine = grown;
          capm = nc;
        }
        mine[2 * nm] = (int32_t)i;
        mine[2 * nm + 1] = (int32_t)j;
        ++nm;
      }
    }
#pragma omp critical
    {
      if (nm > 0) {
        int32_t* grown = (int32_t*)realloc(all, (size_t)(nall + nm) * 2 * sizeof(int32_t));
        if (!grown) bad = 1;
        else {
          all = grown;
          memcpy(all + 2 * nall, mine, (size_t)nm * 2 * sizeof(int32_t));
          nall += nm;
        }
      }
    }
    free(mine);
  }
  if (bad) { free(all); return ORACLE_ERR_ARG; }
  if (nall > 1) qsort(all, (size_t)nall, 2 * sizeof(int32_t), pair_cmp);
  *total = nall;
  int rc = ORACLE_OK;
  if (!pairs || cap < nall) rc = ORACLE_ERR_CAPACITY;
  else if (nall > 0) memcpy(pairs, all, (size_t)nall * 2 * sizeof(int32_t));
  free(all);
  return rc;
}

/*
 * Two-locus (Sec. 6).  g is int8 [S][m1+m2], genotype of SNP s for subject t at g[s*(m1+m2)+t];
 * subjects 0..m1-1 are cases (matrix A), m1..m1+m2-1 controls (matrix B).
 * For a pair (i, j) and a group, tab[3*a+b] counts the subjects with g_i = a and g_j = b;
 * the matches of Sec. 2 are u = tab[0] + tab[4] + tab[8], the correlation of Sec. 5.3 is
 * u / (group size), so |P_A - P_B| * m1 * m2 = |u_A * m2 - u_B * m1|.
 */
static void table_of(const int8_t* gi, const int8_t* gj, int64_t lo, int64_t hi, int32_t* tab) {
  for (int q = 0; q < 9; ++q) tab[q] = 0;
  for (int64_t t = lo; t < hi; ++t) tab[3 * gi[t] + gj[t]] += 1;
}

static int64_t score_of(const int32_t* ta, const int32_t* tb, int64_t m1, int64_t m2) {
  int64_t ua = (int64_t)ta[0] + ta[4] + ta[8];
  int64_t ub = (int64_t)tb[0] + tb[4] + tb[8];
  int64_t s = ua * m2 - ub * m1;
  return s < 0 ? -s : s;
}

static int geno_ok(const int8_t* g, int64_t S, int64_t m) {
  for (int64_t q = 0; q < S * m; ++q)
    if (g[q] < 0 || g[q] > 2) return 0;
  return 1;
}

/* (score, i, j) beats (bs, bi, bj): larger score first, then smaller i, then smaller j */
static int tl_better(int64_t s, int64_t i, int64_t j, int64_t bs, int64_t bi, int64_t bj) {
  if (s != bs) return s > bs;
  if (i != bi) return i < bi;
  return j < bj;
}

int oracle_twolocus(const int8_t* g, int64_t S, int64_t m1, int64_t m2, int64_t* bi, int64_t* bj,
                    int64_t* score, int32_t* countsA, int32_t* countsB) {
  if (!g || S < 0 || m1 < 1 || m2 < 1 || !bi || !bj || !score) return ORACLE_ERR_ARG;
  int64_t m = m1 + m2;
  if (!geno_ok(g, S, m)) return ORACLE_ERR_ARG;
  int64_t best = -1, best_i = -1, best_j = -1;
#pragma omp parallel
  {
    int64_t ls = -1, li = -1, lj = -1;
    int32_t ta[9], tb[9];
#pragma omp for schedule(dynamic, 8)
    for (int64_t i = 0; i < S; ++i) {
      for (int64_t j = i + 1; j < S; ++j) {
        table_of(g + i * m, g + j * m, 0, m1, ta);
        table_of(g + i * m, g + j * m, m1, m, tb);
        int64_t s = score_of(ta, tb, m1, m2);
        if (li < 0 || tl_better(s, i, j, ls, li, lj)) { ls = s; li = i; lj = j; }
      }
    }
#pragma omp critical
    {
      if (li >= 0 && (best_i < 0 || tl_better(ls, li, lj, best, best_i, best_j))) {
        best = ls; best_i = li; best_j = lj;
      }
    }
  }
  *bi = best_i; *bj = best_j; *score = best;
  if (best_i >= 0) {
    int32_t ta[9], tb[9];
    table_of(g + best_i * m, g + best_j * m, 0, m1, ta);
    table_of(g + best_i * m, g + best_j * m, m1, m, tb);
    if (countsA) memcpy(countsA, ta, sizeof ta);
    if (countsB) memcpy(countsB, tb, sizeof tb);
  }
  return ORACLE_OK;
}

/* 3x3 tables and score for chosen pairs; tabA/tabB are [np][9]. */
int oracle_twolocus_tables(const int8_t* g, int64_t S, int64_t m1, int64_t m2, const int64_t* I,
                           const int64_t* J, int64_t np, int32_t* tabA, int32_t* tabB, int64_t* score) {
  if (!g || m1 < 1 || m2 < 1 || !I || !J || np < 0 || !tabA || !tabB || !score) return ORACLE_ERR_ARG;
  int64_t m = m1 + m2;
  for (int64_t p = 0; p < np; ++p) {
    if (I[p] < 0 || I[p] >= S || J[p] < 0 || J[p] >= S) return ORACLE_ERR_ARG;
    table_of(g + I[p] * m, g + J[p] * m, 0, m1, tabA + 9 * p);
    table_of(g + I[p] * m, g + J[p] * m, m1, m, tabB + 9 * p);
    score[p] = score_of(tabA + 9 * p, tabB + 9 * p, m1, m2);
  }
  return ORACLE_OK;
}

/* For each chosen SNP r: its best partner j != r (score, then lowest (min, max) pair). */
int oracle_twolocus_rows(const int8_t* g, int64_t S, int64_t m1, int64_t m2, const int64_t* rows,
                         int64_t nr, int64_t* best_j, int64_t* best_score) {
  if (!g || m1 < 1 || m2 < 1 || !rows || nr < 0 || !best_j || !best_score) return ORACLE_ERR_ARG;
  int64_t m = m1 + m2;
  for (int64_t p = 0; p < nr; ++p)
    if (rows[p] < 0 || rows[p] >= S) return ORACLE_ERR_ARG;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < nr; ++p) {
    int64_t r = rows[p], bs = -1, bjj = -1;
    int32_t ta[9], tb[9];
    for (int64_t j = 0; j < S; ++j) {
      if (j == r) continue;
      int64_t lo = r < j ? r : j, hi = r < j ? j : r;
      table_of(g + lo * m, g + hi * m, 0, m1, ta);
      table_of(g + lo * m, g + hi * m, m1, m, tb);
      int64_t s = score_of(ta, tb, m1, m2);
      int64_t blo = bjj < 0 ? 0 : (r < bjj ? r : bjj), bhi = bjj < 0 ? 0 : (r < bjj ? bjj : r);
      if (bjj < 0 || tl_better(s, lo, hi, bs, blo, bhi)) { bs = s; bjj = j; }
    }
    best_j[p] = bjj;
    best_score[p] = bs;
  }
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ Pearson two-locus */
/* Pearson's r of the genotype values (0, 1, 2) of SNPs i and j over the subjects [lo, hi):
 * r = (m Sxy - Sx Sy) / sqrt(vx vy), vx = m Sxx - Sx^2, vy = m Syy - Sy^2, all sums exact in
 * integers (vx and vy each exact in FP64); their product vx vy, which can exceed 2^53, is one
 * rounded FP64 multiplication, followed by the square root and the division; 0 when vx or vy is 0. */
static double pearson_of(const int8_t* gi, const int8_t* gj, int64_t lo, int64_t hi) {
  int64_t sx = 0, sy = 0, sxx = 0, syy = 0, sxy = 0, m = hi - lo;
  for (int64_t t = lo; t < hi; ++t) {
    int64_t x = gi[t], y = gj[t];
    sx += x; sy += y; sxx += x * x; syy += y * y; sxy += x * y;
  }
  int64_t vx = m * sxx - sx * sx, vy = m * syy - sy * sy;
  if (vx == 0 || vy == 0) return 0.0;
  double num = (double)(m * sxy - sx * sy);
  double den = sqrt((double)vx * (double)vy);
  return num / den;
}

static int pearson_better(double s, int64_t i, int64_t j, double bs, int64_t bi, int64_t bj) {
  if (s != bs) return s > bs;
  if (i != bi) return i < bi;
  return j < bj;
}

/* argmax over i < j of |r_A(i,j) - r_B(i,j)| (cases [0, m1), controls [m1, m1 + m2)). */
int oracle_twolocus_pearson(const int8_t* g, int64_t S, int64_t m1, int64_t m2, int64_t* bi, int64_t* bj,
                            double* score) {
  if (!g || S < 0 || m1 < 1 || m2 < 1 || m1 >= (1 << 20) || m2 >= (1 << 20) || !bi || !bj || !score)
    return ORACLE_ERR_ARG;
  int64_t m = m1 + m2;
  if (!geno_ok(g, S, m)) return ORACLE_ERR_ARG;
  double best = -1.0;
  int64_t best_i = -1, best_j = -1;
#pragma omp parallel
  {
    double ls = -1.0;
    int64_t li = -1, lj = -1;
#pragma omp for schedule(dynamic, 8)
    for (int64_t i = 0; i < S; ++i) {
      for (int64_t j = i + 1; j < S; ++j) {
        double ra = pearson_of(g + i * m, g + j * m, 0, m1);
        double rb = pearson_of(g + i * m, g + j * m, m1, m);
        double s = fabs(ra - rb);
        if (li < 0 || pearson_better(s, i, j, ls, li, lj)) { ls = s; li = i; lj = j; }
      }
    }
#pragma omp critical
    {
      if (li >= 0 && (best_i < 0 || pearson_better(ls, li, lj, best, best_i, best_j))) {
        best = ls; best_i = li; best_j = lj;
      }
    }
  }
  *bi = best_i; *bj = best_j; *score = best;
  return ORACLE_OK;
}

/* ------------------------------------------------------------------ Hamming strings */
/* Closest pair (least = 0: fewest mismatches) or least correlated pair (least = 1: most
 * mismatches) of n strings s[i][0..t) over symbols 0 .. sigma-1; ties to the smallest (i, j). */
int oracle_hamming(const uint8_t* s, int64_t n, int64_t t, int64_t sigma, int least, int64_t* bi, int64_t* bj,
                   int64_t* dist) {
  if (!s || n < 0 || t < 1 || sigma < 2 || sigma > 256 || !bi || !bj || !dist) return ORACLE_ERR_ARG;
  for (int64_t e = 0; e < n * t; ++e)
    if ((int64_t)s[e] >= sigma) return ORACLE_ERR_ARG;
  int64_t best = -1, best_i = -1, best_j = -1;
#pragma omp parallel
  {
    int64_t ld = -1, li = -1, lj = -1;
#pragma omp for schedule(dynamic, 8)
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = i + 1; j < n; ++j) {
        int64_t h = 0;
        for (int64_t k = 0; k < t; ++k) h += s[i * t + k] != s[j * t + k];
        int better = li < 0 || (least ? h > ld : h < ld) || (h == ld && (i < li || (i == li && j < lj)));
        if (better) { ld = h; li = i; lj = j; }
      }
    }
#pragma omp critical
    {
      if (li >= 0) {
        int better = best_i < 0 || (least ? ld > best : ld < best) ||
                     (ld == best && (li < best_i || (li == best_i && lj < best_j)));
        if (better) { best = ld; best_i = li; best_j = lj; }
      }
    }
  }
  *bi = best_i; *bj = best_j; *dist = best;
  return ORACLE_OK;
}

/* ---- MLBA, Sec. 4 (closest pair) and Sec. 5.4-5.5 (least correlated pair) ---------------------
 *
 * The rows the algorithm sorts:
 *   least = 0: the n strings themselves, columns 0 .. t-1 (Sec. 4 sorts the strings over the
 *              alphabet directly; no mapping);
 *   least = 1: the 2n columns of the matrix D of Sec. 5.4: row r < n is A'_r, the one-hot string of
 *              string r (symbol a at position p sets bit p*sigma + a, the mapping of Sec. 5.5), and
 *              row n + r is its bitwise complement; columns 0 .. sigma*t - 1.
 * Iteration `it` looks only at the L columns cols[it*L .. it*L + L - 1] (the random draw is made by
 * the caller).  The rows are sorted by their characters in those columns, taken in the given
 * order (ties by row number), so rows with equal characters form runs: the buckets.  Every pair
 * of rows in a bucket is a candidate; for least = 1 only a row A'_i with a complement row of A'_j,
 * i != j.  The pair {i, j} shares a bucket as (A'_i, comp A'_j) exactly when it shares one as
 * (A'_j, comp A'_i) (complementing all characters maps one bucket onto the other), so the oracle
 * counts the representative with i < j: each unordered pair at most once per iteration.
 * Candidates are counted with repetition across iterations.  Verification (the last step of the
 * algorithm) computes the Hamming distance of every candidate on the original strings; the answer
 * is the candidate with the fewest (least = 0) or most (least = 1) mismatches, ties to the smallest
 * (i, j).  No candidate: i = j = -1, mismatches = -1. */

typedef struct {
  const uint8_t* s;
  int64_t n, t, sigma;
  int least;
  const int32_t* cols;  // this iteration's L columns
  int64_t L;
} mlba_ctx;

/* character of row r in column c of the matrix being sorted */
static int mlba_char(const mlba_ctx* q, int64_t r, int64_t c) {
  if (!q->least) return q->s[r * q->t + c];
  const int64_t i = r < q->n ? r : r - q->n;
  const int bit = q->s[i * q->t + c / q->sigma] == (uint8_t)(c % q->sigma);
  return r < q->n ? bit : 1 - bit;
}

/* -1, 0, 1: the rows' characters in the sampled columns, compared in column order */
static int mlba_cmp_key(const mlba_ctx* q, int64_t a, int64_t b) {
  for (int64_t k = 0; k < q->L; ++k) {
    const int ca = mlba_char(q, a, q->cols[k]), cb = mlba_char(q, b, q->cols[k]);
    if (ca != cb) return ca < cb ? -1 : 1;
  }
  return 0;
}

/* bottom-up merge sort of idx[0..m) by (key, row) */
static void mlba_sort(const mlba_ctx* q, int64_t* idx, int64_t* tmp, int64_t m) {
  for (int64_t w = 1; w < m; w *= 2) {
    for (int64_t lo = 0; lo < m; lo += 2 * w) {
      const int64_t mid = lo + w < m ? lo + w : m, hi = lo + 2 * w < m ? lo + 2 * w : m;
      int64_t a = lo, b = mid, o = lo;
      while (a < mid && b < hi) {
        const int c = mlba_cmp_key(q, idx[a], idx[b]);
        if (c < 0 || (c == 0 && idx[a] < idx[b])) tmp[o++] = idx[a++];
        else tmp[o++] = idx[b++];
      }
      while (a < mid) tmp[o++] = idx[a++];
      while (b < hi) tmp[o++] = idx[b++];
    }
    memcpy(idx, tmp, (size_t)m * sizeof(int64_t));
  }
}

int oracle_mlba(const uint8_t* s, int64_t n, int64_t t, int64_t sigma, int least, const int32_t* cols, int64_t iters,
                int64_t L, int64_t* bi, int64_t* bj, int64_t* dist, int64_t* ncand) {
  if (!s || n < 0 || t < 1 || sigma < 2 || sigma > 256 || iters < 0 || L < (least ? 1 : 0) || !bi || !bj || !dist ||
      !ncand || (iters > 0 && L > 0 && !cols))
    return ORACLE_ERR_ARG;
  for (int64_t e = 0; e < n * t; ++e)
    if ((int64_t)s[e] >= sigma) return ORACLE_ERR_ARG;
  const int64_t width = least ? sigma * t : t;
  for (int64_t e = 0; e < iters * L; ++e)
    if (cols[e] < 0 || cols[e] >= width) return ORACLE_ERR_ARG;
  const int64_t m = least ? 2 * n : n;
  int64_t* idx = (int64_t*)malloc((size_t)(m + 1) * sizeof(int64_t));
  int64_t* tmp = (int64_t*)malloc((size_t)(m + 1) * sizeof(int64_t));
  if (!idx || !tmp) { free(idx); free(tmp); return ORACLE_ERR_CAPACITY; }
  int64_t best = -1, best_i = -1, best_j = -1, cand = 0;
  for (int64_t it = 0; it < iters; ++it) {
    mlba_ctx q = {s, n, t, sigma, least, cols ? cols + it * L : NULL, L};
    for (int64_t r = 0; r < m; ++r) idx[r] = r;
    mlba_sort(&q, idx, tmp, m);
    for (int64_t a = 0; a < m;) {
      int64_t b = a + 1;
      while (b < m && mlba_cmp_key(&q, idx[a], idx[b]) == 0) ++b;
      /* bucket idx[a .. b) */
      for (int64_t x = a; x < b; ++x) {
        for (int64_t y = x + 1; y < b; ++y) {
          int64_t i, j;
          if (!least) {
            i = idx[x] < idx[y] ? idx[x] : idx[y];
            j = idx[x] < idx[y] ? idx[y] : idx[x];
          } else {
            const int64_t rx = idx[x], ry = idx[y];
            if ((rx < n) == (ry < n)) continue;  /* two originals or two complements */
            i = rx < n ? rx : ry;                /* the original row */
            j = rx < n ? ry - n : rx - n;        /* the string whose complement it met */
            if (i >= j) continue;                /* the pair is counted as (A'_j, comp A'_i) instead */
          }
          ++cand;
          int64_t h = 0;
          for (int64_t k = 0; k < t; ++k) h += s[i * t + k] != s[j * t + k];
          const int better = best_i < 0 || (least ? h > best : h < best) ||
                             (h == best && (i < best_i || (i == best_i && j < best_j)));
          if (better) { best = h; best_i = i; best_j = j; }
        }
      }
      a = b;
    }
  }
  free(idx);
  free(tmp);
  *bi = best_i; *bj = best_j; *dist = best; *ncand = cand;
  return ORACLE_OK;
}
