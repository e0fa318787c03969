/*
 * FP64 CPU oracle for the linear-complexity Silhouette (arXiv 2303.14102).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the package smoke check and the
 * bench's CPU-baseline leg use it.  It shares no code, header, table or
 * helper with the CUDA library; the two meet only through arrays produced by
 * the seeded input generators.
 *
 * Everything is plain double-precision C, written for a reader to check
 * against the paper's equations by eye: no blocking, no fusion, no reordering
 * beyond what each equation states.  OpenMP only splits independent points
 * (or independent row ranges of a sum) across threads.
 *
 * Functions and the passages they follow
 *   oracle_aggregate   Sec. III-A Eq. 6 (Psi, sum of squared norms) and
 *                      Eq. 8 (Y, sum of vectors), jointly in one pass as the
 *                      footnote to Eq. 9 states; Sec. III-B Eq. 15-16
 *                      (Omega, sum of normalised vectors) for cosine.
 *   oracle_bruteforce  Sec. II Eq. 1-2 and the mean S; Sec. III Eq. 3 with
 *                      the pairwise distance of Eq. 4 (squared Euclidean) or
 *                      Eq. 12 (cosine distance 1 - cs).  O(N^2 D).  Also the
 *                      plain Euclidean distance (Sec. II names it; the
 *                      Limitations section says the linear method cannot
 *                      give it exactly) and the approximation that section
 *                      suggests: the square root of each point-to-cluster
 *                      mean of squared distances (RMS).
 *   oracle_linear      Sec. III-A Eq. 10-11 and Sec. III-B Eq. 17-18: every
 *                      point scored from the per-cluster aggregates only;
 *                      for the RMS approximation, Eq. 10-11 followed by the
 *                      square root of each mean.
 *   oracle_linear_grad dS/dX of the linear form with labels fixed (the
 *                      derivation is written out in the design notes: the
 *                      paper has no backward pass).
 *
 * Readings of the paper taken here (see the design notes for the list):
 *   - own cluster: the mean over the OTHER n_c - 1 members (Rousseeuw's a_i);
 *     Eq. 3/11/18 divide every cluster by N_k, the self term being zero;
 *   - a point alone in its cluster has s_i = 0 and still counts in N;
 *   - max{a_i, b_i} = 0 gives s_i = 0;
 *   - empty label ids are skipped in the min for b_i;
 *   - fewer than two non-empty clusters: S is NaN, status ORACLE_EDEGENERATE;
 *   - ties in the argmin for b_i go to the lowest cluster index;
 *   - a == b takes the a <= b branch of Eq. 2 (both give 0);
 *   - Eq. 15 normalises by the norm of X_i (the printed ||X|| is a typo);
 *   - the Euclidean approximation of the Limitations section takes the square
 *     root of each point-to-cluster mean of SQUARED distances (own cluster
 *     over n_c - 1 as above); a negative rounding residue of that mean is 0.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL 1
#define ORACLE_ELABEL 2
#define ORACLE_EDEGENERATE 3
#define ORACLE_EZERONORM 4

#define METRIC_SQEUCLIDEAN 0
#define METRIC_COSINE 1
#define METRIC_EUCLIDEAN 2     /* exact ||x - y||: quadratic form only */
#define METRIC_EUCLIDEAN_RMS 3 /* sqrt of the mean squared distance to a cluster */

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the OpenMP loops below from now on (n >= 1; 1 = one thread). */
void oracle_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

static int check_labels(const int32_t* labels, int64_t N, int32_t K) {
  for (int64_t i = 0; i < N; ++i)
    if (labels[i] < 0 || labels[i] >= K) return ORACLE_ELABEL;
  return ORACLE_OK;
}

/* Euclidean norm of one row (Eq. 12 denominator / Eq. 15). */
static double row_norm(const double* x, int32_t D) {
  double s = 0.0;
  for (int32_t l = 0; l < D; ++l) s += x[l] * x[l];
  return sqrt(s);
}

static int check_norms(const double* X, int64_t N, int32_t D) {
  for (int64_t i = 0; i < N; ++i)
    if (row_norm(X + i * D, D) == 0.0) return ORACLE_EZERONORM;
  return ORACLE_OK;
}

static int metric_ok(int metric) { return metric >= METRIC_SQEUCLIDEAN && metric <= METRIC_EUCLIDEAN_RMS; }

/* Pairwise distance: Eq. 4 left-hand side (squared Euclidean, also what the
 * RMS approximation averages), its square root (Euclidean), or 1 - cs with
 * cs from Eq. 12 (cosine). */
static double pair_distance(const double* x, const double* y, int32_t D, int metric) {
  if (metric != METRIC_COSINE) {
    double s = 0.0;
    for (int32_t l = 0; l < D; ++l) {
      double t = x[l] - y[l];
      s += t * t;
    }
    return metric == METRIC_EUCLIDEAN ? sqrt(s) : s;
  }
  double dot = 0.0;
  for (int32_t l = 0; l < D; ++l) dot += x[l] * y[l];
  return 1.0 - dot / (row_norm(x, D) * row_norm(y, D));
}

/* Mean distance from a point to a cluster, from the summed distance and the
 * number of members it runs over (Eq. 3, Eq. 11, Eq. 18).  The RMS
 * approximation then takes the square root of that mean of squared distances
 * (a mean of squares is >= 0: a negative rounding residue of the expanded
 * Eq. 10 counts as 0). */
static double cluster_mean(double summed, double members, int metric) {
  double m = summed / members;
  if (metric == METRIC_EUCLIDEAN_RMS) return m > 0.0 ? sqrt(m) : 0.0;
  return m;
}

/* Eq. 1 / Eq. 2 with the readings above. */
static double silhouette_of(double a, double b) {
  double m = a > b ? a : b;
  if (m == 0.0) return 0.0;
  if (a <= b) return 1.0 - a / b;
  return b / a - 1.0;
}

/*
 * Per-cluster aggregates in one pass over the data.
 *   sq-Euclidean: count[k] = N_k, s1[k*D+l] = Y_{k,l} (Eq. 8),
 *                 s2[k] = Psi_k = sum of xi_{C_j} (Eq. 5-6).
 *   cosine:       count[k] = N_k, s1[k*D+l] = Omega_{k,l} (Eq. 16) with the
 *                 normalised vectors of Eq. 15, s2[k] = sum of ||x_hat||^2.
 * Rows are split into fixed contiguous ranges, one per thread, and the
 * per-thread sums are added in thread order, so the result is deterministic
 * for a given thread count.
 */
int oracle_aggregate(const double* X, int64_t N, int32_t D, const int32_t* labels,
                     int32_t K, int metric, int64_t* count, double* s1, double* s2) {
  if (N < 0 || D <= 0 || K <= 0 || !metric_ok(metric)) return ORACLE_EINVAL;
  int st = check_labels(labels, N, K);
  if (st) return st;
  if (metric == METRIC_COSINE && (st = check_norms(X, N, D))) return st;
  int T = oracle_num_threads();
  int64_t* cnt_t = (int64_t*)calloc((size_t)T * K, sizeof(int64_t));
  double* s1_t = (double*)calloc((size_t)T * K * D, sizeof(double));
  double* s2_t = (double*)calloc((size_t)T * K, sizeof(double));
  if (!cnt_t || !s1_t || !s2_t) {
    free(cnt_t); free(s1_t); free(s2_t);
    return ORACLE_EINVAL;
  }
#pragma omp parallel num_threads(T)
  {
    int t = 0;
#ifdef _OPENMP
    t = omp_get_thread_num();
#endif
    int64_t lo = N * t / T, hi = N * (t + 1) / T;
    for (int64_t i = lo; i < hi; ++i) {
      const double* x = X + i * D;
      int32_t k = labels[i];
      double scale = 1.0;
      if (metric == METRIC_COSINE) scale = 1.0 / row_norm(x, D);
      double sq = 0.0;
      for (int32_t l = 0; l < D; ++l) {
        double v = x[l] * scale;
        s1_t[((size_t)t * K + k) * D + l] += v;
        sq += v * v;
      }
      s2_t[(size_t)t * K + k] += sq;
      cnt_t[(size_t)t * K + k] += 1;
    }
  }
  for (int32_t k = 0; k < K; ++k) {
    count[k] = 0;
    s2[k] = 0.0;
    for (int32_t l = 0; l < D; ++l) s1[(size_t)k * D + l] = 0.0;
  }
  for (int t = 0; t < T; ++t)
    for (int32_t k = 0; k < K; ++k) {
      count[k] += cnt_t[(size_t)t * K + k];
      s2[k] += s2_t[(size_t)t * K + k];
      for (int32_t l = 0; l < D; ++l) s1[(size_t)k * D + l] += s1_t[((size_t)t * K + k) * D + l];
    }
  free(cnt_t); free(s1_t); free(s2_t);
  return ORACLE_OK;
}

static int count_nonempty(const int64_t* count, int32_t K) {
  int ne = 0;
  for (int32_t k = 0; k < K; ++k) ne += count[k] > 0;
  return ne;
}

/*
 * Standard quadratic Silhouette straight from the definition: for every point
 * the mean distance to every cluster (Eq. 3) from all N pairwise distances,
 * a_i over the other members of its own cluster, b_i the smallest mean over
 * the other non-empty clusters, s_i by Eq. 2, S the mean of all s_i.
 * Outputs s, a, b (double[N]) and kstar (int32[N], the argmin cluster of b_i)
 * may be NULL.  *S_out receives S, or NaN when fewer than two clusters are
 * non-empty.
 */
int oracle_bruteforce(const double* X, int64_t N, int32_t D, const int32_t* labels,
                      int32_t K, int metric, double* s, double* a, double* b,
                      int32_t* kstar, double* S_out) {
  if (N < 0 || D <= 0 || K <= 0 || !metric_ok(metric)) return ORACLE_EINVAL;
  int st = check_labels(labels, N, K);
  if (st) return st;
  if (metric == METRIC_COSINE && (st = check_norms(X, N, D))) return st;
  int64_t* count = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  for (int64_t i = 0; i < N; ++i) count[labels[i]] += 1;
  int degenerate = count_nonempty(count, K) < 2;
  double total = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : total)
  for (int64_t i = 0; i < N; ++i) {
    double* sums = (double*)calloc((size_t)K, sizeof(double));
    const double* xi = X + i * D;
    for (int64_t j = 0; j < N; ++j) {
      if (j == i) continue; /* a_i excludes the point itself */
      sums[labels[j]] += pair_distance(xi, X + j * D, D, metric);
    }
    int32_t c = labels[i];
    double ai = count[c] > 1 ? cluster_mean(sums[c], (double)(count[c] - 1), metric) : 0.0;
    double bi = INFINITY;
    int32_t kb = -1;
    for (int32_t k = 0; k < K; ++k) {
      if (k == c || count[k] == 0) continue;
      double m = cluster_mean(sums[k], (double)count[k], metric);
      if (m < bi) { bi = m; kb = k; }
    }
    double si = (count[c] > 1 && kb >= 0) ? silhouette_of(ai, bi) : 0.0;
    if (s) s[i] = si;
    if (a) a[i] = ai;
    if (b) b[i] = bi;
    if (kstar) kstar[i] = kb;
    total += si;
    free(sums);
  }
  free(count);
  if (S_out) *S_out = degenerate ? NAN : (N > 0 ? total / (double)N : NAN);
  return degenerate ? ORACLE_EDEGENERATE : ORACLE_OK;
}

/*
 * Linear-complexity scoring from the aggregates of oracle_aggregate.
 * For a point X_i and a cluster k the summed distance is
 *   sq-Euclidean (Eq. 10): N_k xi_i + Psi_k - 2 sum_l Y_{k,l} x_{il}
 *   cosine       (Eq. 17): N_k - sum_l xihat_{il} Omega_{k,l}
 * and the mean divides it by N_k (Eq. 11 / Eq. 18) for the other clusters,
 * by N_c - 1 for the point's own cluster c (the self term is zero).
 * Scores the M points listed in idx (all N points when idx is NULL);
 * outputs are indexed like idx.
 */
int oracle_linear(const double* X, int64_t N, int32_t D, const int32_t* labels, int32_t K,
                  int metric, const int64_t* count, const double* s1, const double* s2,
                  const int64_t* idx, int64_t M, double* s, double* a, double* b,
                  int32_t* kstar) {
  /* the plain Euclidean distance has no aggregate form (Limitations) */
  if (N < 0 || D <= 0 || K <= 0 || !metric_ok(metric) || metric == METRIC_EUCLIDEAN) return ORACLE_EINVAL;
  if (!idx) M = N;
  int st = ORACLE_OK;
  for (int64_t q = 0; q < M; ++q) {
    int64_t i = idx ? idx[q] : q;
    if (i < 0 || i >= N) return ORACLE_EINVAL;
    if (labels[i] < 0 || labels[i] >= K) return ORACLE_ELABEL;
    if (metric == METRIC_COSINE && row_norm(X + i * D, D) == 0.0) return ORACLE_EZERONORM;
  }
  int degenerate = count_nonempty(count, K) < 2;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < M; ++q) {
    int64_t i = idx ? idx[q] : q;
    const double* x = X + i * D;
    int32_t c = labels[i];
    double xi_sq = 0.0; /* Eq. 5 */
    for (int32_t l = 0; l < D; ++l) xi_sq += x[l] * x[l];
    double inv_norm = 1.0 / sqrt(xi_sq); /* Eq. 15, cosine only */
    double ai = 0.0, bi = INFINITY;
    int32_t kb = -1;
    for (int32_t k = 0; k < K; ++k) {
      if (count[k] == 0) continue;
      double dot = 0.0;
      for (int32_t l = 0; l < D; ++l) dot += s1[(size_t)k * D + l] * x[l];
      double numer;
      if (metric != METRIC_COSINE)
        numer = (double)count[k] * xi_sq + s2[k] - 2.0 * dot; /* Eq. 10 */
      else
        numer = (double)count[k] - dot * inv_norm; /* Eq. 17 */
      if (k == c) {
        ai = count[c] > 1 ? cluster_mean(numer, (double)(count[c] - 1), metric) : 0.0;
      } else {
        double m = cluster_mean(numer, (double)count[k], metric); /* Eq. 11 / Eq. 18 */
        if (m < bi) { bi = m; kb = k; }
      }
    }
    double si = (count[c] > 1 && kb >= 0) ? silhouette_of(ai, bi) : 0.0;
    if (s) s[q] = si;
    if (a) a[q] = ai;
    if (b) b[q] = bi;
    if (kstar) kstar[q] = kb;
  }
  (void)st;
  return degenerate ? ORACLE_EDEGENERATE : ORACLE_OK;
}

/* ds/da and ds/db of Eq. 2 at (a, b); zero where s is pinned to 0. */
static void silhouette_partials(double a, double b, double* dsa, double* dsb) {
  double m = a > b ? a : b;
  if (m == 0.0) { *dsa = 0.0; *dsb = 0.0; return; }
  if (a <= b) { *dsa = -1.0 / b; *dsb = a / (b * b); }
  else { *dsa = -b / (a * a); *dsb = 1.0 / a; }
}

/*
 * dS/dX (times gS) of the Silhouette with labels fixed and the b_i argmin
 * k*_i held at its value (a subgradient at ties), via per-cluster sums:
 *   alpha_i = (ds_i/da_i)/(N_c - 1),  beta_i = (ds_i/db_i)/N_{k*_i}
 *   A_k = sum_{c(i)=k} alpha_i,  P_k = sum_{c(i)=k} alpha_i v_i
 *   B_k = sum_{k*_i=k} beta_i,   Q_k = sum_{k*_i=k} beta_i v_i
 * with v = x (sq-Euclidean) or x_hat (cosine).  For a point m in cluster c
 * with neighbour k* = k*_m:
 *   sq-Euclidean  dS/dx_m = (2/N)[alpha_m (N_c x_m - Y_c)
 *                      + beta_m (N_k* x_m - Y_k*) + A_c x_m - P_c + B_c x_m - Q_c]
 *   cosine        g = -(1/N)[alpha_m Omega_c + beta_m Omega_k* + P_c + Q_c],
 *                 dS/dx_m = (g - x_hat (x_hat . g)) / ||x_m||.
 * Writes dX (double[N*D]).  Returns the scoring status.
 */
int oracle_linear_grad(const double* X, int64_t N, int32_t D, const int32_t* labels,
                       int32_t K, int metric, double gS, double* dX) {
  if (N <= 0 || D <= 0 || K <= 0) return ORACLE_EINVAL;
  if (metric != METRIC_SQEUCLIDEAN && metric != METRIC_COSINE) return ORACLE_EINVAL;
  int64_t* count = (int64_t*)calloc((size_t)K, sizeof(int64_t));
  double* s1 = (double*)calloc((size_t)K * D, sizeof(double));
  double* s2 = (double*)calloc((size_t)K, sizeof(double));
  double* a = (double*)malloc((size_t)N * sizeof(double));
  double* b = (double*)malloc((size_t)N * sizeof(double));
  int32_t* ks = (int32_t*)malloc((size_t)N * sizeof(int32_t));
  double* alpha = (double*)calloc((size_t)N, sizeof(double));
  double* beta = (double*)calloc((size_t)N, sizeof(double));
  double* A = (double*)calloc((size_t)K, sizeof(double));
  double* Bs = (double*)calloc((size_t)K, sizeof(double));
  double* P = (double*)calloc((size_t)K * D, sizeof(double));
  double* Q = (double*)calloc((size_t)K * D, sizeof(double));
  int st = oracle_aggregate(X, N, D, labels, K, metric, count, s1, s2);
  if (st == ORACLE_OK) st = oracle_linear(X, N, D, labels, K, metric, count, s1, s2, NULL, N,
                                          NULL, a, b, ks);
  if (st == ORACLE_OK) {
    for (int64_t i = 0; i < N; ++i) {
      int32_t c = labels[i];
      if (count[c] < 2 || ks[i] < 0) continue; /* s_i pinned to 0 */
      double dsa, dsb;
      silhouette_partials(a[i], b[i], &dsa, &dsb);
      alpha[i] = dsa / (double)(count[c] - 1);
      beta[i] = dsb / (double)count[ks[i]];
    }
    for (int64_t i = 0; i < N; ++i) {
      const double* x = X + i * D;
      double sc = metric == METRIC_COSINE ? 1.0 / row_norm(x, D) : 1.0;
      int32_t c = labels[i];
      A[c] += alpha[i];
      for (int32_t l = 0; l < D; ++l) P[(size_t)c * D + l] += alpha[i] * x[l] * sc;
      if (ks[i] >= 0) {
        Bs[ks[i]] += beta[i];
        for (int32_t l = 0; l < D; ++l) Q[(size_t)ks[i] * D + l] += beta[i] * x[l] * sc;
      }
    }
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < N; ++m) {
      const double* x = X + m * D;
      double* g = dX + m * D;
      int32_t c = labels[m];
      int32_t k = ks[m];
      if (metric == METRIC_SQEUCLIDEAN) {
        for (int32_t l = 0; l < D; ++l) {
          double v = A[c] * x[l] - P[(size_t)c * D + l] + Bs[c] * x[l] - Q[(size_t)c * D + l];
          if (alpha[m] != 0.0) v += alpha[m] * ((double)count[c] * x[l] - s1[(size_t)c * D + l]);
          if (k >= 0 && beta[m] != 0.0) v += beta[m] * ((double)count[k] * x[l] - s1[(size_t)k * D + l]);
          g[l] = gS * 2.0 / (double)N * v;
        }
      } else {
        double nrm = row_norm(x, D);
        double proj = 0.0;
        for (int32_t l = 0; l < D; ++l) {
          double v = P[(size_t)c * D + l] + Q[(size_t)c * D + l];
          if (alpha[m] != 0.0) v += alpha[m] * s1[(size_t)c * D + l];
          if (k >= 0 && beta[m] != 0.0) v += beta[m] * s1[(size_t)k * D + l];
          g[l] = -v / (double)N;
          proj += g[l] * x[l] / nrm;
        }
        for (int32_t l = 0; l < D; ++l) g[l] = gS * (g[l] - proj * x[l] / nrm) / nrm;
      }
    }
  }
  free(count); free(s1); free(s2); free(a); free(b); free(ks);
  free(alpha); free(beta); free(A); free(Bs); free(P); free(Q);
  return st;
}
