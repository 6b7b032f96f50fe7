/*
 * FP64 CPU oracle for the kernel-matrix products of kernel quantile
 * regression (Deng, Li, Zhang, arxiv 2510.07929).
 *
 * TEST INFRASTRUCTURE ONLY.  Plain C with OpenMP threads, float64 throughout,
 * kernel entries from their definition (Sec. 1, text after eq. (1.1)):
 *   RBF        k(x, x') = exp(-gamma ||x - x'||_2^2)
 *   Laplacian  k(x, x') = exp(-gamma ||x - x'||_1)
 * with exp from libm.  It exists so that the oracle can form K and K.V at the
 * sizes where numpy's broadcasting is too slow (n = 200000); it shares no
 * code with the CUDA library and is pinned against the numpy oracle
 * (oracle/kqr_oracle.py) by the CPU tests.  No blocking beyond a column
 * buffer, no reordering of the sums: each output is the left-to-right sum
 * over j of k(x_i, x_j) V[j][c].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_COLS 512

/* Squared-Euclidean (kind 0) or L1 (kind 1) distances from the point xi (p
 * coordinates) to the points cols[j0 .. j0 + cnt) of the feature-major array
 * XT (p x nz), written to dist[0 .. cnt). */
static void distances(const double* xi, const double* XT, int64_t nz, int64_t p, int kind, int64_t j0,
                      int64_t cnt, double* dist) {
  for (int64_t j = 0; j < cnt; ++j) dist[j] = 0.0;
  for (int64_t k = 0; k < p; ++k) {
    const double a = xi[k];
    const double* col = XT + k * nz + j0;
    if (kind == 0) {
      for (int64_t j = 0; j < cnt; ++j) {
        const double d = a - col[j];
        dist[j] += d * d;
      }
    } else {
      for (int64_t j = 0; j < cnt; ++j) dist[j] += fabs(a - col[j]);
    }
  }
}

static double* transpose(const double* Z, int64_t nz, int64_t p) {
  double* ZT = (double*)malloc(sizeof(double) * (size_t)(nz * p));
  if (!ZT) return NULL;
  for (int64_t j = 0; j < nz; ++j)
    for (int64_t k = 0; k < p; ++k) ZT[k * nz + j] = Z[j * p + k];
  return ZT;
}

#define ORACLE_ROWS 16

/* U[r][c] = sum_j k(x_{rows[r]}, x_j) V[j][c] for r < nrows (rows == NULL: all n
 * rows, in order), c < m.  X: n x p row-major; V: n x m row-major; U: nrows x m.
 * Rows are taken ORACLE_ROWS at a time so that each slice of X read from memory
 * serves several rows; every output is still the left-to-right sum over j.
 * threads <= 0: the OpenMP default.  Returns 0, or -1 if memory ran out. */
int oracle_kmatvec(const double* X, int64_t n, int64_t p, int kind, double gamma, const double* V, int64_t m,
                   const int64_t* rows, int64_t nrows, double* U, int threads) {
  double* XT = transpose(X, n, p);
  if (!XT) return -1;
  int failed = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  const int64_t nblocks = (nrows + ORACLE_ROWS - 1) / ORACLE_ROWS;
#pragma omp parallel
  {
    double* dist = (double*)malloc(sizeof(double) * ORACLE_ROWS * ORACLE_COLS);
    double* acc = (double*)malloc(sizeof(double) * ORACLE_ROWS * (size_t)m);
    if (!dist || !acc) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int64_t blk = 0; blk < nblocks; ++blk) {
        const int64_t r0 = blk * ORACLE_ROWS;
        const int64_t nr = (nrows - r0 < ORACLE_ROWS) ? nrows - r0 : ORACLE_ROWS;
        for (int64_t q = 0; q < nr * m; ++q) acc[q] = 0.0;
        for (int64_t j0 = 0; j0 < n; j0 += ORACLE_COLS) {
          const int64_t cnt = (n - j0 < ORACLE_COLS) ? n - j0 : ORACLE_COLS;
          for (int64_t q = 0; q < nr; ++q) {
            const int64_t i = rows ? rows[r0 + q] : r0 + q;
            distances(X + i * p, XT, n, p, kind, j0, cnt, dist + q * ORACLE_COLS);
          }
          for (int64_t q = 0; q < nr; ++q) {
            double* aq = acc + q * m;
            const double* dq = dist + q * ORACLE_COLS;
            for (int64_t j = 0; j < cnt; ++j) {
              const double e = exp(-gamma * dq[j]);
              const double* vj = V + (j0 + j) * m;
              for (int64_t c = 0; c < m; ++c) aq[c] += e * vj[c];
            }
          }
        }
        for (int64_t q = 0; q < nr * m; ++q) U[r0 * m + q] = acc[q];
      }
    }
    free(dist);
    free(acc);
  }
  free(XT);
  return failed ? -1 : 0;
}

/* G[i][j] = k(x_i, z_j) for X (nx x p) and Z (nz x p), both row-major; G is
 * nx x nz row-major.  Returns 0, or -1 if memory ran out. */
int oracle_gram(const double* X, int64_t nx, const double* Z, int64_t nz, int64_t p, int kind, double gamma,
                double* G, int threads) {
  double* ZT = transpose(Z, nz, p);
  if (!ZT) return -1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nx; ++i) {
    double* row = G + i * nz;
    for (int64_t j0 = 0; j0 < nz; j0 += ORACLE_COLS) {
      const int64_t cnt = (nz - j0 < ORACLE_COLS) ? nz - j0 : ORACLE_COLS;
      distances(X + i * p, ZT, nz, p, kind, j0, cnt, row + j0);
      for (int64_t j = 0; j < cnt; ++j) row[j0 + j] = exp(-gamma * row[j0 + j]);
    }
  }
  free(ZT);
  return 0;
}

/* Number of threads an OpenMP parallel region uses here (1 without OpenMP). */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
