/*
 * FP64 streamed kernel-matrix products for the oracle.
 * TEST INFRASTRUCTURE ONLY: called from tests/ and the CPU-baseline leg of
 * bench.py, never from the product library.
 *
 * Kernel (arXiv 2109.09817, Sec. 4: "Matern 5/2 kernel"; ARD reading):
 *   r^2 = sum_j ((x_j - x'_j) / l_j)^2       (direct differences, never the
 *                                             norm expansion)
 *   k(x, x') = s (1 + sqrt(5) r + 5 r^2 / 3) exp(-sqrt(5) r)
 * Noisy training covariance (Sec. 2.2, after Eq. pred): K-hat = K + sigma2 I.
 * The products below are the blackbox MVM/MMM of Sec. 3.1-3.2: rows of
 * K-hat are formed one at a time and never stored.
 *
 * Features arrive as float32 (the inputs are float32) and are widened to
 * double exactly; every operation after that is double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double matern52_r2(double r2, double s) {
  double r = sqrt(r2);
  double a = sqrt(5.0) * r;
  return s * (1.0 + a + (5.0 / 3.0) * r2) * exp(-a);
}

static double sqdist(const float* xa, const float* xb, const double* inv_l, int d) {
  double acc = 0.0;
  for (int j = 0; j < d; ++j) {
    double u = ((double)xa[j] - (double)xb[j]) * inv_l[j];
    acc += u * u;
  }
  return acc;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* out[i, c] = sum_b k(x_{rows[i]}, x_b) V[b, c] + sigma2 V[rows[i], c]
 * X: N x d float32 row-major; V: N x t double row-major; out: nrows x t. */
void oracle_khat_rows(const float* X, int64_t N, int d, const double* l,
                      double s, double sigma2, const double* V, int t,
                      const int64_t* rows, int64_t nrows, double* out) {
  double* inv_l = (double*)malloc(sizeof(double) * (size_t)d);
  for (int j = 0; j < d; ++j) inv_l[j] = 1.0 / l[j];
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < nrows; ++i) {
    const int64_t a = rows[i];
    const float* xa = X + a * d;
    double* o = out + i * t;
    for (int c = 0; c < t; ++c) o[c] = sigma2 * V[a * t + c];
    for (int64_t b = 0; b < N; ++b) {
      double kab = matern52_r2(sqdist(xa, X + b * d, inv_l, d), s);
      const double* vb = V + b * t;
      for (int c = 0; c < t; ++c) o[c] += kab * vb[c];
    }
  }
  free(inv_l);
}

/* out[i, c] = sum_b k(x'_i, x_b) V[b, c]   (cross covariance, Eq. pred) */
void oracle_kcross_rows(const float* Xp, int64_t M, const float* X, int64_t N,
                        int d, const double* l, double s, const double* V,
                        int t, double* out) {
  double* inv_l = (double*)malloc(sizeof(double) * (size_t)d);
  for (int j = 0; j < d; ++j) inv_l[j] = 1.0 / l[j];
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < M; ++i) {
    const float* xa = Xp + i * d;
    double* o = out + i * t;
    for (int c = 0; c < t; ++c) o[c] = 0.0;
    for (int64_t b = 0; b < N; ++b) {
      double kab = matern52_r2(sqdist(xa, X + b * d, inv_l, d), s);
      const double* vb = V + b * t;
      for (int c = 0; c < t; ++c) o[c] += kab * vb[c];
    }
  }
  free(inv_l);
}

/* out = K(X1, X2), n1 x n2 row-major, by direct differences. */
void oracle_kernel_block(const float* X1, int64_t n1, const float* X2,
                         int64_t n2, int d, const double* l, double s,
                         double* out) {
  double* inv_l = (double*)malloc(sizeof(double) * (size_t)d);
  for (int j = 0; j < d; ++j) inv_l[j] = 1.0 / l[j];
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n1; ++i) {
    for (int64_t b = 0; b < n2; ++b)
      out[i * n2 + b] = matern52_r2(sqdist(X1 + i * d, X2 + b * d, inv_l, d), s);
  }
  free(inv_l);
}
