/*
 * CPU oracle for the eigenvector back-transformations of the two-stage
 * symmetric / Hermitian eigensolver (arXiv 2002.10991, Eq. 6): tridiagonal
 * -> band (Eq. 6d) and band -> full (Eq. 6e), with the reductions that
 * produce their reflectors.
 *
 * TEST INFRASTRUCTURE ONLY. Plain, slow, obviously correct C in double
 * precision. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does. It shares no code with
 * the CUDA library.
 *
 * Contents
 *   orc_num_reflectors / orc_reflector_rows   store geometry (Sec. 2.2.1)
 *   orc_bulge_chase_{d,z}                     band -> tridiagonal (Eq. 6b)
 *   orc_tridiag_ql                            T X = X Sigma (Eq. 6c), implicit QL
 *   orc_back_transform_{d,z}                  Z = Q^* X (Eq. 6d / Eq. 8)
 *   orc_full_to_band_{d,z}                    full -> band (Eq. 6a)
 *   orc_back_transform_full_{d,z}             C = P^* Y (Eq. 6e)
 *   orc_jacobi                                brute-force dense eigensolver
 */
#define _GNU_SOURCE
#include <complex.h>
#include <sched.h>
#include <unistd.h>
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* store geometry                                                            */
/* ------------------------------------------------------------------------ */

/*
 * Number of reflectors the reduction generates: stage i (0-based, 0..n-3)
 * has ceil((n-i-2)/b) sweeps. The paper prints "(N-i)/b" (Sec. 2.2.1); its
 * own example (N=17, b=4: the fourth stage has 3 sweeps, Fig. 2; reflector
 * (1,4) touches the last four rows, Fig. 3) fixes the count used here.
 * A Hermitian reduction adds one length-1 reflector (stage n-2).
 */
int64_t orc_num_reflectors(int64_t n, int64_t b, int is_complex) {
  int64_t K = 0;
  for (int64_t i = 0; i + 3 <= n; ++i) K += (n - i - 2 + b - 1) / b;
  if (is_complex && n >= 2) K += 1;
  return K;
}

/* First row r_k and length L_k of every reflector, in generation order. */
void orc_reflector_rows(int64_t n, int64_t b, int is_complex, int64_t *r, int64_t *L) {
  int64_t k = 0;
  for (int64_t i = 0; i + 3 <= n; ++i) {
    int64_t ns = (n - i - 2 + b - 1) / b;
    for (int64_t j = 0; j < ns; ++j) {
      r[k] = i + 1 + j * b;
      L[k] = (n - r[k] < b) ? n - r[k] : b;
      ++k;
    }
  }
  if (is_complex && n >= 2) {
    r[k] = n - 1;
    L[k] = 1;
  }
}

/* Stage and sweep of every reflector (for the paper's index facts). */
void orc_reflector_stage_sweep(int64_t n, int64_t b, int is_complex, int64_t *stage, int64_t *sweep) {
  int64_t k = 0;
  for (int64_t i = 0; i + 3 <= n; ++i) {
    int64_t ns = (n - i - 2 + b - 1) / b;
    for (int64_t j = 0; j < ns; ++j) {
      stage[k] = i;
      sweep[k] = j;
      ++k;
    }
  }
  if (is_complex && n >= 2) {
    stage[k] = n - 2;
    sweep[k] = 0;
  }
}

/* ------------------------------------------------------------------------ */
/* the two instantiations                                                    */
/* ------------------------------------------------------------------------ */

#define SCALAR double
#define SFX d
#define CONJ(x) (x)
#define RE(x) (x)
#define IM(x) (0.0 * (x))
#define IS_COMPLEX 0
#include "tbbt_oracle_impl.h"
#undef SCALAR
#undef SFX
#undef CONJ
#undef RE
#undef IM
#undef IS_COMPLEX

#define SCALAR double complex
#define SFX z
#define CONJ(x) conj(x)
#define RE(x) creal(x)
#define IM(x) cimag(x)
#define IS_COMPLEX 1
#include "tbbt_oracle_impl.h"
#undef SCALAR
#undef SFX
#undef CONJ
#undef RE
#undef IM
#undef IS_COMPLEX

/* ------------------------------------------------------------------------ */
/* tridiagonal eigensolver (Eq. 6c): implicit QL with Wilkinson shifts       */
/* ------------------------------------------------------------------------ */

/*
 * Symmetric tridiagonal T (diagonal d[0..n-1], sub-diagonal e[0..n-2]).
 * On return d holds the eigenvalues in ascending order and z (n x n,
 * column-major, ldz) the orthonormal eigenvectors, z[:, k] for d[k].
 * Textbook implicit QL (Golub & Van Loan Sec. 8.3; Numerical Recipes
 * "tqli"): deflate when |e_m| <= eps (|d_m| + |d_{m+1}|), shift by the
 * eigenvalue of the leading 2x2 block closer to d_l, chase the bulge upward
 * with Givens rotations that are accumulated into z. Returns 0, or -1 if an
 * eigenvalue needs more than 30 iterations.
 */
int orc_tridiag_ql(int64_t n, double *d, const double *e_in, double *z, int64_t ldz) {
  double *e = (double *)calloc((size_t)(n + 1), sizeof(double));
  for (int64_t i = 0; i + 1 < n; ++i) e[i] = e_in[i];
  for (int64_t c = 0; c < n; ++c)
    for (int64_t r = 0; r < n; ++r) z[r + c * ldz] = (r == c) ? 1.0 : 0.0;
  int rc = 0;
  for (int64_t l = 0; l < n; ++l) {
    int iter = 0;
    for (;;) {
      int64_t m = l;
      while (m + 1 < n) {
        double dd = fabs(d[m]) + fabs(d[m + 1]);
        if (fabs(e[m]) <= DBL_EPSILON * dd) break;
        ++m;
      }
      if (m == l) break;
      if (++iter > 30) {
        rc = -1;
        goto done;
      }
      /* shift: eigenvalue of [[d_l, e_l], [e_l, d_{l+1}]] closest to d_l */
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double rr = hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? rr : -rr));
      double s = 1.0, c = 1.0, p = 0.0;
      int64_t i;
      int early = 0;
      for (i = m - 1; i >= l; --i) {
        double f = s * e[i];
        double bb = c * e[i];
        rr = hypot(f, g);
        e[i + 1] = rr;
        if (rr == 0.0) { /* underflow: deflate and restart */
          d[i + 1] -= p;
          e[m] = 0.0;
          early = 1;
          break;
        }
        s = f / rr;
        c = g / rr;
        g = d[i + 1] - p;
        rr = (d[i] - g) * s + 2.0 * c * bb;
        p = s * rr;
        d[i + 1] = g + p;
        g = c * rr - bb;
        double *zi = z + i * ldz, *zi1 = z + (i + 1) * ldz;
        for (int64_t k = 0; k < n; ++k) {
          double t = zi1[k];
          zi1[k] = s * zi[k] + c * t;
          zi[k] = c * zi[k] - s * t;
        }
      }
      if (early) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
  /* sort ascending (selection sort, swapping eigenvector columns) */
  for (int64_t i = 0; i + 1 < n; ++i) {
    int64_t k = i;
    for (int64_t j = i + 1; j < n; ++j)
      if (d[j] < d[k]) k = j;
    if (k != i) {
      double t = d[i];
      d[i] = d[k];
      d[k] = t;
      for (int64_t r = 0; r < n; ++r) {
        double u = z[r + i * ldz];
        z[r + i * ldz] = z[r + k * ldz];
        z[r + k * ldz] = u;
      }
    }
  }
done:
  free(e);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* brute force: cyclic Jacobi on a dense real symmetric matrix               */
/* ------------------------------------------------------------------------ */

/*
 * Eigenvalues of the dense symmetric a (n x n, column-major, overwritten)
 * by cyclic Jacobi rotations until the off-diagonal Frobenius norm is below
 * 1e-14 times the Frobenius norm; w gets the eigenvalues ascending, v (if
 * given) the eigenvectors. Hermitian matrices are handled by the caller
 * through the real embedding [[Re, -Im], [Im, Re]] (every eigenvalue twice).
 */
int orc_jacobi(int64_t n, double *a, double *w, double *v) {
  if (v)
    for (int64_t c = 0; c < n; ++c)
      for (int64_t r = 0; r < n; ++r) v[r + c * n] = (r == c) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int64_t i = 0; i < n * n; ++i) fro += a[i] * a[i];
  fro = sqrt(fro);
  int rc = -1;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int64_t c = 0; c < n; ++c)
      for (int64_t r = 0; r < n; ++r)
        if (r != c) off += a[r + c * n] * a[r + c * n];
    if (sqrt(off) <= 1e-14 * fro || fro == 0.0) {
      rc = 0;
      break;
    }
    for (int64_t p = 0; p < n; ++p)
      for (int64_t q = p + 1; q < n; ++q) {
        double apq = a[p + q * n];
        if (apq == 0.0) continue;
        double app = a[p + p * n], aqq = a[q + q * n];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int64_t k = 0; k < n; ++k) { /* columns p, q */
          double akp = a[k + p * n], akq = a[k + q * n];
          a[k + p * n] = c * akp - s * akq;
          a[k + q * n] = s * akp + c * akq;
        }
        for (int64_t k = 0; k < n; ++k) { /* rows p, q */
          double apk = a[p + k * n], aqk = a[q + k * n];
          a[p + k * n] = c * apk - s * aqk;
          a[q + k * n] = s * apk + c * aqk;
        }
        if (v)
          for (int64_t k = 0; k < n; ++k) {
            double vkp = v[k + p * n], vkq = v[k + q * n];
            v[k + p * n] = c * vkp - s * vkq;
            v[k + q * n] = s * vkp + c * vkq;
          }
      }
  }
  for (int64_t i = 0; i < n; ++i) w[i] = a[i + i * n];
  for (int64_t i = 0; i + 1 < n; ++i) /* ascending */
    for (int64_t j = i + 1; j < n; ++j)
      if (w[j] < w[i]) {
        double t = w[i];
        w[i] = w[j];
        w[j] = t;
        if (v)
          for (int64_t k = 0; k < n; ++k) {
            double u = v[k + i * n];
            v[k + i * n] = v[k + j * n];
            v[k + j * n] = u;
          }
      }
  return rc;
}

/* Number of hardware threads this process may run on (for the CPU baseline). */
int orc_num_cpus(void) {
  cpu_set_t set;
  CPU_ZERO(&set);
  if (sched_getaffinity(0, sizeof(set), &set) == 0) {
    int c = CPU_COUNT(&set);
    if (c > 0) return c;
  }
  long c = sysconf(_SC_NPROCESSORS_ONLN);
  return c > 0 ? (int)c : 1;
}
