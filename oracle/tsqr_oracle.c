/*
 * TSQR oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 Householder QR of a whole m x n matrix, with no
 * reduction tree, no blocking and no reordering.  TSQR reaches exactly this factorization:
 * the product of the tree's orthogonal factors is orthogonal, and the thin QR of a full-rank
 * matrix is unique up to the signs of diag(R) (Sec. 2, the discussion after the parallel
 * factorization equation par4:final).  So the oracle is that definition written out:
 *
 *   geqr2   : for j = 0..n-1, build the reflector H_j = I - tau_j v_j v_j^T that zeroes
 *             column j below the diagonal, then apply it to columns j+1..n-1.  The reflectors
 *             overwrite the strict lower trapezoid and tau is kept apart (Sec. 4.2, the
 *             storage described before Algorithm 1 and in Algorithm 2).
 *   org2r   : thin Q = H_0 H_1 ... H_{n-1} [I_n; 0], applied right to left (Sec. 2: the
 *             m x n thin factor; Sec. 7.2: explicit Q formation).
 *   apply_qt: Q^T B = H_{n-1} ... H_0 B  (Sec. 4.1: applying Q^T is a reduction).
 *   apply_q : Q B   = H_0 ... H_{n-1} B  (Sec. 4.1: applying Q is a broadcast).
 *   signs   : D = diag(sign(R_jj)), sign(0) = +1; R <- D R, Q <- Q D.  The paper fixes no
 *             sign; this is the reading taken for "unique up to signs of diag(R)".
 *
 * Reflector convention (the paper names only a tau array and unit-top vectors [I; Y]):
 *   alpha = x_0, beta = -sign(alpha) * ||x||_2 with sign(0) = +1, tau = (beta - alpha)/beta,
 *   v = x / (alpha - beta) with v_0 = 1.  If ||x_{1:}|| = 0 then tau = 0 (H = I), R_jj = alpha.
 * Norms use two-pass max scaling so that they neither overflow nor underflow.
 *
 * Storage is row-major: element (i, j) of an m x n matrix M with leading dimension ldm is
 * M[i*ldm + j].
 *
 * The loops over the columns a reflector is applied to carry an OpenMP pragma.  The default build
 * ignores it.  A second build with -fopenmp exists only to time the oracle on all host cores.
 * Each column's sums run in the same order either way, so both builds give the same bits.  Only tests/, the smoke check and the CPU-baseline leg of the benchmark may
 * load this library.  It shares no code, header or constant with the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ||x||_2 of len entries spaced inc apart: scale by the largest magnitude, sum squares. */
static double scaled_norm(int64_t len, const double* x, int64_t inc) {
  double mx = 0.0;
  for (int64_t i = 0; i < len; ++i) {
    double a = fabs(x[i * inc]);
    if (a > mx || a != a) mx = a;
  }
  if (mx == 0.0) return 0.0;
  double s = 0.0;
  for (int64_t i = 0; i < len; ++i) {
    double t = x[i * inc] / mx;
    s += t * t;
  }
  return mx * sqrt(s);
}

/* Builds the reflector of x (len entries, stride inc) in place: x_{1:} <- v_{1:}.
 * Returns beta, the entry H x leaves in position 0; *tau receives tau. */
static double make_reflector(int64_t len, double* x, int64_t inc, double* tau) {
  double alpha = x[0];
  double tail = scaled_norm(len - 1, x + inc, inc);
  if (tail == 0.0) {
    *tau = 0.0;
    return alpha;
  }
  double nrm = scaled_norm(len, x, inc);
  double beta = (alpha >= 0.0) ? -nrm : nrm;
  *tau = (beta - alpha) / beta;
  double denom = alpha - beta;
  for (int64_t i = 1; i < len; ++i) x[i * inc] = x[i * inc] / denom;
  return beta;
}

/* Applies H = I - tau v v^T (v_0 = 1, v_{1:} stored in column `col` of V below row `top`)
 * to the k columns of B, rows top..m-1. */
static void apply_reflector(int64_t m, int64_t top, const double* V, int64_t ldv, int64_t col,
                            double tau, int64_t k, double* B, int64_t ldb) {
  if (tau == 0.0) return;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < k; ++c) {
    double w = B[top * ldb + c];
    for (int64_t i = top + 1; i < m; ++i) w += V[i * ldv + col] * B[i * ldb + c];
    B[top * ldb + c] -= tau * w;
    for (int64_t i = top + 1; i < m; ++i) B[i * ldb + c] -= tau * w * V[i * ldv + col];
  }
}

/* Householder QR in place (m >= n).  On return the upper triangle of A holds R and the strict
 * lower trapezoid holds v_{1:} of each reflector; tau[j] holds tau_j. */
void oracle_geqr2(int64_t m, int64_t n, double* A, int64_t lda, double* tau) {
  for (int64_t j = 0; j < n; ++j) {
    double beta = make_reflector(m - j, &A[j * lda + j], lda, &tau[j]);
    A[j * lda + j] = beta;
    if (tau[j] == 0.0) continue;
#pragma omp parallel for schedule(static)
    for (int64_t c = j + 1; c < n; ++c) {
      double w = A[j * lda + c];
      for (int64_t i = j + 1; i < m; ++i) w += A[i * lda + j] * A[i * lda + c];
      A[j * lda + c] -= tau[j] * w;
      for (int64_t i = j + 1; i < m; ++i) A[i * lda + c] -= tau[j] * w * A[i * lda + j];
    }
  }
}

/* Thin Q (m x n) = H_0 ... H_{n-1} [I_n; 0] from the reflectors left by oracle_geqr2. */
void oracle_org2r(int64_t m, int64_t n, const double* V, int64_t ldv, const double* tau,
                  double* Q, int64_t ldq) {
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) Q[i * ldq + c] = (i == c) ? 1.0 : 0.0;
  for (int64_t j = n - 1; j >= 0; --j) apply_reflector(m, j, V, ldv, j, tau[j], n, Q, ldq);
}

/* B (m x k) <- Q^T B = H_{n-1} ... H_0 B. */
void oracle_apply_qt(int64_t m, int64_t n, const double* V, int64_t ldv, const double* tau,
                     int64_t k, double* B, int64_t ldb) {
  for (int64_t j = 0; j < n; ++j) apply_reflector(m, j, V, ldv, j, tau[j], k, B, ldb);
}

/* B (m x k) <- Q B = H_0 ... H_{n-1} B. */
void oracle_apply_q(int64_t m, int64_t n, const double* V, int64_t ldv, const double* tau,
                    int64_t k, double* B, int64_t ldb) {
  for (int64_t j = n - 1; j >= 0; --j) apply_reflector(m, j, V, ldv, j, tau[j], k, B, ldb);
}

/* D_j = sign(R_jj) with sign(0) = +1, read from the diagonal left by oracle_geqr2. */
void oracle_signs(int64_t n, const double* V, int64_t ldv, double* D) {
  for (int64_t j = 0; j < n; ++j) D[j] = (V[j * ldv + j] < 0.0) ? -1.0 : 1.0;
}

/* Full reference: R (n x n, lower zeroed) = D R_raw and, if Q != NULL, thin Q = Q_raw D.
 * V (m x n, ld n) and tau (n) receive the reflectors; D (n) the signs.  A is not modified. */
void oracle_qr(int64_t m, int64_t n, const double* A, int64_t lda, double* V, double* tau,
               double* D, double* R, int64_t ldr, double* Q, int64_t ldq) {
  for (int64_t i = 0; i < m; ++i) memcpy(&V[i * n], &A[i * lda], (size_t)n * sizeof(double));
  oracle_geqr2(m, n, V, n, tau);
  oracle_signs(n, V, n, D);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < n; ++c) R[i * ldr + c] = (c >= i) ? D[i] * V[i * n + c] : 0.0;
  if (Q) {
    oracle_org2r(m, n, V, n, tau, Q, ldq);
    for (int64_t i = 0; i < m; ++i)
      for (int64_t c = 0; c < n; ++c) Q[i * ldq + c] *= D[c];
  }
}

/* ||A - Q R||_F / ||A||_F for A, Q (m x n) and upper triangular R (n x n). */
double oracle_backward_error(int64_t m, int64_t n, const double* A, int64_t lda, const double* Q,
                             int64_t ldq, const double* R, int64_t ldr) {
  /* Both Frobenius norms are taken relative to the largest |A_ic|, so that neither underflows
   * for tiny A nor overflows for huge A; the ratio is the same. */
  double amax = 0.0;
  for (int64_t i = 0; i < m; ++i)
    for (int64_t c = 0; c < n; ++c) {
      double a = fabs(A[i * lda + c]);
      if (a > amax || a != a) amax = a;
    }
  const double scale = (amax > 0.0) ? 1.0 / amax : 1.0;
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    for (int64_t c = 0; c < n; ++c) {
      double s = 0.0;
      for (int64_t p = 0; p <= c; ++p) s += Q[i * ldq + p] * (R[p * ldr + c] * scale);
      double a = A[i * lda + c] * scale;
      double d = a - s;
      num += d * d;
      den += a * a;
    }
  }
  return den > 0.0 ? sqrt(num / den) : sqrt(num);
}

/* ||I - Q^T Q||_F for Q (m x n). */
double oracle_orthogonality(int64_t m, int64_t n, const double* Q, int64_t ldq) {
  double acc = 0.0;
  for (int64_t a = 0; a < n; ++a) {
    for (int64_t b = 0; b < n; ++b) {
      double s = 0.0;
      for (int64_t i = 0; i < m; ++i) s += Q[i * ldq + a] * Q[i * ldq + b];
      double d = ((a == b) ? 1.0 : 0.0) - s;
      acc += d * d;
    }
  }
  return sqrt(acc);
}
