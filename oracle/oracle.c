/*
 * oracle.c -- plain FP64 CPU oracle for randomized blocked QR with column
 * pivoting and its orthonormal-pivot (URV) variant (Martinsson 2015).
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path. It shares no code
 * with the CUDA library. Loops are written out in the order the paper states
 * the steps; OpenMP only splits independent columns across threads, which does
 * not change any rounding (each output element is computed by one thread in a
 * fixed order).
 *
 * Readings of the paper adopted here (the paper is silent or garbled):
 *  - sign(0) = +1 in the reflector of Sec. 3.1; a zero vector gives H = I.
 *  - Fig. "QR" pivots by the FP64 sum of squares of the remaining rows,
 *    recomputed every step; ties go to the lowest position. A column of
 *    length 1 gets no reflector (n-1 steps for square input, Sec. 3.2).
 *  - Inside a blockQR panel no second pivoting is done (P^ = I).
 *  - The sketch is carried from block to block by the downdate
 *    Y <- Y(:,b:) - (G Q~)(:, :b) R12 (not in the paper; exact in real
 *    arithmetic) or re-drawn per block (the paper's literal Fig. blockQR).
 *  - p is the over-sampling parameter (Sec. 4.3 calls it r); l = b + p.
 *  - URV: orthonormalisation between power steps (Sec. 6.3 prints the power
 *    without it) and the l -> b reduction through the SVD of the sketch's R.
 *  - Sec. 6.2 completion of Vt for a zero singular value: the first unit
 *    vector left with norm above 1/2 by Gram-Schmidt, else the largest.
 *
 * What pins each routine (tests/test_oracle_pins.py, CPU), other than itself:
 *  orc_house         the worked examples of Sec. 3.1, the unit-vector form of H
 *  orc_qrcp          closed-form pivots of orthogonal columns, brute-force
 *                    greedy selection on tiny inputs, LAPACK dgeqp3 (scipy)
 *  orc_geqr2         LAPACK dgeqrf (scipy)
 *  orc_larft         the product of the reflectors; T^-1 = diag(1/tau) +
 *                    striu(V^T V) and its back substitution
 *  orc_apply_block   the product of the reflectors
 *  orc_rqrcp(_ex)    G = I reduces it to Fig. QR; the sketch stays G X''; gap-
 *                    separated pivot sets; ||R||_F = ||A||_F, sum log|R_ii|
 *  orc_rurv(_diag)   Eckart-Young lower bounds, the gap case, diagonal blocks
 *                    equal to the SVDs (LAPACK) of the undiagonalised blocks
 *  orc_reduce_sketch the projector onto the b dominant left singular
 *                    vectors of Z (numpy SVD), on inputs where it differs
 *                    by O(1) from the span of Z's first b columns
 *  orc_jacobi_svd    LAPACK SVD (numpy)
 *  orc_complete_column  orthonormality, and the all-ones complement case
 *  orc_philox4x32_10 the published known-answer vectors
 *  orc_gauss_fill    moments of N(0, 1) and prefix consistency of the stream
 * Parity unpinned (statistical only): the paper's qualitative Sec. 7 claims.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

static double sgn0(double x) { return x < 0.0 ? -1.0 : 1.0; }

static void* xcalloc(size_t n, size_t s) {
  void* p = calloc(n ? n : 1, s);
  if (!p) abort();
  return p;
}

/* ------------------------------------------------------------------ Sec. 3.1 */
void orc_house(int k, const double* a, int inca, double* v, double* tau, double* beta) {
  if (k <= 0) { *tau = 0.0; *beta = 0.0; return; }
  double alpha = a[0];
  double s = 0.0;
  for (int i = 0; i < k; ++i) s += a[(size_t)i * inca] * a[(size_t)i * inca];
  double nrm = sqrt(s);
  v[0] = 1.0;
  if (nrm == 0.0) {
    for (int i = 1; i < k; ++i) v[i] = 0.0;
    *tau = 0.0;
    *beta = 0.0;
    return;
  }
  double bt = -sgn0(alpha) * nrm;
  double d = alpha - bt;
  for (int i = 1; i < k; ++i) v[i] = a[(size_t)i * inca] / d;
  *tau = (bt - alpha) / bt;
  *beta = bt;
}

/* H = I - tau v v^T applied from the left to rows r0..r0+k-1 of columns c0..c1-1. */
static void apply_house_left(int k, const double* v, double tau, double* A, int lda, int r0, int c0, int c1) {
  if (tau == 0.0) return;
#pragma omp parallel for schedule(static)
  for (int c = c0; c < c1; ++c) {
    double* col = A + IX(r0, c, lda);
    double w = 0.0;
    for (int i = 0; i < k; ++i) w += v[i] * col[i];
    w *= tau;
    for (int i = 0; i < k; ++i) col[i] -= w * v[i];
  }
}

static void swap_cols(double* A, int lda, int rows, int c1, int c2) {
  if (c1 == c2) return;
  double* x = A + IX(0, c1, lda);
  double* y = A + IX(0, c2, lda);
  for (int i = 0; i < rows; ++i) { double t = x[i]; x[i] = y[i]; y[i] = t; }
}

/* Fig. "QR" restricted to rows r0..m-1 and columns c0..c1-1; swaps move whole
 * columns (all m rows, `rows_all`) and perm entries. At most max_steps steps. */
static void qrcp_range(int m, double* A, int lda, int rows_all, int r0, int c0, int c1, int* perm,
                       double* tau, int max_steps) {
  int nc = c1 - c0, mr = m - r0;
  int steps = nc < mr - 1 ? nc : mr - 1;
  if (steps < 0) steps = 0;
  if (max_steps >= 0 && steps > max_steps) steps = max_steps;
  double* v = (double*)xcalloc((size_t)(mr > 0 ? mr : 1), sizeof(double));
  for (int j = 0; j < steps; ++j) {
    int row = r0 + j, col = c0 + j;
    int best = col;
    double bestn = -1.0;
    for (int c = col; c < c1; ++c) {
      const double* x = A + IX(0, c, lda);
      double s = 0.0;
      for (int i = row; i < m; ++i) s += x[i] * x[i];
      if (s > bestn) { bestn = s; best = c; }
    }
    if (best != col) {
      swap_cols(A, lda, rows_all, best, col);
      if (perm) { int t = perm[best]; perm[best] = perm[col]; perm[col] = t; }
    }
    double t, bt;
    orc_house(m - row, A + IX(row, col, lda), 1, v, &t, &bt);
    apply_house_left(m - row, v, t, A, lda, row, col + 1, c1);
    A[IX(row, col, lda)] = bt;
    for (int i = 1; i < m - row; ++i) A[IX(row + i, col, lda)] = v[i];
    if (tau) tau[j] = t;
  }
  if (tau)
    for (int j = steps; j < nc; ++j) tau[j] = 0.0;
  free(v);
}

void orc_qrcp(int m, int n, double* A, int lda, int* perm, double* tau) {
  for (int j = 0; j < n; ++j) perm[j] = j;
  qrcp_range(m, A, lda, m, 0, 0, n, perm, tau, -1);
}

/* ------------------------------------------------------------------ Sec. 3.2 */
void orc_geqr2(int m, int n, double* A, int lda, double* tau) {
  int steps = n < m - 1 ? n : m - 1;
  if (steps < 0) steps = 0;
  double* v = (double*)xcalloc((size_t)(m > 0 ? m : 1), sizeof(double));
  for (int j = 0; j < steps; ++j) {
    double t, bt;
    orc_house(m - j, A + IX(j, j, lda), 1, v, &t, &bt);
    apply_house_left(m - j, v, t, A, lda, j, j + 1, n);
    A[IX(j, j, lda)] = bt;
    for (int i = 1; i < m - j; ++i) A[IX(j + i, j, lda)] = v[i];
    tau[j] = t;
  }
  for (int j = steps; j < n; ++j) tau[j] = 0.0;
  free(v);
}

/* V(i,j) of a unit lower trapezoidal V stored LAPACK-style. */
static double vget(const double* V, int ldv, int i, int j) {
  if (i < j) return 0.0;
  if (i == j) return 1.0;
  return V[IX(i, j, ldv)];
}

/* ----------------------------------------------------- Sec. 5.1, WY remark */
void orc_larft(int m, int k, const double* V, int ldv, const double* tau, double* T, int ldt) {
  double* w = (double*)xcalloc((size_t)(k > 0 ? k : 1), sizeof(double));
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < k; ++i) T[IX(i, j, ldt)] = 0.0;
    T[IX(j, j, ldt)] = tau[j];
    /* w = V(:, 0:j)^T v_j */
    for (int i = 0; i < j; ++i) {
      double s = 0.0;
      for (int r = j; r < m; ++r) s += vget(V, ldv, r, i) * vget(V, ldv, r, j);
      w[i] = s;
    }
    /* T(0:j, j) = -tau_j T(0:j, 0:j) w */
    for (int i = 0; i < j; ++i) {
      double s = 0.0;
      for (int l = i; l < j; ++l) s += T[IX(i, l, ldt)] * w[l];
      T[IX(i, j, ldt)] = -tau[j] * s;
    }
  }
  free(w);
}

void orc_apply_block(int m, int n, int k, const double* V, int ldv, const double* T, int ldt, int trans,
                     double* C, int ldc) {
  if (k <= 0 || m <= 0 || n <= 0) return;
#pragma omp parallel
  {
    double* w = (double*)xcalloc((size_t)k, sizeof(double));
    double* w2 = (double*)xcalloc((size_t)k, sizeof(double));
#pragma omp for schedule(static)
    for (int c = 0; c < n; ++c) {
      double* col = C + IX(0, c, ldc);
      /* w = V^T c */
      for (int i = 0; i < k; ++i) {
        double s = 0.0;
        for (int r = i; r < m; ++r) s += vget(V, ldv, r, i) * col[r];
        w[i] = s;
      }
      /* w2 = T w (trans = 0) or T^T w (trans = 1) */
      for (int i = 0; i < k; ++i) {
        double s = 0.0;
        if (!trans)
          for (int l = i; l < k; ++l) s += T[IX(i, l, ldt)] * w[l];
        else
          for (int l = 0; l <= i; ++l) s += T[IX(l, i, ldt)] * w[l];
        w2[i] = s;
      }
      /* c -= V w2 */
      for (int i = 0; i < k; ++i) {
        double s = w2[i];
        if (s == 0.0) continue;
        for (int r = i; r < m; ++r) col[r] -= vget(V, ldv, r, i) * s;
      }
    }
    free(w);
    free(w2);
  }
}

/* C (r x c) = A (r x kk) * B (kk x c), all column-major, plain loops. */
static void matmul_nn(int r, int c, int kk, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < c; ++j) {
    double* cj = C + IX(0, j, ldc);
    for (int i = 0; i < r; ++i) cj[i] = 0.0;
    for (int l = 0; l < kk; ++l) {
      double bl = B[IX(l, j, ldb)];
      const double* al = A + IX(0, l, lda);
      for (int i = 0; i < r; ++i) cj[i] += al[i] * bl;
    }
  }
}

/* C (r x c) = A^T B with A (kk x r), B (kk x c). */
static void matmul_tn(int r, int c, int kk, const double* A, int lda, const double* B, int ldb, double* C, int ldc) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < c; ++j) {
    const double* bj = B + IX(0, j, ldb);
    for (int i = 0; i < r; ++i) {
      const double* ai = A + IX(0, i, lda);
      double s = 0.0;
      for (int l = 0; l < kk; ++l) s += ai[l] * bj[l];
      C[IX(i, j, ldc)] = s;
    }
  }
}

/* ------------------------------------------------ Sec. 4.1, 4.3, 5.1, 5.2 */
int orc_rqrcp(int m, int n, double* A, int lda, int b, int p, const double* G, int ldg, int mode, double* T,
              int ldt, int* perm, int max_blocks) {
  return orc_rqrcp_ex(m, n, A, lda, b, p, G, ldg, mode, T, ldt, perm, max_blocks, NULL, NULL);
}

int orc_rqrcp_ex(int m, int n, double* A, int lda, int b, int p, const double* G, int ldg, int mode, double* T,
                 int ldt, int* perm, int max_blocks, double* Yout, double* Gout) {
  const int l = b + p;
  for (int j = 0; j < n; ++j) perm[j] = j;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < b; ++i) T[IX(i, j, ldt)] = 0.0;
  double* Y = (double*)xcalloc((size_t)l * n, sizeof(double));  /* l x n', ld l */
  double* Yw = (double*)xcalloc((size_t)l * n, sizeof(double));
  double* Gc = NULL;                                            /* current G, l x m', ld l */
  double* tau = (double*)xcalloc((size_t)b, sizeof(double));
  double* v = (double*)xcalloc((size_t)l, sizeof(double));
  size_t goff = 0;
  if (mode == ORC_SKETCH_DOWNDATE) {
    Gc = (double*)xcalloc((size_t)l * m, sizeof(double));
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < l; ++i) Gc[IX(i, c, l)] = G[IX(i, c, ldg)];
    /* Y = G A (Sec. 4.1: Y^T = A^T Omega with Omega = G^T) */
    matmul_nn(l, n, m, Gc, l, A, lda, Y, l);
  }
  int k0 = 0, blocks = 0;
  while (k0 < n) {
    if (max_blocks > 0 && blocks >= max_blocks) break;
    const int np = n - k0, mp = m - k0;
    if (np <= b) {
      /* Fig. blockQR, final step: classical pivoted QR of the remaining block. */
      double* tq = (double*)xcalloc((size_t)np, sizeof(double));
      qrcp_range(m, A, lda, m, k0, k0, n, perm, tq, -1);
      orc_larft(mp, np, A + IX(k0, k0, lda), lda, tq, T + IX(0, k0, ldt), ldt);
      free(tq);
      k0 = n;
      ++blocks;
      break;
    }
    const int bi = b;
    if (mode == ORC_SKETCH_RESAMPLE) {
      /* Y = G_i A(k0:m, k0:n), the paper's re-sketch of the remaining block */
      matmul_nn(l, np, mp, G + goff, l, A + IX(k0, k0, lda), lda, Y, l);
      goff += (size_t)l * mp;
    }
    /* Sec. 4.1/4.3: first b steps of Fig. "QR" on a working copy of Y. */
    memcpy(Yw, Y, sizeof(double) * (size_t)l * np);
    for (int j = 0; j < bi; ++j) {
      int best = j;
      double bestn = -1.0;
      for (int c = j; c < np; ++c) {
        double s = 0.0;
        for (int i = j; i < l; ++i) s += Yw[IX(i, c, l)] * Yw[IX(i, c, l)];
        if (s > bestn) { bestn = s; best = c; }
      }
      if (best != j) {
        swap_cols(Yw, l, l, j, best);
        swap_cols(Y, l, l, j, best);
        swap_cols(A, lda, m, k0 + j, k0 + best);
        int t = perm[k0 + j]; perm[k0 + j] = perm[k0 + best]; perm[k0 + best] = t;
      }
      if (l - j >= 2) {
        double t, bt;
        orc_house(l - j, Yw + IX(j, j, l), 1, v, &t, &bt);
        apply_house_left(l - j, v, t, Yw, l, j, j + 1, np);
      }
    }
    /* Sec. 5.1: unpivoted Householder QR of the m' x b panel, then T. */
    double* P = A + IX(k0, k0, lda);
    orc_geqr2(mp, bi, P, lda, tau);
    double* Tb = T + IX(0, k0, ldt);
    orc_larft(mp, bi, P, lda, tau, Tb, ldt);
    /* Trailing update A(k0:m, k0+b:n) <- (I - V T V^T)^T A(k0:m, k0+b:n). */
    const int n2 = np - bi;
    double* A2 = A + IX(k0, k0 + bi, lda);
    orc_apply_block(mp, n2, bi, P, lda, Tb, ldt, 1, A2, lda);
    if (mode == ORC_SKETCH_DOWNDATE) {
      /* Gq = G - (G V) T V^T, all l x m' */
      double* GV = (double*)xcalloc((size_t)l * bi, sizeof(double));
      double* GVT = (double*)xcalloc((size_t)l * bi, sizeof(double));
#pragma omp parallel for schedule(static)
      for (int c = 0; c < bi; ++c)
        for (int i = 0; i < l; ++i) {
          double s = 0.0;
          for (int r = c; r < mp; ++r) s += Gc[IX(i, r, l)] * vget(P, lda, r, c);
          GV[IX(i, c, l)] = s;
        }
      for (int c = 0; c < bi; ++c)
        for (int i = 0; i < l; ++i) {
          double s = 0.0;
          for (int t = 0; t <= c; ++t) s += GV[IX(i, t, l)] * Tb[IX(t, c, ldt)];
          GVT[IX(i, c, l)] = s;
        }
#pragma omp parallel for schedule(static)
      for (int r = 0; r < mp; ++r) {
        int cmax = r < bi - 1 ? r : bi - 1;
        for (int i = 0; i < l; ++i) {
          double s = 0.0;
          for (int c = 0; c <= cmax; ++c) s += GVT[IX(i, c, l)] * vget(P, lda, r, c);
          Gc[IX(i, r, l)] -= s;
        }
      }
      /* Y <- Y(:, b:n') - Gq(:, 0:b) R12, with R12 = A(k0:k0+b, k0+b:n) */
      double* Yn = (double*)xcalloc((size_t)l * (n2 > 0 ? n2 : 1), sizeof(double));
#pragma omp parallel for schedule(static)
      for (int c = 0; c < n2; ++c)
        for (int i = 0; i < l; ++i) {
          double s = 0.0;
          for (int t = 0; t < bi; ++t) s += Gc[IX(i, t, l)] * A[IX(k0 + t, k0 + bi + c, lda)];
          Yn[IX(i, c, l)] = Y[IX(i, bi + c, l)] - s;
        }
      memcpy(Y, Yn, sizeof(double) * (size_t)l * n2);
      free(Yn);
      /* G <- Gq(:, b:m') */
      memmove(Gc, Gc + IX(0, bi, l), sizeof(double) * (size_t)l * (mp - bi));
      free(GV);
      free(GVT);
    }
    k0 += bi;
    ++blocks;
  }
  if (mode == ORC_SKETCH_DOWNDATE && k0 < n) {
    if (Yout) memcpy(Yout, Y, sizeof(double) * (size_t)l * (n - k0));
    if (Gout) memcpy(Gout, Gc, sizeof(double) * (size_t)l * (m - k0));
  }
  free(Y);
  free(Yw);
  free(Gc);
  free(tau);
  free(v);
  return k0;
}

/* ------------------------------------------------------- one-sided Jacobi */
int orc_jacobi_svd(int r, int c, double* M, int ldm, double* sv, double* J, int ldj) {
  for (int j = 0; j < c; ++j)
    for (int i = 0; i < c; ++i) J[IX(i, j, ldj)] = (i == j) ? 1.0 : 0.0;
  const double tol = 1e-15;
  int sweep = 0;
  for (sweep = 1; sweep <= 80; ++sweep) {
    int rotated = 0;
    for (int i = 0; i < c - 1; ++i)
      for (int j = i + 1; j < c; ++j) {
        double* x = M + IX(0, i, ldm);
        double* y = M + IX(0, j, ldm);
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int t = 0; t < r; ++t) { al += x[t] * x[t]; be += y[t] * y[t]; ga += x[t] * y[t]; }
        if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
        rotated = 1;
        double zeta = (be - al) / (2.0 * ga);
        double t = sgn0(zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int k = 0; k < r; ++k) {
          double xi = x[k], yi = y[k];
          x[k] = cs * xi - sn * yi;
          y[k] = sn * xi + cs * yi;
        }
        double* u = J + IX(0, i, ldj);
        double* w = J + IX(0, j, ldj);
        for (int k = 0; k < c; ++k) {
          double ui = u[k], wi = w[k];
          u[k] = cs * ui - sn * wi;
          w[k] = sn * ui + cs * wi;
        }
      }
    if (!rotated) break;
  }
  /* norms, then selection sort into descending order (columns of M and J) */
  for (int j = 0; j < c; ++j) {
    double s = 0.0;
    for (int t = 0; t < r; ++t) s += M[IX(t, j, ldm)] * M[IX(t, j, ldm)];
    sv[j] = sqrt(s);
  }
  for (int a = 0; a < c; ++a) {
    int bst = a;
    for (int j = a + 1; j < c; ++j)
      if (sv[j] > sv[bst]) bst = j;
    if (bst != a) {
      double t = sv[a]; sv[a] = sv[bst]; sv[bst] = t;
      swap_cols(M, ldm, r, a, bst);
      swap_cols(J, ldj, c, a, bst);
    }
  }
  return sweep;
}

/* Thin Q of the r x c matrix Z (Householder, Sec. 3.2): Q is r x min(r, c). */
static int thin_q(int r, int c, const double* Z, int ldz, double* Q, int ldq) {
  int kq = r < c ? r : c;
  double* F = (double*)xcalloc((size_t)r * c, sizeof(double));
  for (int j = 0; j < c; ++j)
    for (int i = 0; i < r; ++i) F[IX(i, j, r)] = Z[IX(i, j, ldz)];
  double* tau = (double*)xcalloc((size_t)c, sizeof(double));
  orc_geqr2(r, c, F, r, tau);
  for (int j = 0; j < kq; ++j)
    for (int i = 0; i < r; ++i) Q[IX(i, j, ldq)] = (i == j) ? 1.0 : 0.0;
  double* v = (double*)xcalloc((size_t)r, sizeof(double));
  for (int j = kq - 1; j >= 0; --j) {
    if (tau[j] == 0.0) continue;
    v[0] = 1.0;
    for (int i = 1; i < r - j; ++i) v[i] = F[IX(j + i, j, r)];
    apply_house_left(r - j, v, tau[j], Q, ldq, j, 0, kq);
  }
  free(v);
  free(tau);
  free(F);
  return kq;
}

/* Thin QR with explicit R (kq x c) next to Q. */
static int thin_qr(int r, int c, const double* Z, int ldz, double* Q, int ldq, double* R, int ldr) {
  int kq = thin_q(r, c, Z, ldz, Q, ldq);
  /* R = Q^T Z */
  matmul_tn(kq, c, r, Q, ldq, Z, ldz, R, ldr);
  return kq;
}

/* ------------------------------------------------ Sec. 4.2 + 4.3 reduction */
void orc_reduce_sketch(int r, int c, int b, const double* Z, int ldz, double* Zr, int ldzr) {
  int kk = r < c ? r : c;
  double* Qz = (double*)xcalloc((size_t)r * kk, sizeof(double));
  double* Rz = (double*)xcalloc((size_t)kk * c, sizeof(double));
  thin_qr(r, c, Z, ldz, Qz, r, Rz, kk);
  /* one-sided Jacobi on M = Rz^T (c x kk): J = left singular vectors of Rz */
  double* M = (double*)xcalloc((size_t)c * kk, sizeof(double));
  for (int j = 0; j < kk; ++j)
    for (int i = 0; i < c; ++i) M[IX(i, j, c)] = Rz[IX(j, i, kk)];
  double* sv = (double*)xcalloc((size_t)kk, sizeof(double));
  double* J = (double*)xcalloc((size_t)kk * kk, sizeof(double));
  orc_jacobi_svd(c, kk, M, c, sv, J, kk);
  /* Zr = Qz J(:, 0:b): the b dominant left singular vectors of Z */
  matmul_nn(r, b, kk, Qz, r, J, kk, Zr, ldzr);
  free(Qz);
  free(Rz);
  free(M);
  free(sv);
  free(J);
}

/* ------------------------------------------------ Sec. 6.2 completion */
/* Column c of the bi x bi matrix V (ld ldv), orthogonal to its orthonormal
 * columns 0..c-1, for a zero singular value: the first unit vector e_k that
 * Gram-Schmidt (twice) against those columns leaves with norm above 1/2, or,
 * if none does, the one left with the largest norm (at least (bi-c)/bi in
 * squared norm, summed over k), normalised. */
void orc_complete_column(int bi, int c, double* V, int ldv) {
  double* v = V + IX(0, c, ldv);
  int best = 0;
  double best_nv = -1.0;
  for (int pick = 0; pick < 2; ++pick) {
    for (int e = 0; e < bi; ++e) {
      if (pick == 1 && e != best) continue;
      for (int i = 0; i < bi; ++i) v[i] = (i == e) ? 1.0 : 0.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int t = 0; t < c; ++t) {
          const double* u = V + IX(0, t, ldv);
          double d = 0.0;
          for (int i = 0; i < bi; ++i) d += u[i] * v[i];
          for (int i = 0; i < bi; ++i) v[i] -= d * u[i];
        }
      double nv = 0.0;
      for (int i = 0; i < bi; ++i) nv += v[i] * v[i];
      nv = sqrt(nv);
      if (nv > 0.5 || pick == 1) {
        for (int i = 0; i < bi; ++i) v[i] /= nv;
        return;
      }
      if (nv > best_nv) {
        best_nv = nv;
        best = e;
      }
    }
  }
}

/* ------------------------------------------------ Sec. 4.2, 6.3, 6.4 */
/* Sec. 6.2 (Fig. blockRRQR): diagonalise the bi x bi diagonal block R11 of the
 * block that starts at k0, after its left QR and trailing update. The SVD is
 * R11 = U' D Vt^T: one-sided Jacobi on M = R11^T gives M J = Vt D with J = U'
 * (columns sorted by descending norm); the columns of Vt are those of M J over
 * their norms, and a zero column is completed by orc_complete_column. Then A(0:k0, block) <- A(0:k0, block) Vt, R12 <- U'^T R12, R11 <- D
 * (the strictly lower part of the block, the Householder vectors, is kept),
 * and U' and Vt go to DU(0:bi, k0:k0+bi) and DV(0:bi, k0:k0+bi). */
static void diag_block(int n, double* A, int lda, int k0, int bi, double* DU, int lddu, double* DV, int lddv) {
  double* M = (double*)xcalloc((size_t)bi * bi, sizeof(double));
  double* J = (double*)xcalloc((size_t)bi * bi, sizeof(double));
  double* sv = (double*)xcalloc((size_t)bi, sizeof(double));
  for (int j = 0; j < bi; ++j)
    for (int i = 0; i <= j; ++i) M[IX(j, i, bi)] = A[IX(k0 + i, k0 + j, lda)]; /* M = R11^T */
  orc_jacobi_svd(bi, bi, M, bi, sv, J, bi);
  double* Vt = DV + IX(0, k0, lddv);
  double* Up = DU + IX(0, k0, lddu);
  for (int j = 0; j < bi; ++j)
    for (int i = 0; i < bi; ++i) Up[IX(i, j, lddu)] = J[IX(i, j, bi)];
  for (int c = 0; c < bi; ++c) {
    if (sv[c] > 0.0) {
      for (int i = 0; i < bi; ++i) Vt[IX(i, c, lddv)] = M[IX(i, c, bi)] / sv[c];
      continue;
    }
    orc_complete_column(bi, c, Vt, lddv);
  }
  /* A(0:k0, block) <- A(0:k0, block) Vt */
  double* row = (double*)xcalloc((size_t)bi, sizeof(double));
  for (int r = 0; r < k0; ++r) {
    for (int j = 0; j < bi; ++j) {
      double acc = 0.0;
      for (int t = 0; t < bi; ++t) acc += A[IX(r, k0 + t, lda)] * Vt[IX(t, j, lddv)];
      row[j] = acc;
    }
    for (int j = 0; j < bi; ++j) A[IX(r, k0 + j, lda)] = row[j];
  }
  /* R12 <- U'^T R12 (columns k0+bi..n-1) */
  for (int col = k0 + bi; col < n; ++col) {
    for (int i = 0; i < bi; ++i) {
      double acc = 0.0;
      for (int t = 0; t < bi; ++t) acc += Up[IX(t, i, lddu)] * A[IX(k0 + t, col, lda)];
      row[i] = acc;
    }
    for (int i = 0; i < bi; ++i) A[IX(k0 + i, col, lda)] = row[i];
  }
  /* R11 <- D */
  for (int j = 0; j < bi; ++j)
    for (int i = 0; i <= j; ++i) A[IX(k0 + i, k0 + j, lda)] = (i == j) ? sv[j] : 0.0;
  free(row);
  free(M);
  free(J);
  free(sv);
}

int orc_rurv(int m, int n, double* A, int lda, int b, int p, int q, int k, const double* G, double* TU, int ldtu,
             double* WV, int ldwv, double* TV, int ldtv) {
  return orc_rurv_diag(m, n, A, lda, b, p, q, k, G, TU, ldtu, WV, ldwv, TV, ldtv, NULL, 0, NULL, 0);
}

int orc_rurv_diag(int m, int n, double* A, int lda, int b, int p, int q, int k, const double* G, double* TU,
                  int ldtu, double* WV, int ldwv, double* TV, int ldtv, double* DU, int lddu, double* DV, int lddv) {
  const int l = b + p;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < b; ++i) { TU[IX(i, j, ldtu)] = 0.0; TV[IX(i, j, ldtv)] = 0.0; }
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) WV[IX(i, j, ldwv)] = 0.0;
  size_t goff = 0;
  int k0 = 0;
  while (k0 < n) {
    const int np = n - k0, mp = m - k0;
    const int bi = np < b ? np : b;
    double* X = A + IX(k0, k0, lda);
    /* Z = (G_i X)^T, n' x l */
    double* Ysk = (double*)xcalloc((size_t)l * np, sizeof(double));
    matmul_nn(l, np, mp, G + goff, l, X, lda, Ysk, l);
    goff += (size_t)l * mp;
    int zc = l;
    double* Z = (double*)xcalloc((size_t)np * l, sizeof(double));
    for (int c = 0; c < l; ++c)
      for (int i = 0; i < np; ++i) Z[IX(i, c, np)] = Ysk[IX(c, i, l)];
    free(Ysk);
    /* Sec. 6.3 power steps with orthonormalisation between products */
    for (int t = 0; t < q; ++t) {
      double* Qz = (double*)xcalloc((size_t)np * zc, sizeof(double));
      int kz = thin_q(np, zc, Z, np, Qz, np);
      double* XW = (double*)xcalloc((size_t)mp * kz, sizeof(double));
      matmul_nn(mp, kz, np, X, lda, Qz, np, XW, mp);
      double* Qw = (double*)xcalloc((size_t)mp * kz, sizeof(double));
      int kw = thin_q(mp, kz, XW, mp, Qw, mp);
      /* Z = X^T Qw, n' x kw */
      matmul_tn(np, kw, mp, X, lda, Qw, mp, Z, np);
      zc = kw;
      free(Qz);
      free(XW);
      free(Qw);
    }
    /* l -> b_i reduction through the SVD of R_z */
    double* Zb = Z;
    double* Zr = NULL;
    if (zc > bi) {
      Zr = (double*)xcalloc((size_t)np * bi, sizeof(double));
      orc_reduce_sketch(np, zc, bi, Z, np, Zr, np);
      Zb = Zr;
    }
    /* Householder QR of Z (n' x b_i) gives S = I - W TS W^T (Sec. 4.2) */
    double* taus = (double*)xcalloc((size_t)bi, sizeof(double));
    orc_geqr2(np, bi, Zb, np, taus);
    for (int j = 0; j < bi; ++j)
      for (int i = j + 1; i < np; ++i) WV[IX(k0 + i, k0 + j, ldwv)] = Zb[IX(i, j, np)];
    double* TS = TV + IX(0, k0, ldtv);
    orc_larft(np, bi, WV + IX(k0, k0, ldwv), ldwv, taus, TS, ldtv);
    /* A(0:m, k0:n) <- A(0:m, k0:n) S: rows are independent; row x -> x - ((x W) TS) W^T */
    {
      const double* Wm = WV + IX(k0, k0, ldwv);
#pragma omp parallel
      {
        double* xw = (double*)xcalloc((size_t)bi, sizeof(double));
        double* xwt = (double*)xcalloc((size_t)bi, sizeof(double));
#pragma omp for schedule(static)
        for (int r = 0; r < m; ++r) {
          for (int j = 0; j < bi; ++j) {
            double s = 0.0;
            for (int i = j; i < np; ++i) s += A[IX(r, k0 + i, lda)] * vget(Wm, ldwv, i, j);
            xw[j] = s;
          }
          for (int j = 0; j < bi; ++j) {
            double s = 0.0;
            for (int t = 0; t <= j; ++t) s += xw[t] * TS[IX(t, j, ldtv)];
            xwt[j] = s;
          }
          for (int i = 0; i < np; ++i) {
            int jmax = i < bi - 1 ? i : bi - 1;
            double s = 0.0;
            for (int j = 0; j <= jmax; ++j) s += xwt[j] * vget(Wm, ldwv, i, j);
            A[IX(r, k0 + i, lda)] -= s;
          }
        }
        free(xw);
        free(xwt);
      }
    }
    /* panel QR + T + trailing update (Fig. blockQR) */
    double* tau = (double*)xcalloc((size_t)bi, sizeof(double));
    orc_geqr2(mp, bi, X, lda, tau);
    double* Tb = TU + IX(0, k0, ldtu);
    orc_larft(mp, bi, X, lda, tau, Tb, ldtu);
    if (np > bi) orc_apply_block(mp, np - bi, bi, X, lda, Tb, ldtu, 1, A + IX(k0, k0 + bi, lda), lda);
    if (DU && DV) diag_block(n, A, lda, k0, bi, DU, lddu, DV, lddv);
    free(tau);
    free(taus);
    free(Z);
    free(Zr);
    k0 += bi;
    if (k > 0 && k0 >= k) break;
  }
  return k0;
}

/* ------------------------------------------------- Philox4x32-10 (SC'11) */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c0, p1 = (uint64_t)M1 * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    if (r < 9) { k0 += W0; k1 += W1; }
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Element e of stream (seed, stream): block e/4 of Philox with counter
 * {e/4 low, e/4 high, stream low, stream high} and key {seed low, seed high};
 * uniforms u = (x + 0.5) 2^-32; pairs (out0,out1) and (out2,out3) go through
 * Box-Muller r = sqrt(-2 ln u1), z = (r cos 2 pi u2, r sin 2 pi u2). */
void orc_gauss_fill(uint64_t seed, uint64_t stream, int64_t count, double* out) {
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(static)
  for (int64_t blk = 0; blk < (count + 3) / 4; ++blk) {
    uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)((uint64_t)blk >> 32), (uint32_t)stream, (uint32_t)(stream >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    double z[4];
    for (int h = 0; h < 2; ++h) {
      double u1 = ((double)x[2 * h] + 0.5) * 2.3283064365386963e-10;
      double u2 = ((double)x[2 * h + 1] + 0.5) * 2.3283064365386963e-10;
      double r = sqrt(-2.0 * log(u1));
      z[2 * h] = r * cos(two_pi * u2);
      z[2 * h + 1] = r * sin(two_pi * u2);
    }
    for (int t = 0; t < 4; ++t)
      if (4 * blk + t < count) out[4 * blk + t] = z[t];
  }
}
