// adjoint.cu -- reverse-mode derivative of the (truncated) QR factorization
// X = A P = Q R with the column transformation P held fixed (the pivots of
// randomized QRCP, or the orthonormal P of the URV method), for the
// differentiable form of the library. Not in the paper.
//
// With X = [X1 X2] (k and n - k columns), X1 = Q1 R11 (thin QR, Q1 m x k) and
// R12 = Q1^T X2, the outputs are Q1 and R1 = [R11 R12]. Given the cotangents
// Q1b (m x k) and R1b = [R11b R12b] (k x n):
//   X2b  = Q1 R12b
//   Q1b' = Q1b + X2 R12b^T
//   M    = R11 R11b^T - Q1b'^T Q1          (k x k)
//   X1b  = (Q1b' + Q1 copyltu(M)) R11^-T   copyltu(M) = tril(M) + tril(M, -1)^T
// (the thin-QR adjoint of Walter and Lehmann 2018, Liao et al. 2019, applied
// to the leading block, and the product rule for R12). The result is the
// cotangent of X = A P; with a permutation P it is scattered back to A's
// columns (Ab(:, perm[j]) = Xb(:, j)).
#include <algorithm>

#include "common.cuh"

namespace rqr {

namespace {

// M <- tril(M) + tril(M, -1)^T for a k x k matrix (ld ldm).
__global__ void k_copyltu(int k, double* M, int ldm) {
  const int64_t nn = (int64_t)k * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    if (i < j) M[i + (size_t)j * ldm] = M[j + (size_t)i * ldm];
  }
}

// Rows of X (m x nb, ld ldx) <- X R^-T for the nb x nb upper-triangular
// diagonal block R (ld ldr): row x solves R x^T = x_old^T by back
// substitution, one thread per row, R in shared memory. A zero diagonal
// entry (rank-deficient R11) sets the status word and leaves the row.
constexpr int kTrsmNb = 64;
__global__ void __launch_bounds__(256) k_trsm_diag(int m, int nb, const double* __restrict__ R, int ldr, double* X,
                                                   int ldx, int* status) {
  __shared__ double Rs[kTrsmNb][kTrsmNb + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, j = e / nb;
    Rs[i][j] = i <= j ? R[i + (size_t)j * ldr] : 0.0;
  }
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double x[kTrsmNb];
#pragma unroll
  for (int j = 0; j < kTrsmNb; ++j) x[j] = j < nb ? X[r + (size_t)j * ldx] : 0.0;
  bool bad = false;
#pragma unroll
  for (int i = kTrsmNb - 1; i >= 0; --i) {
    if (i >= nb) continue;
    double s = x[i];
#pragma unroll
    for (int j = i + 1; j < kTrsmNb; ++j)
      if (j < nb) s -= Rs[i][j] * x[j];
    if (Rs[i][i] == 0.0) bad = true;
    x[i] = Rs[i][i] != 0.0 ? s / Rs[i][i] : 0.0;
  }
  if (bad) atomicCAS(status, 0, RQR_ERR_NONFINITE);
#pragma unroll
  for (int j = 0; j < kTrsmNb; ++j)
    if (j < nb) X[r + (size_t)j * ldx] = x[j];
}

// Ab(:, perm[j]) = Xb(:, j).
__global__ void k_scatter_cols(int m, int n, const double* __restrict__ Xb, int ldx, const int32_t* __restrict__ perm,
                               double* Ab, int lda) {
  const int64_t nn = (int64_t)m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    Ab[i + (size_t)perm[j] * lda] = Xb[i + (size_t)j * ldx];
  }
}

// X2(:, j) = A(:, perm[k + j]), j < n - k.
__global__ void k_gather_cols(int m, int nk, const double* __restrict__ A, int lda, const int32_t* __restrict__ perm,
                              double* X2, int ldx) {
  const int64_t nn = (int64_t)m * nk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % m), j = (int)(e / m);
    X2[i + (size_t)j * ldx] = A[i + (size_t)perm[j] * lda];
  }
}

// Upper triangle of the first k rows of F into R (k x n), zeros below.
__global__ void k_copy_upper(int k, int n, const double* __restrict__ F, int ldf, double* R, int ldr) {
  const int64_t nn = (int64_t)k * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % k), j = (int)(e / k);
    R[i + (size_t)j * ldr] = i <= j ? F[i + (size_t)j * ldf] : 0.0;
  }
}

int grid_for(int64_t n, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sms * 8));
}

}  // namespace

size_t qr_adjoint_work_elems(int m, int n, int k, int sms) {
  // M, R11, R11b (k x k each), Q1b' (m x k), Xb (m x n), gathered X2
  // (m x (n - k)), split-K partials
  return 3 * (size_t)k * k + (size_t)m * k + (size_t)m * n + (size_t)m * (n - k) + (size_t)8 * sms * 64 * 64;
}

void copy_upper(const Ctx& c, int k, int n, const double* F, int ldf, double* R, int ldr) {
  if (k <= 0 || n <= 0) return;
  k_copy_upper<<<grid_for((int64_t)k * n, c.sms), 256, 0, c.stream>>>(k, n, F, ldf, R, ldr);
  note_launch(c);
}

// X <- X R^-T for the k x k upper-triangular R: blocks of 64 columns from the
// last, each first updated by the solved blocks to its right (one product on
// the FP64 pipe), then solved against its diagonal block.
void trsm_right_upper_t(const Ctx& c, int m, int k, const double* R, int ldr, double* X, int ldx, double* part,
                        size_t cap) {
  if (m <= 0 || k <= 0) return;
  const int nblk = ceil_div(k, kTrsmNb);
  for (int J = nblk - 1; J >= 0; --J) {
    const int j0 = J * kTrsmNb, jb = std::min(kTrsmNb, k - j0), je = j0 + jb;
    if (je < k)  // X_J -= X(:, je:k) R(j0:je, je:k)^T
      gemm<double>(c, false, true, m, jb, k - je, -1.0, X + (size_t)je * ldx, ldx, R + j0 + (size_t)je * ldr, ldr,
                   1.0, X + (size_t)j0 * ldx, ldx, part, cap);
    k_trsm_diag<<<ceil_div(m, 256), 256, 0, c.stream>>>(m, jb, R + j0 + (size_t)j0 * ldr, ldr,
                                                        X + (size_t)j0 * ldx, ldx, c.status);
    note_launch(c);
  }
}

// The adjoint described at the top of the file. F holds R1 in the upper
// triangle of its first k rows (ld ldf); Q1 is m x k; Rb is k x n (only the
// upper triangle of its leading k x k block is used: R11's structural zeros
// carry no cotangent). With perm, P is that permutation: X2 is gathered from A
// (needed when k < n) and the result is scattered to A's columns; without
// perm, X2 = A P(:, k:) is given and the result is the cotangent of X = A P.
// work: qr_adjoint_work_elems doubles.
int qr_adjoint(const Ctx& c, int m, int n, int k, const double* Q1, int ldq, const double* F, int ldf, const double* A,
               int lda, const int32_t* perm, const double* X2, int ldx2, const double* Qb, int ldqb, const double* Rb,
               int ldrb, double* Ab, int ldab, double* work) {
  double* M = work;
  double* R11 = M + (size_t)k * k;    // explicit upper-triangular copy of R11
  double* R11b = R11 + (size_t)k * k;  // upper triangle of the leading block of Rb
  double* Qb2 = R11b + (size_t)k * k;
  double* Xb = Qb2 + (size_t)m * k;
  double* X2g = Xb + (size_t)m * n;
  double* part = X2g + (size_t)m * (n - k);
  const size_t cap = (size_t)8 * c.sms * 64 * 64;
  if (perm && k < n) {
    k_gather_cols<<<grid_for((int64_t)m * (n - k), c.sms), 256, 0, c.stream>>>(m, n - k, A, lda, perm + k, X2g, m);
    note_launch(c);
    X2 = X2g;
    ldx2 = m;
  }
  // X written directly into Ab when no permutation is applied
  double* X = perm ? Xb : Ab;
  const int ldxx = perm ? m : ldab;
  copy_mat<double>(c, m, k, Qb, ldqb, Qb2, m);
  if (k < n) {
    // X2b = Q1 R12b; Q1b' += X2 R12b^T
    gemm<double>(c, false, false, m, n - k, k, 1.0, Q1, ldq, Rb + (size_t)k * ldrb, ldrb, 0.0, X + (size_t)k * ldxx,
                 ldxx, part, cap);
    gemm<double>(c, false, true, m, k, n - k, 1.0, X2, ldx2, Rb + (size_t)k * ldrb, ldrb, 1.0, Qb2, m, part, cap);
  }
  // M = R11 R11b^T - Q1b'^T Q1 (F holds Householder vectors below R11's
  // diagonal, so R11 is copied out with zeros below)
  copy_upper(c, k, k, F, ldf, R11, k);
  copy_upper(c, k, k, Rb, ldrb, R11b, k);
  gemm<double>(c, false, true, k, k, k, 1.0, R11, k, R11b, k, 0.0, M, k, part, cap);
  gemm<double>(c, true, false, k, k, m, -1.0, Qb2, m, Q1, ldq, 1.0, M, k, part, cap);
  k_copyltu<<<grid_for((int64_t)k * k, c.sms), 256, 0, c.stream>>>(k, M, k);
  note_launch(c);
  // X1b = (Q1b' + Q1 copyltu(M)) R11^-T
  copy_mat<double>(c, m, k, Qb2, m, X, ldxx);
  gemm<double>(c, false, false, m, k, k, 1.0, Q1, ldq, M, k, 1.0, X, ldxx, part, cap);
  trsm_right_upper_t(c, m, k, R11, k, X, ldxx, part, cap);
  if (perm) {
    k_scatter_cols<<<grid_for((int64_t)m * n, c.sms), 256, 0, c.stream>>>(m, n, Xb, m, perm, Ab, ldab);
    note_launch(c);
  }
  return RQR_OK;
}

}  // namespace rqr
