/*
 * oracle.h -- plain, slow FP64 CPU oracle for randomized blocked QR with column
 * pivoting (Martinsson, "Blocked rank-revealing QR factorizations: how
 * randomized sampling can be used to avoid single-vector pivoting", 2015).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or load
 * this code; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg use it. It shares no source with the CUDA library.
 *
 * Conventions: every matrix is column-major double with a leading dimension;
 * indices are 0-based; permutations are stored as perm[k] = original column
 * that sits at position k of A*P. Householder vectors are stored LAPACK-style
 * below the diagonal with an implicit unit first entry; Q = I - V T V^T per
 * block with T upper triangular (forward, column-wise accumulation).
 *
 * Functions whose correctness is pinned only by invariants or statistical
 * claims, not by a closed form or an independent algorithm, say so in the
 * comment beside them ("parity unpinned").
 */
#ifndef RQR_ORACLE_H
#define RQR_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* Sec. 3.1: Householder reflector H(a) of a k-vector a (stride inca).
 * beta = -sign(a[0])*||a|| with sign(0) = +1; v[0] = 1, v = (a - beta e1)/(a[0]-beta);
 * tau = (beta - a[0])/beta so that H = I - tau v v^T equals I - 2 vhat vhat^T.
 * ||a|| = 0 gives tau = 0, beta = 0, v = e1 (H = I). */
void orc_house(int k, const double* a, int inca, double* v, double* tau, double* beta);

/* Sec. 3.3, Fig. "QR" (basicQR): classical Householder QR with column pivoting of
 * the m x n matrix A (m >= n). Pivot = largest remaining column by FP64 sum of
 * squares, recomputed exactly at every step; ties go to the lowest position.
 * Steps j = 0 .. min(n, m-1)-1 (n-1 steps when m = n). On exit R is in the upper
 * triangle, reflectors below it, tau[n] (0 where no reflector), perm[n]. */
void orc_qrcp(int m, int n, double* A, int lda, int* perm, double* tau);

/* Sec. 3.2: unpivoted Householder QR of the m x n matrix A, same storage. */
void orc_geqr2(int m, int n, double* A, int lda, double* tau);

/* Sec. 5.1 (compact WY remark): k x k upper-triangular T with
 * H_0 H_1 ... H_{k-1} = I - V T V^T, V = m x k unit lower trapezoidal (the
 * strictly lower part of V is read, its diagonal is taken as 1). */
void orc_larft(int m, int k, const double* V, int ldv, const double* tau, double* T, int ldt);

/* Applies the block reflector Q~ = I - V T V^T (m x k, T k x k) or its transpose
 * to the m x n matrix C from the left: C <- Q~ C (trans=0) or Q~^T C (trans=1). */
void orc_apply_block(int m, int n, int k, const double* V, int ldv, const double* T, int ldt,
                     int trans, double* C, int ldc);

/* Sketch modes of orc_rqrcp. */
#define ORC_SKETCH_DOWNDATE 0
#define ORC_SKETCH_RESAMPLE 1

/* Sec. 4.1 + 4.3 + 5.1 + 5.2 (Method 1 with over-sampling p): randomized blocked
 * QR with column pivoting, A P = Q R, m >= n, block size b, l = b + p.
 *   DOWNDATE: G is l x m (ldg >= l), drawn once; Y = G A; after every block
 *     Gq = G (I - V T V^T), Y <- Y(:, b:) - Gq(:, :b) R12, G <- Gq(:, b:)
 *     (the sketch update is not in the paper; it keeps Y = G X'' exactly).
 *   RESAMPLE: the paper's literal re-sketch Y = G_i A(k0:m, k0:n) per block;
 *     G holds the blocks G_i (l x m_i, m_i = m - k0) one after another with
 *     leading dimension l (ldg ignored).
 * Per block: the first b_i steps of Fig. "QR" on a copy of Y pick the pivots
 * (swaps mirrored on Y, on all m rows of A and on perm); unpivoted Householder
 * QR of the panel; T by orc_larft; A22 <- (I - V T V^T)^T A22. The last block
 * (n - k0 <= b) is finished with Fig. "QR" (Fig. blockQR, final step).
 * T is b x n (ldt >= b): block starting at column k0 stores its T at
 * T(0:b_i, k0:k0+b_i). max_blocks > 0 stops after that many blocks (the final
 * classical step counts as a block). Returns the number of columns finished. */
int orc_rqrcp(int m, int n, double* A, int lda, int b, int p, const double* G, int ldg, int mode,
              double* T, int ldt, int* perm, int max_blocks);

/* orc_rqrcp that also returns, when it stops early in DOWNDATE mode, the
 * carried sketch Y (l x (n-k0), ld l) and Gaussian G (l x (m-k0), ld l), so a
 * test can check the invariant Y = G A(k0:m, k0:n). NULL skips either. */
int orc_rqrcp_ex(int m, int n, double* A, int lda, int b, int p, const double* G, int ldg, int mode,
                 double* T, int ldt, int* perm, int max_blocks, double* Yout, double* Gout);

/* Sec. 4.2 + 6.3 + 6.4 (Methods 2/3 without the diagonalisation step): blocked
 * QR with orthonormal pivoting A P = Q R, P = S_0 S_1 ... with each
 * S_i = I - W_i TS_i W_i^T acting on columns k0..n.
 * Per block with X = A(k0:m, k0:n) (m' x n'), G_i (l x m', stored as in the
 * RESAMPLE layout above):
 *   Z = (G_i X)^T; q times { Z <- orth(Z); W <- orth(X Z); Z <- X^T W };
 *   if Z has more than b_i columns: Z = Qz Rz, Rz = Ur S Vr^T (one-sided Jacobi),
 *   Z <- Qz Ur(:, 0:b_i); Householder QR of Z gives (W_i, TS_i);
 *   A(0:m, k0:n) <- A(0:m, k0:n) S_i; then panel QR + trailing update as blockQR.
 * Outputs: R/V in A, TU (b x n) for the left reflectors, WV (n x n, ldwv >= n;
 * block i stores W_i below the diagonal of WV(k0:n, k0:k0+b_i)), TV (b x n).
 * k > 0 stops once k0 >= k (truncated rank-k factorization).
 * Returns the number of columns finished. Parity unpinned beyond the invariants
 * and bounds listed in the test suite (the method is randomized). */
int orc_rurv(int m, int n, double* A, int lda, int b, int p, int q, int k, const double* G,
             double* TU, int ldtu, double* WV, int ldwv, double* TV, int ldtv);

/* orc_rurv with the diagonal blocks diagonalised (Sec. 6.2, Fig. blockRRQR,
 * Method 3): after the left QR and trailing update of each block,
 * R11 = U' D Vt^T (one-sided Jacobi), A(0:k0, block) <- A(0:k0, block) Vt,
 * R12 <- U'^T R12, R11 <- D. U' and Vt (b_i x b_i) are stored at
 * DU(0:b_i, k0:k0+b_i) and DV(0:b_i, k0:k0+b_i) (b x n each). Then
 * A P = Q R with Q = prod_i H_i diag(I_k0, U'_i, I), P = prod_i S_i diag(I_k0, Vt_i, I).
 * DU = DV = NULL is orc_rurv. */
int orc_rurv_diag(int m, int n, double* A, int lda, int b, int p, int q, int k, const double* G,
                  double* TU, int ldtu, double* WV, int ldwv, double* TV, int ldtv, double* DU, int lddu,
                  double* DV, int lddv);

/* The l -> b reduction of the orthonormal pivot (Sec. 4.2 with the
 * over-sampling of Sec. 4.3), the step orc_rurv applies to its r x c sketch
 * Z when c > b: thin Householder QR Z = Qz Rz, one-sided Jacobi SVD of
 * Rz^T (whose right singular vectors are the left ones of Rz, sorted by
 * descending singular value), Zr (r x b, ld ldzr) = Qz Ur(:, 0:b). So Zr is an
 * orthonormal basis of the b dominant left singular vectors of Z (b <= min(r, c)).
 * Pinned against the projector of numpy's SVD of Z. */
void orc_reduce_sketch(int r, int c, int b, const double* Z, int ldz, double* Zr, int ldzr);

/* One-sided Jacobi SVD (Hestenes 1958) of the r x c matrix M (overwritten by
 * M*J): on exit sv[c] holds the column norms of M*J sorted descending and J
 * (c x c, ldj) the matching right singular vectors. Returns the sweep count. */
int orc_jacobi_svd(int r, int c, double* M, int ldm, double* sv, double* J, int ldj);
/* Sec. 6.2: column c of V (bi x bi, ld ldv) for a zero singular value, from
 * the orthonormal columns 0..c-1 (the first unit vector Gram-Schmidt leaves
 * with norm above 1/2, else the one left with the largest norm). */
void orc_complete_column(int bi, int c, double* V, int ldv);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): one block. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Standard normals from Philox4x32-10 + Box-Muller: element e (0-based) of the
 * stream (seed, stream) is lane e%4 of the block with counter
 * {lo(e/4), hi(e/4), lo(stream), hi(stream)} and key {lo(seed), hi(seed)};
 * lanes (0,1) and (2,3) are Box-Muller pairs of u = (x + 0.5) 2^-32. */
void orc_gauss_fill(uint64_t seed, uint64_t stream, int64_t count, double* out);

#ifdef __cplusplus
}
#endif
#endif
