/*
 * rqr.h -- C ABI of the GB300 (sm_103a) library for randomized blocked QR
 * factorizations (Martinsson, "Blocked rank-revealing QR factorizations: how
 * randomized sampling can be used to avoid single-vector pivoting", 2015).
 *
 * Storage conventions for every entry point:
 *  - Matrices are column-major with an explicit leading dimension (ld >= rows).
 *    Element (i, j) of A sits at A[i + j*lda]; indices are 0-based.
 *  - Pointers marked (device) must point to memory of the GPU that is current
 *    when the handle was created; (host) pointers are ordinary host memory.
 *  - The caller owns every buffer. A factor call allocates nothing: scratch
 *    comes from the caller's workspace (size from rqr_workspace_bytes).
 *  - Householder vectors are stored below the diagonal of the factored matrix
 *    with an implicit unit first entry; the orthonormal factor of one block is
 *    Q_i = I - V_i T_i V_i^T with T_i upper triangular (compact WY, Sec. 5.1).
 *  - perm[k] is the original column that ends up at position k of A*P.
 *  - All work is queued on the handle's stream. When `info` is non-NULL the
 *    call waits for the stream and writes the device status word to *info
 *    (0 = ok); with info == NULL the call returns as soon as the work is queued.
 *
 * Return values: 0 on success; -i when argument i (1-based, as listed) is
 * invalid (LAPACK convention; nothing is queued); a positive RQR_ERR_* code on
 * a runtime failure. No C++ exception crosses this interface.
 */
#ifndef RQR_H
#define RQR_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rqr_handle_s* rqr_handle_t;

/* Arithmetic of the factorization (the `prec` argument).
 * FP64: every step in FP64 on the FP64 pipe (A, G, T are double).
 * FP32: A, G, T are float; the large products run on the tensor cores as
 *   3xTF32 (FP32-level accuracy, FP32 accumulation), the rest in FP32.
 * TF32, 3XBF16, 3XTF32 (mixed precision): A, G, T are double; the panel
 *   Householder QR, its Gram matrix V^T V and T, the pivot steps on the
 *   sketch and the small products stay in FP64, so Q = prod(I - V T V^T) is
 *   orthogonal to FP64 rounding; the large products (sketch, trailing update,
 *   sketch downdate; for the URV method also the power steps and the right
 *   apply) run on the tcgen05 tensor cores with FP32 accumulation and
 *   operands rounded to one TF32 value (TF32), to a bf16 hi + lo pair with
 *   the products hi*hi + hi*lo + lo*hi (3XBF16, about 16 bits), or to a TF32
 *   big + small pair with big*big + big*small + small*big (3XTF32, about FP32
 *   accuracy). The residual ||AP - QR||/||A|| then follows the product
 *   precision (of order 1e-3, 1e-5, 1e-6 at n = 16384).
 * FP64X: FP64 data and FP64 panel/pivot/T steps; the large products
 *   (sketch, trailing update, downdate, Gram) are FP64-accurate splittings
 *   onto the bf16 tensor cores (Ozaki scheme): FP64-level residual. */
#define RQR_FP64 0
#define RQR_FP32 1
#define RQR_TF32 2
#define RQR_3XBF16 3
#define RQR_3XTF32 4
#define RQR_FP64X 5

/* How the sketch follows the factorization from block to block (`sketch`). */
#define RQR_SKETCH_DOWNDATE 0 /* draw G once, update Y = G X after each block */
#define RQR_SKETCH_RESAMPLE 1 /* draw a fresh G_i for every block (Fig. blockQR) */

/* Runtime status codes (positive return values / *info). */
#define RQR_OK 0
#define RQR_ERR_CUDA 1        /* a CUDA call failed, or a kernel found an
                                 internal index out of range and skipped the
                                 work; the handle stays usable                 */
#define RQR_ERR_NONFINITE 2   /* a NaN/Inf reached a panel norm               */
#define RQR_ERR_TIMEOUT 3     /* a bounded wait inside a kernel ran out (see
                                 rqr_set_wait_limit_ns)                         */
#define RQR_ERR_WORKSPACE 4   /* lwork smaller than rqr_workspace_bytes        */
#define RQR_ERR_UNSUPPORTED 5 /* a combination this build does not implement  */
#define RQR_ERR_HANDLE 6      /* NULL or destroyed handle                      */
#define RQR_ERR_SIZE 7        /* problem larger than a fixed internal buffer   */

/* Creates a handle bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = legacy default stream). (host) h receives the handle.
 * The handle owns only a few bytes of device memory for its status word. */
int rqr_create(rqr_handle_t* h, void* stream);

/* Destroys the handle after waiting for its stream. */
int rqr_destroy(rqr_handle_t h);

/* Rebinds the handle to another stream (cudaStream_t). */
int rqr_set_stream(rqr_handle_t h, void* stream);

/* Limit, in nanoseconds of GPU global time, of every wait of the cooperative
 * pivot and panel kernels for a value another CTA publishes (the steps that
 * exchange values between all CTAs once per column, as flagged words). A wait that runs out makes the call finish with
 * RQR_ERR_TIMEOUT in *info: every later kernel of the call sees the status
 * word and does no swap, panel or pivot work on values of the aborted step
 * (the output is then undefined, but every access stays inside the caller's
 * buffers). ns = 0 restores the default of 2 s. The tensor-core product
 * kernel keeps its own fixed 2 s limit on its pipeline waits. Returns -1 for
 * an invalid handle. No counterpart in the paper: it bounds device waits. */
int rqr_set_wait_limit_ns(rqr_handle_t h, uint64_t ns);

/* Bytes of device workspace that rqrcp_factor (q < 0) or rurv_factor (q >= 0)
 * needs for the given shape, block size b, over-sampling p and precision.
 * (host) bytes receives the size. */
int rqr_workspace_bytes(int m, int n, int b, int p, int q, int prec, int sketch, size_t* bytes);

/* Randomized blocked QR with column pivoting, A P = Q R (Sec. 4.1, 4.3, 5.1, 5.2;
 * Method 1 of Sec. 7 with over-sampling p).
 *   m, n     rows and columns, m >= n >= 0.
 *   A        (device, in/out) m x n, ld lda. On exit R is in the upper triangle
 *            and the Householder vectors of every block below the diagonal.
 *   b        block size, 1 <= b <= 512; p >= 0 over-sampling, b + p <= 1024; the
 *            sketch has l = b + p rows.
 *   seed     Philox4x32-10 key for the Gaussian sketch when G == NULL.
 *   G        (device, optional) the Gaussian: DOWNDATE: l x m, ld ldg.
 *            RESAMPLE: the blocks G_i (l x (m - k0)), ld l, one after another,
 *            for every block that is not the last. NULL: drawn from `seed`
 *            (stream = block index for RESAMPLE, 0 for DOWNDATE).
 *   T        (device, out) b x n, ld ldt >= b: the block starting at column k0
 *            stores its upper-triangular T at T(0:b_i, k0:k0+b_i).
 *   perm     (device, out) n int32.
 *   prec     RQR_FP64, RQR_FP64X (FP64 data, tensor-core products) or RQR_FP32
 *            (then A, G, T are float).
 *   sketch   RQR_SKETCH_DOWNDATE or RQR_SKETCH_RESAMPLE.
 *   work     (device) workspace of lwork bytes, 256-byte aligned.
 *   info     (host, optional) see the header comment.
 * The last block (n - k0 <= b) is finished by classical pivoted QR (Fig. QR). */
int rqrcp_factor(rqr_handle_t h, int m, int n, void* A, int lda, int b, int p, uint64_t seed,
                 const void* G, int ldg, void* T, int ldt, int32_t* perm, int prec, int sketch,
                 void* work, size_t lwork, int* info);

/* Blocked QR with orthonormal pivoting A P = Q R, P = S_0 S_1 ... (Sec. 4.2,
 * 6.3, 6.4; Method 2 of Sec. 7, and with the power scheme and DU, DV given,
 * Method 3 / Fig. blockRRQR with diagonalised diagonal blocks, Sec. 6.2).
 *   A        (device, in/out) m x n, ld lda: R above, left reflectors below.
 *   b, p, q  block size 1 <= b <= 512, over-sampling p >= 0 (l = b + p <= 1024),
 *            power steps 0 <= q <= 64.
 *   k        stop once k0 >= k (truncated rank-k URV); k <= 0 or k >= n: full.
 *   seed, G  Gaussian blocks G_i (l x (m - k0), ld l, one after another,
 *            one per block including the last), or NULL to draw from seed.
 *   TU       (device, out) b x n, ld ldtu: T of the left reflectors per block.
 *   WV       (device, out) n x n, ld ldwv: block i keeps the Householder vectors
 *            of S_i below the diagonal of WV(k0:n, k0:k0+b_i).
 *   TV       (device, out) b x n, ld ldtv: T of S_i per block.
 *   DU, DV   (device, out, optional: both or neither) b x n, ld lddu / lddv >= b.
 *            Given, each diagonal block is diagonalised after its left QR and
 *            trailing update: R11 = U' D Vt^T (one-sided Jacobi), A(0:k0, block)
 *            <- A(0:k0, block) Vt, R12 <- U'^T R12, R11 <- D (descending); U' is
 *            stored at DU(0:b_i, k0:k0+b_i), Vt at DV(0:b_i, k0:k0+b_i). Then
 *            Q = Q_house blockdiag(U'_i) and P = S_0 S_1 ... blockdiag(Vt_i).
 *            A zero singular value gets the column of Vt that completes the
 *            others to an orthonormal basis (Gram-Schmidt of a unit vector).
 *   prec     RQR_FP64. */
int rurv_factor(rqr_handle_t h, int m, int n, void* A, int lda, int b, int p, int q, int k,
                uint64_t seed, const void* G, void* TU, int ldtu, void* WV, int ldwv, void* TV,
                int ldtv, void* DU, int lddu, void* DV, int lddv, int prec, void* work, size_t lwork,
                int* info);

/* Forms the first `ncols` columns of Q = Q_0 Q_1 ... from the block reflectors
 * that a factor call left in F (m x n, ld ldf) and T (b x n, ld ldt).
 * Q (device, out) m x ncols, ld ldq; prec RQR_FP64 or RQR_FP32. */
int rqr_form_q(rqr_handle_t h, int m, int n, int b, const void* F, int ldf, const void* T, int ldt,
               void* Q, int ldq, int ncols, int prec, void* work, size_t lwork);

/* rqr_form_q without a workspace argument, for callers that cannot allocate
 * device memory: code that must not call cudaMalloc (for example while a CUDA
 * graph is being captured), real-time or signal-safe paths, and plug-ins whose
 * host application owns every allocation and passes in only the input and
 * output buffers. The paper has no counterpart; it is a deployment aid.
 * Arguments and result are those of rqr_form_q without work/lwork. The
 * scratch is one static device array of RQR_FORM_Q_NOALLOC_MAX_BYTES in the
 * library, present on every GPU that loads it until the process exits. With
 * e = 8 (RQR_FP64) or 4 (RQR_FP32) bytes per value and r(x) = x rounded up to
 * a multiple of 256, a problem is accepted when
 *   r(m*b*e) + 2 r(b*ncols*e) <= RQR_FORM_Q_NOALLOC_MAX_BYTES
 * (with m, ncols counted as at least 1), else it returns RQR_ERR_SIZE and
 * queues nothing; what is left of the array holds split-K partial sums, so
 * near the limit the products run with fewer K splits or none. The call
 * allocates nothing. All calls share the array: calls whose GPU work overlaps
 * (other streams or handles on the same device) race on it. The first call
 * with a handle of a given device looks up that device's copy of the array
 * (cudaGetSymbolAddress, with the handle's device made current for the
 * lookup and the caller's current device restored); make that first call
 * before any stream capture. The looked-up address does not survive
 * cudaDeviceReset of that device. */
#define RQR_FORM_Q_NOALLOC_MAX_BYTES (8u << 20)
int rqr_form_q_noalloc(rqr_handle_t h, int m, int n, int b, const void* F, int ldf, const void* T, int ldt,
                       void* Q, int ldq, int ncols, int prec);

/* The dense products of the method, exposed for reuse and testing:
 * C = alpha op(A) op(B) + beta C (column-major, op = transpose when ta / tb is
 * non-zero; A is M x K or K x M, B is K x N or N x K, all device memory).
 * prec RQR_FP64 (DMMA), RQR_FP32 (FFMA) or RQR_FP64X (FP64 accuracy from bf16
 * digit planes: 8 digits of 7 bits per value, 36 digit-pair products on the
 * tcgen05 tensor cores with exact FP32 window sums, Ozaki et al. 2012);
 * alpha, beta are converted to the precision. The FP64X error is bounded
 * norm-wise: |error_ij| <~ K u max_k |a_ik| sum_k |b_kj| (u = 2^-53), like
 * FP64's own product bound up to the row/column scaling.
 * work (device) of at least rqr_gemm_workspace_bytes bytes (for FP64X it holds
 * the digit planes of op(A) and of op(B): 16 bytes per element of each). */
int rqr_gemm(rqr_handle_t h, int prec, int ta, int tb, int M, int N, int K, double alpha, const void* A, int lda,
             const void* B, int ldb, double beta, void* C, int ldc, void* work, size_t lwork);
int rqr_gemm_workspace_bytes(int prec, int M, int N, int K, size_t* bytes);

/* Differentiable form (no counterpart in the paper): reverse-mode derivative
 * of the truncated factorization X = A P = [Q1 Q2] [R11 R12; 0 R22] with the
 * column transformation P held fixed (the pivots of rqrcp_factor, or the
 * orthonormal P of rurv_factor), outputs Q1 (m x k) and R1 = [R11 R12]
 * (k x n), 1 <= k <= n <= m, FP64 data. Given the cotangents Qbar (m x k) and
 * Rbar (k x n; only the upper triangle of its leading k x k block is read),
 *   X2bar = Q1 R12bar,  Q1bar' = Qbar + X2 R12bar^T,
 *   M = R11 R11bar^T - Q1bar'^T Q1,
 *   X1bar = (Q1bar' + Q1 (tril(M) + tril(M, -1)^T)) R11^-T
 * (the thin-QR adjoint applied to the leading block, plus the product rule
 * for R12 = Q1^T X2).
 *   Q        (device) Q1, m x k, ld ldq (e.g. from rqr_form_q with ncols = k).
 *   F        (device) the factored matrix of the factor call: R11, R12 in the
 *            upper triangle of its first k rows, ld ldf.
 *   perm     (device, optional) the pivots of rqrcp_factor: then X2 is
 *            gathered from A (device, m x n, ld lda, read only when k < n) and
 *            Abar(:, perm[j]) = Xbar(:, j), so Abar is the cotangent of A.
 *            NULL: X2 (device, m x (n - k), ld ldx2, = A P(:, k:n), read only
 *            when k < n) is given, and Abar receives Xbar, the cotangent of
 *            X = A P (the caller applies P^T).
 *   Abar     (device, out) m x n, ld ldab.
 *   work     (device) rqr_qr_adjoint_workspace_bytes bytes.
 * A zero diagonal entry of R11 (rank-deficient leading block) gives
 * RQR_ERR_NONFINITE in *info; the rows it touches are left unsolved. */
int rqr_qr_adjoint(rqr_handle_t h, int m, int n, int k, const void* Q, int ldq, const void* F, int ldf,
                   const void* A, int lda, const int32_t* perm, const void* X2, int ldx2, const void* Qbar,
                   int ldqb, const void* Rbar, int ldrb, void* Abar, int ldab, void* work, size_t lwork,
                   int* info);
int rqr_qr_adjoint_workspace_bytes(int m, int n, int k, size_t* bytes);

/* R (device, out, k x n, ld ldr) = upper triangle of the first k rows of the
 * factored matrix F (device, ld ldf), zeros below; FP64. */
int rqr_copy_r(rqr_handle_t h, int k, int n, const void* F, int ldf, void* R, int ldr);

/* Batched form (config C5; the paper factors one matrix at a time): many
 * small FP32 matrices of different shapes factored in ONE persistent launch.
 * Each CTA takes the next matrix from a queue (one atomic) and runs every step
 * of the method for it. method:
 *   RQR_BATCH_QRCP  randomized QRCP, Method 1 with over-sampling p and a fresh
 *                   Gaussian per block (RESAMPLE layout), as rqrcp_factor;
 *   RQR_BATCH_URV   orthonormal pivots with q power steps (Method 2), no
 *                   over-sampling (p must be 0), truncated once k columns
 *                   are done (k <= 0: all); in the last block the Householder
 *                   QR of the power sketch's first b_i columns gives the
 *                   pivot (any orthonormal basis of the remaining columns).
 * desc (device, count x RQR_BATCH_DESC_LEN int64), per matrix:
 *   {m, n, b, k, a_off, t_off, p_off, w_off, tv_off, g_off}: shape m x n
 *   (1 <= n <= m <= max_m, n <= max_n, m <= 1024, n <= 512), block size
 *   1 <= b <= max_b <= 32 (b + p <= 64), rank k (URV); element offsets of the
 *   matrix in A (column-major, ld m), of its T (QRCP) or TU (URV) in T
 *   (b x n, ld b), of its perm (QRCP, n int32) in perm, of its WV (URV, n x n,
 *   ld n) in WV, of its TV (URV, b x n, ld b) in TV, of its Gaussians in G.
 * order (device, optional) count int32: the queue order (e.g. longest first).
 * A (device, in/out) float: R above, reflectors below, as rqrcp_factor.
 * G (device, optional) float: per matrix the blocks G_i of l x (m - k0)
 *   (QRCP: every block but the last, l = b + p; URV: every block, l = b), one
 *   after another at g_off; NULL: drawn in the kernel, block i of matrix j
 *   from the rqr_gauss_fill stream (seed, (j << 16) | i), rounded to FP32.
 * work (device) rqr_batched_workspace_bytes bytes (a per-CTA scratch sized by
 *   max_m, max_n, max_b). A matrix outside those limits is skipped and the
 *   status word reads RQR_ERR_SIZE. The launch allocates nothing and, with
 *   info == NULL, does not wait: it can be captured in a CUDA graph. */
#define RQR_BATCH_QRCP 0
#define RQR_BATCH_URV 1
#define RQR_BATCH_DESC_LEN 10
int rqr_batched_factor(rqr_handle_t h, int method, int count, const int64_t* desc, const int32_t* order, float* A,
                       float* T, int32_t* perm, float* WV, float* TV, const float* G, int p, int q, uint64_t seed,
                       int max_m, int max_n, int max_b, void* work, size_t lwork, int* info);
int rqr_batched_workspace_bytes(int method, int count, int max_m, int max_n, int max_b, int p, size_t* bytes);

/* Fills out[0:count] (device) with N(0,1) samples: element e is lane e%4 of
 * Philox4x32-10 block e/4 with counter {lo(e/4), hi(e/4), lo(stream),
 * hi(stream)} and key {lo(seed), hi(seed)}, through Box-Muller on the pairs
 * (lane0, lane1), (lane2, lane3) with u = (x + 0.5) 2^-32. prec selects
 * double (RQR_FP64) or float (RQR_FP32) output. */
int rqr_gauss_fill(rqr_handle_t h, uint64_t seed, uint64_t stream, int64_t count, void* out, int prec);

/* Raw Philox4x32-10 blocks: out[4*i + t] = lane t of the block with counter
 * {ctr0 + i, 0, ctr2, ctr3} (device out, count blocks). */
int rqr_philox_raw(rqr_handle_t h, uint32_t ctr0, uint32_t ctr2, uint32_t ctr3, uint32_t key0,
                   uint32_t key1, int64_t count, uint32_t* out);

/* Tracing: steps of the method timed with CUDA events on the handle's stream.
 * Phase indices for rqr_profile_read (paper section in brackets): */
#define RQR_PHASE_SKETCH 0   /* Gaussian draw and Y = G A, power steps [Sec. 4.1, 6.3] */
#define RQR_PHASE_PIVOT 1    /* pivots from the sketch: b steps of Fig. QR, or the
                                orthonormal pivot (QR, l->b SVD) [Sec. 4.1-4.3] */
#define RQR_PHASE_SWAP 2     /* column swaps of A, Y, perm [Fig. blockQR]        */
#define RQR_PHASE_PANEL 3    /* panel Householder QR and T [Sec. 3.2, 5.1]       */
#define RQR_PHASE_UPDATE 4   /* trailing update (I - V T V^T)^T A22 [Fig. blockQR] */
#define RQR_PHASE_DOWNDATE 5 /* sketch downdate (not in the paper)               */
#define RQR_PHASE_FINAL 6    /* last block by Fig. QR [Fig. blockQR, last step]  */
#define RQR_PHASE_RIGHT 7    /* orthonormal pivot applied from the right [Fig. blockRRQR] */
#define RQR_NUM_PHASES 8

/* Turns per-phase event recording on (on != 0) or off and clears the counters. */
int rqr_profile_enable(rqr_handle_t h, int on);

/* Waits for the handle's stream, then writes per phase (host arrays of nphase
 * entries, any may be NULL): ms = summed event time, flops = algorithmic flop
 * count of the work queued in that phase, launches = kernels launched in it
 * (counted whether or not recording is on). Clears the counters. */
int rqr_profile_read(rqr_handle_t h, double* ms, double* flops, int64_t* launches, int nphase);

/* Waits for the handle's stream, then writes the summed CUDA-event time (ms),
 * the algorithmic tensor-core flops, the algorithmic DRAM bytes and the launch
 * count of the tcgen05 product kernels launched while tracing was on (host
 * outputs, any may be NULL); clears them. FP64X kernel: 36 bf16 digit-pair
 * products of 2 M N K flops each, bytes = both operands' 8 digit planes (16
 * bytes per element) once plus C read and written. Mixed-mode kernel: 1
 * (TF32) or 3 (3XBF16, 3XTF32) products of 2 M N K, bytes = both operands'
 * planes (4 or 8 bytes per element) once plus C read and written. */
int rqr_profile_kernel_read(rqr_handle_t h, double* ms, double* flops, double* bytes, int64_t* launches);

/* Library version string (static storage). */
const char* rqr_version(void);

#ifdef __cplusplus
}
#endif
#endif
