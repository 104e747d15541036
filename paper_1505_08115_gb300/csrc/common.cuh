// common.cuh -- shared helpers for the sm_103a kernels of the randomized
// blocked QR library: launch checks, warp reductions, the workspace carver and
// the GEMM entry used by every dense contraction of the method.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <vector>

#include "../../include/rqr.h"

namespace rqr {

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs (queried at run time too)

// Event timing of one kernel class (the tcgen05 product kernel) while
// profiling is on: CUDA events around each launch on the launch stream.
struct KernelTimer {
  int on = 0;
  std::vector<cudaEvent_t> pool;  // 2 events per recorded launch
  size_t used = 0;                // pairs recorded
  double flops = 0.0;             // algorithmic tensor-core flops of the recorded launches
  double bytes = 0.0;             // algorithmic DRAM bytes of the recorded launches
  int64_t launches = 0;
  // Records the start event of a launch; false when timing is off or an event cannot be made.
  bool start(cudaStream_t s) {
    if (!on) return false;
    while (pool.size() < 2 * used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      pool.push_back(e);
    }
    cudaEventRecord(pool[2 * used], s);
    return true;
  }
  void stop(cudaStream_t s, double fl, double by) {
    cudaEventRecord(pool[2 * used + 1], s);
    ++used;
    flops += fl;
    bytes += by;
    ++launches;
  }
};

struct Ctx {
  cudaStream_t stream;
  int sms;             // multiprocessor count of the device
  int* status;         // device status word (RQR_ERR_* or 0)
  int64_t* nlaunch;    // host-side count of kernel launches (may be null)
  KernelTimer* kt = nullptr;  // optional per-launch timing of the tcgen05 products
  int device = -1;            // CUDA device of the handle (its stream belongs to it)
  unsigned long long wait_ns = 2000000000ull;  // limit of the persistent kernels' waits for other CTAs' words
};

// Counts kernel launches issued through a context (tracing aid).
inline void note_launch(const Ctx& c, int64_t n = 1) {
  if (c.nlaunch) *c.nlaunch += n;
}

// ---------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sign with sign(0) = +1 (reflector convention, Sec. 3.1).
template <typename T>
__device__ __forceinline__ T sgn0(T x) { return x < T(0) ? T(-1) : T(1); }

// ---------------------------------------------------------------- workspace
// Bump allocator over the caller's workspace; every carve is 256-byte aligned.
struct Carver {
  char* base;
  size_t cap, used;
  bool dry;  // size query only
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + used);
    used += bytes;
    return p;
  }
  bool ok() const { return dry || used <= cap; }
};

inline int ceil_div(int a, int b) { return (a + b - 1) / b; }
inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------- GEMM
// C = alpha * op(A) * op(B) + beta * C, column-major, M x N result, inner K.
// op(A) = A (ta = false, A is M x K) or A^T (ta = true, A is K x M); same for B.
// `part` is scratch for split-K partial sums (capacity part_cap elements);
// the contraction runs in the precision of T (FP64 on the DMMA pipe, FP32 on
// the FFMA pipe).
template <typename T>
void gemm(const Ctx& c, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda, const T* B,
          int ldb, T beta, T* C, int ldc, T* part, size_t part_cap);

// Split-K partial-buffer elements that gemm() may use for this shape.
size_t gemm_part_elems(int M, int N, int K, int sms);

// ---------------------------------------------------------------- kernels
// Gaussian fill (rng.cu)
template <typename T>
void gauss_fill(const Ctx& c, uint64_t seed, uint64_t stream, int64_t count, T* out);
// 2-D fill of an r x cols column-major block (ld) from the stream; element
// (i, j) takes stream index i + j*r.
template <typename T>
void gauss_fill_2d(const Ctx& c, uint64_t seed, uint64_t stream, int r, int cols, T* out, int ld);

void philox_raw(const Ctx& c, uint32_t ctr0, uint32_t ctr2, uint32_t ctr3, uint32_t k0, uint32_t k1,
                int64_t count, uint32_t* out);

// Matrix copy / fill helpers (util in panel.cu)
template <typename T>
void copy_mat(const Ctx& c, int r, int cols, const T* src, int lds, T* dst, int ldd);
template <typename T>
void set_mat(const Ctx& c, int r, int cols, T val, T* dst, int ldd);
// dst (cols x r, ld ldd) = src (r x cols, ld lds)^T.
template <typename T>
void transpose_mat(const Ctx& c, int r, int cols, const T* src, int lds, T* dst, int ldd);

// Explicit unit-lower-trapezoidal V (m' x kb, ld ldv) from the factored panel.
template <typename T>
void make_vx(const Ctx& c, int mp, int kb, const T* F, int ldf, T* V, int ldv);

// Strictly lower part of the factored panel (V without its unit diagonal).
template <typename T>
void make_vlow(const Ctx& c, int mp, int kb, const T* F, int ldf, T* V, int ldv);
// dst += alpha * src (r x cols).
template <typename T>
void add_mat(const Ctx& c, int r, int cols, T alpha, const T* src, int lds, T* dst, int ldd);

// ---------------------------------------------------------------- panel QR
struct PanelWork;
template <typename T>
struct PanelBufs {
  T* part;      // [2][C][nc + 1] partial sums (ping-pong)
  T* rowbuf;    // [2][nc] published row values (ping-pong)
  T* tau;       // [nc]
  int* ipart;   // unused placeholder for alignment
  int C;        // number of CTAs
  int rows;     // rows per CTA
};

template <typename T>
size_t panel_scratch_elems(int mp, int nc, int sms);
// flagged 8-byte words of the persistent panel's exchange (persist.cu)
size_t panel_exchange_words(int nc, int C, size_t elem);

// Unpivoted Householder QR of the mp x nc panel P (ld ldp), Sec. 3.2.
// tau receives nc scaling factors (0 where no reflector).
template <typename T>
void panel_qr(const Ctx& c, int mp, int nc, T* P, int ldp, T* tau, T* scratch);

// The same panel QR as one cooperative launch (persist.cu); false when the
// panel does not fit (nothing queued). C, R: CTAs and rows per CTA.
template <typename T>
bool panel_qr_persist(const Ctx& c, int mp, int nc, T* P, int ldp, T* tau, T* scratch, int C, int R);

// Classical pivoted QR (Fig. QR) of rows r0..m-1, columns c0..c0+nc-1 of the
// m x * matrix A; swaps move all m rows and perm[c0..].
template <typename T>
void qrcp_block(const Ctx& c, int m, int r0, int c0, int nc, T* A, int lda, int32_t* perm, T* tau,
                T* scratch);

// T factor from the Gram matrix of V (kb x kb, ld ldg) and tau (Sec. 5.1).
template <typename T>
void larft_tri(const Ctx& c, int kb, const T* gram, int ldg, const T* tau, T* Tm, int ldt);

// Gram matrix of V = E + L (unit diagonal E, strictly lower L, ld ldl) from
// gram = L^T L on entry: adds I + L1 + L1^T (L1 = top kb x kb block of L).
template <typename T>
void gram_from_lower(const Ctx& c, int kb, const T* L, int ldl, T* gram, int ldg);

// ---------------------------------------------------------------- sketch pivots
template <typename T>
size_t ypick_scratch_elems(int l, int np, int b, int sms);

// First bsteps steps of Fig. QR on the l x np sketch Y (read only); writes the
// picked positions (sequential-swap semantics) to picks[bsteps].
template <typename T>
void ypick(const Ctx& c, int l, int np, int bsteps, const T* Y, int ldy, int* picks, T* scratch);

// The same b pivot steps as one cooperative launch with the sketch resident in
// shared memory (persist.cu); false when it does not apply (nothing queued).
size_t ypick_persist_scratch_bytes(int l, int np, int sms);
template <typename T>
bool ypick_persist(const Ctx& c, int l, int np, int bsteps, const T* Y, int ldy, int* picks, void* scratch);

// Applies the swaps (j, picks[j]), j = 0..kb-1, in order to columns k0.. of
// A (all m rows), to columns y0.. of Y (l rows, optional) and to perm[k0..].
// np: positions in play (every pick lies in [j, np)); nothing is swapped once
// the status word is set.
template <typename T>
void apply_swaps(const Ctx& c, int kb, int np, const int* picks, int m, T* A, int lda, int k0, int l, T* Y, int ldy,
                 int y0, int32_t* perm, T* tmp, int* imap);

// FP64-accurate product on the bf16 tensor cores (ozaki.cu); iscr holds
// ozaki_scratch_elems(M, N) ints.
size_t ozaki_scratch_elems(int M, int N);
void gemm_f64x(const Ctx& c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
               const double* B, int ldb, double beta, double* C, int ldc, int* iscr, double* part, size_t part_cap);

// The same products on the tcgen05 tensor cores with TMA-staged digit planes
// (oztc.cu). Returns false, with nothing queued, when the tensor-map encoder is
// unavailable or the op(A) planes do not fit (the caller then falls back).
struct TcScratch {
  int* emax;      // M + N ints
  uint16_t* pa;   // digit planes of op(A): pa_cap bf16
  size_t pa_cap;
  uint16_t* pb;   // digit planes of a column chunk of op(B): pb_cap bf16
  size_t pb_cap;
};
size_t oztc_plane_elems(int rows, int K);
bool oztc_available();
bool gemm_f64x_tc(const Ctx& c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
                  const double* B, int ldb, double beta, double* C, int ldc, int* emax, uint16_t* pa, size_t pa_cap,
                  uint16_t* pb, size_t pb_cap, double* part, size_t part_cap);

// Products of the mixed-precision modes (tcmix.cu): C = alpha op(A) op(B) +
// beta C with operands rounded to TF32 / split into bf16 hi+lo / TF32
// big+small (mode = RQR_TF32, RQR_3XBF16, RQR_3XTF32) and FP32 accumulation on
// the tcgen05 tensor cores. pa, pb: scratch for the operand planes (bytes;
// op(B) is processed in column chunks that fit pb). Returns false, with
// nothing queued, when the tensor-map encoder is missing or op(A)'s planes do
// not fit.
size_t mix_plane_bytes(int mode, int rows, int K);
template <typename T>
bool gemm_mix_tc(const Ctx& c, int mode, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda,
                 const T* B, int ldb, T beta, T* C, int ldc, void* pa, size_t pa_bytes, void* pb, size_t pb_bytes,
                 T* part, size_t part_cap);

// ---------------------------------------------------------------- small SVD
// One-sided Jacobi on the r x cols matrix M (FP64, overwritten by M J); Js
// (cols x nkeep) receives the columns of J with the nkeep largest norms of
// M J, sv the sorted norms, order the column order; flags: 2 ints of scratch.
void jacobi_svd(const Ctx& c, int r, int cols, double* M, int ldm, double* J, int ldj, int nkeep, double* Js,
                int ldjs, double* sv, int* order, int* flags);
// Diagonalisation of a b_i x b_i block after jacobi_svd of M = R11^T (Sec. 6.2):
// DU <- U' = Js, DV <- Vt (normalised columns of M in sorted order, completed
// where a singular value is zero), upper triangle of F <- diag(sv).
void diag_finish(const Ctx& c, int bi, const double* M, int ldm, const int* order, const double* sv, const double* Js,
                 int ldjs, double* DU, int lddu, double* DV, int lddv, double* F, int ldf);
// M (cols x kk) = R^T, R = upper triangle of the first kk rows of F.
template <typename T>
void r_transpose(const Ctx& c, int kk, int cols, const T* F, int ldf, T* M, int ldm);
// Strictly lower part of src into dst, zeros elsewhere.
template <typename T>
void copy_lower(const Ctx& c, int r, int cols, const T* src, int lds, T* dst, int ldd);

// Differentiable form (adjoint.cu): the reverse-mode derivative of
// X = A P = Q R, truncated to k columns of Q, with P fixed.
size_t qr_adjoint_work_elems(int m, int n, int k, int sms);
int qr_adjoint(const Ctx& c, int m, int n, int k, const double* Q1, int ldq, const double* F, int ldf, const double* A,
               int lda, const int32_t* perm, const double* X2, int ldx2, const double* Qb, int ldqb, const double* Rb,
               int ldrb, double* Ab, int ldab, double* work);
// R (k x n) = upper triangle of the first k rows of F, zeros below.
void copy_upper(const Ctx& c, int k, int n, const double* F, int ldf, double* R, int ldr);

// Batched persistent factorizations of small FP32 matrices (batched.cu).
size_t batched_workspace_bytes(int method, int count, int max_m, int max_n, int max_b, int p, int sms);
int batched_factor(const Ctx& c, int method, int count, const long long* desc, const int* order, float* A, float* T,
                   int32_t* perm, float* WV, float* TV, const float* G, int p, int q, uint64_t seed, int max_m,
                   int max_n, int max_b, void* work, size_t lwork);

// Context of a live handle (false for a NULL or destroyed handle).
bool handle_ctx(rqr_handle_t h, Ctx* out);

}  // namespace rqr

#define RQR_CUDA_TRY(x)                                  \
  do {                                                   \
    cudaError_t e_ = (x);                                \
    if (e_ != cudaSuccess) return RQR_ERR_CUDA;          \
  } while (0)
