// rqr.cu -- C ABI and block drivers of the randomized blocked QR library.
//
// rqrcp_factor follows Fig. blockQR with permutation pivots (Sec. 4.1, 4.3,
// 5.2): per block of b columns
//   (a) sketch: Y = G A once, then downdated after every block (or, in
//       RESAMPLE mode, Y = G_i A(k0:m, k0:n) redrawn per block);
//   (b) b pivots from the first b steps of Fig. QR on Y (pivot.cu);
//   (c) the swaps applied to all m rows of A, to Y and to perm;
//   (d) unpivoted Householder QR of the m' x b panel (panel.cu), T from the
//       Gram matrix V^T V (Sec. 5.1, WY remark);
//   (e) trailing update A22 <- A22 - V (T^T (V^T A22)) and the sketch
//       downdate Gq = G (I - V T V^T), Y <- Y(:, b:) - Gq(:, :b) R12,
//       G <- Gq(:, b:) (gemm.cu);
// and the last block (n - k0 <= b) by classical pivoted QR (Fig. QR).
// Everything is queued on the handle's stream; no step waits for the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

// Per-phase tracing: CUDA events recorded on the handle's stream around each
// step of the method, the algorithmic flop count of each step, and the number
// of kernel launches it issued.
struct RqrProfile {
  int on = 0;
  std::vector<cudaEvent_t> pool;
  std::vector<int> span_phase;  // span s uses events 2s, 2s+1 of the pool
  double flops[RQR_NUM_PHASES] = {};
  int64_t launches[RQR_NUM_PHASES] = {};
};

struct rqr_handle_s {
  unsigned magic;
  int device;
  int sms;
  cudaStream_t stream;
  int* d_status;
  int64_t nlaunch;
  unsigned long long wait_ns;  // limit of the persistent kernels' waits for other CTAs' words
  RqrProfile prof;
  rqr::KernelTimer kt;
};

namespace {

constexpr unsigned kMagic = 0x52515231u;  // "RQR1"
constexpr unsigned long long kDefaultWaitNs = 2000000000ull;  // 2 s

bool valid(rqr_handle_t h) { return h && h->magic == kMagic; }

bool valid_prec(int prec) {
  return prec == RQR_FP64 || prec == RQR_FP32 || prec == RQR_FP64X || prec == RQR_TF32 || prec == RQR_3XBF16 ||
         prec == RQR_3XTF32;
}

rqr::Ctx make_ctx(rqr_handle_t h) {
  return rqr::Ctx{h->stream, h->sms, h->d_status, &h->nlaunch, &h->kt, h->device, h->wait_ns};
}

// Scope of one phase: start/end events when profiling is on, launches and
// algorithmic flops attributed to the phase.
class Phase {
 public:
  Phase(rqr_handle_t h, int phase, double flops) : h_(h), phase_(phase), l0_(h->nlaunch) {
    RqrProfile& p = h->prof;
    if (!p.on) return;
    const size_t s = p.span_phase.size();
    while (p.pool.size() < 2 * s + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return;
      }
      p.pool.push_back(e);
    }
    p.span_phase.push_back(phase);
    cudaEventRecord(p.pool[2 * s], h->stream);
    p.flops[phase] += flops;
    rec_ = true;
  }
  ~Phase() {
    RqrProfile& p = h_->prof;
    p.launches[phase_] += h_->nlaunch - l0_;
    if (rec_) cudaEventRecord(p.pool[2 * (p.span_phase.size() - 1) + 1], h_->stream);
  }

 private:
  rqr_handle_t h_;
  int phase_;
  int64_t l0_;
  bool rec_ = false;
};

size_t gemm_cap(int sms) { return (size_t)8 * sms * 64 * 64; }

template <typename T>
struct RqrcpWs {
  T *Y, *Gc, *Vx, *W, *W2, *gram, *GV, *GVT, *tau, *part, *pscr, *yscr, *swp;
  int *picks, *imap, *iscr;
  char* pers;
  size_t part_cap;
  rqr::TcScratch tc;
  rqr::TcScratch tcg;  // mixed modes (FP64 data): FP64X scratch of the Gram matrix V^T V
};

// Scratch of the tensor-core products: exponent maxima (FP64X), the operand
// planes of op(A) and of op(B) (op(B) is split in column chunks whose planes
// fit into kTcPlaneBudget bf16 values, 1 GiB).
constexpr size_t kTcPlaneBudget = (size_t)512 << 20;

bool is_mixed(int prec) { return prec == RQR_TF32 || prec == RQR_3XBF16 || prec == RQR_3XTF32; }

// Tensor-core product mode of a factorization precision: FP64X (digit
// planes), a mixed mode, 3XTF32 for FP32 data, or 0 (FP64: no tensor cores).
int tc_mode(int prec) {
  if (prec == RQR_FP64X || is_mixed(prec)) return prec;
  return prec == RQR_FP32 ? RQR_3XTF32 : 0;
}

// Operand planes of `rows` rows of length K, in bf16 units (2 bytes).
size_t tc_plane_units(int mode, int rows, int K) {
  if (mode == RQR_FP64X) return rqr::oztc_plane_elems(rows, K);
  return (rqr::mix_plane_bytes(mode, rows, K) + 1) / 2;
}

void carve_tc(rqr::Carver& cv, size_t emax_elems, size_t pa_elems, size_t pb_elems, rqr::TcScratch& s) {
  s.emax = cv.take<int>(emax_elems);
  s.pa_cap = pa_elems;
  s.pa = cv.take<uint16_t>(pa_elems);
  s.pb_cap = pb_elems;
  s.pb = cv.take<uint16_t>(pb_elems);
}

// Scratch of one tensor-core product through rqr_gemm (mode RQR_FP64X or a
// mixed mode): op(A)'s planes whole, op(B)'s in column chunks of at least one
// output tile (256 columns) within the plane budget.
void gemm_tc_carve(rqr::Carver& cv, int mode, int M, int N, int K, rqr::TcScratch& s) {
  M = std::max(M, 1);
  N = std::max(N, 1);
  K = std::max(K, 1);
  carve_tc(cv, mode == RQR_FP64X ? (size_t)M + N + 64 : 1, tc_plane_units(mode, M, K),
           std::min(tc_plane_units(mode, N, K), std::max(kTcPlaneBudget, tc_plane_units(mode, 256, K))), s);
}

// Dense product of the method: native precision; or, for products large
// enough to pay for the operand splitting, on the tensor cores: the
// FP64-accurate bf16 digit splitting (mode RQR_FP64X: tcgen05 kernel of
// oztc.cu, mma.sync fallback of ozaki.cu), or a mixed-precision mode with FP32
// accumulation (RQR_TF32, RQR_3XBF16, RQR_3XTF32: tcmix.cu).
template <typename T>
struct Gemm {
  const rqr::Ctx& c;
  int mode;  // tc_mode() of the factorization, 0 = native only
  int* iscr;
  T* part;
  size_t cap;
  const rqr::TcScratch* tc;  // null: no tensor-core scratch (FP64X: the mma.sync splitting only)
  void operator()(bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda, const T* B, int ldb, T beta,
                  T* C, int ldc) const {
    // products from about 1e6 multiply-adds up go to the tensor cores: below
    // that the splitting costs more than it saves; above it the FP64 pipe is
    // slower (e.g. the downdate's l x b x b product on a few CTAs: 160 us)
    const bool big = (double)M * N * K >= 1.0e6 && M >= 16 && N >= 16 && K >= 16;
    if (mode && big) {
      if constexpr (sizeof(T) == 8) {
        if (mode == RQR_FP64X) {
          if (tc && tc->pa &&
              rqr::gemm_f64x_tc(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tc->emax, tc->pa,
                                tc->pa_cap, tc->pb, tc->pb_cap, part, cap))
            return;
          rqr::gemm_f64x(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, iscr, part, cap);
          return;
        }
      }
      if (mode != RQR_FP64X && tc && tc->pa &&
          rqr::gemm_mix_tc<T>(c, mode, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, tc->pa, 2 * tc->pa_cap,
                              tc->pb, 2 * tc->pb_cap, part, cap))
        return;
    }
    rqr::gemm<T>(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, part, cap);
  }
};

template <typename T>
size_t carve_rqrcp(rqr::Carver& cv, int m, int n, int b, int p, int sms, RqrcpWs<T>& w, int tcm = 0) {
  const int l = b + p;
  w.Y = cv.take<T>((size_t)l * std::max(n, 1));
  w.Gc = cv.take<T>((size_t)l * std::max(m, 1));
  w.Vx = cv.take<T>((size_t)std::max(m, 1) * b);
  w.W = cv.take<T>((size_t)b * std::max(n, 1));
  w.W2 = cv.take<T>((size_t)b * std::max(n, 1));
  w.gram = cv.take<T>((size_t)b * b);
  w.GV = cv.take<T>((size_t)l * b);
  w.GVT = cv.take<T>((size_t)l * b);
  w.tau = cv.take<T>((size_t)b);
  w.part_cap = gemm_cap(sms);
  w.part = cv.take<T>(w.part_cap);
  w.pscr = cv.take<T>(rqr::panel_scratch_elems<T>(std::max(m, 1), b, sms));
  w.yscr = cv.take<T>(rqr::ypick_scratch_elems<T>(l, std::max(n, 1), b, sms));
  w.swp = cv.take<T>((size_t)(std::max(m, 1) + l) * 2 * b + 2 * (size_t)b + 16);
  w.picks = cv.take<int>((size_t)b);
  w.imap = cv.take<int>(1 + 4 * (size_t)b + 8);
  w.iscr = cv.take<int>(rqr::ozaki_scratch_elems(std::max(m, l), std::max(n, m)));
  w.pers = cv.take<char>(rqr::ypick_persist_scratch_bytes(l, std::max(n, 1), sms));
  w.tc = rqr::TcScratch{};
  if (tcm) {
    // largest op(A): G (l x m) or V^T (b x m') with long K, V (m' x b) with K = b;
    // largest op(B): A (n columns of length m), chunked, or short-K operands
    const int lb = std::max(l, b), mm = std::max(m, 1), nn = std::max(n, 1);
    const size_t pa = std::max(tc_plane_units(tcm, lb, mm), tc_plane_units(tcm, mm, lb));
    const size_t pb = std::max(tc_plane_units(tcm, std::max(nn, mm), lb),
                               std::min(tc_plane_units(tcm, nn, mm), kTcPlaneBudget));
    carve_tc(cv, tcm == RQR_FP64X ? (size_t)mm + nn + lb + 64 : 1, pa, pb, w.tc);
  }
  w.tcg = rqr::TcScratch{};
  if (is_mixed(tcm) && sizeof(T) == 8) {
    const int mm = std::max(m, 1);
    carve_tc(cv, (size_t)2 * b + 64, rqr::oztc_plane_elems(b, mm), rqr::oztc_plane_elems(b, mm), w.tcg);
  }
  return cv.used;
}

__global__ void k_iota(int n, int32_t* perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

int finish(rqr_handle_t h, int* info) {
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    if (info) *info = RQR_ERR_CUDA;
    return RQR_ERR_CUDA;
  }
  if (info) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
      cudaGetLastError();
      *info = RQR_ERR_CUDA;
      return RQR_ERR_CUDA;
    }
    int st = 0;
    if (cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      *info = RQR_ERR_CUDA;
      return RQR_ERR_CUDA;
    }
    *info = st;
  }
  return RQR_OK;
}

template <typename T>
int rqrcp_impl(rqr_handle_t h, int m, int n, T* A, int lda, int b, int p, uint64_t seed, const T* G, int ldg, T* Tm,
               int ldt, int32_t* perm, int sketch, int prec, void* work, size_t lwork, int* info) {
  using namespace rqr;
  const int l = b + p;
  const int tcm = tc_mode(prec);
  // FP64X splits V into its unit diagonal and strictly lower part (below)
  const bool emu = prec == RQR_FP64X;
  Carver cv{static_cast<char*>(work), lwork, 0, false};
  RqrcpWs<T> w;
  carve_rqrcp<T>(cv, m, n, b, p, h->sms, w, tcm);
  if (!cv.ok()) return RQR_ERR_WORKSPACE;
  Ctx c = make_ctx(h);
  const Gemm<T> mm{c, tcm, w.iscr, w.part, w.part_cap, tcm ? &w.tc : nullptr};
  cudaMemsetAsync(h->d_status, 0, sizeof(int), c.stream);
  if (n == 0) return finish(h, info);
  const bool down = sketch == RQR_SKETCH_DOWNDATE;
  {
    Phase ph(h, RQR_PHASE_SKETCH, down && n > b ? 2.0 * l * m * n : 0.0);
    k_iota<<<std::max(1, std::min(ceil_div(n, 256), 1024)), 256, 0, c.stream>>>(n, perm);
    note_launch(c);
    set_mat<T>(c, b, n, T(0), Tm, ldt);
    if (down && n > b) {
      if (G) copy_mat<T>(c, l, m, G, ldg, w.Gc, l);
      else gauss_fill_2d<T>(c, seed, 0, l, m, w.Gc, l);
      mm(false, false, l, n, m, T(1), w.Gc, l, A, lda, T(0), w.Y, l);
    }
  }
  size_t goff = 0;
  int k0 = 0, blk = 0;
  while (k0 < n) {
    const int np = n - k0, mp = m - k0;
    T* P = A + k0 + (size_t)k0 * lda;
    T* Tb = Tm + (size_t)k0 * ldt;
    if (np <= b) {
      // Fig. blockQR, last step: classical pivoted QR of the remaining block.
      Phase ph(h, RQR_PHASE_FINAL, 2.0 * mp * np * (double)np - 2.0 * np * (double)np * np / 3.0);
      qrcp_block<T>(c, m, k0, k0, np, A, lda, perm, w.tau, w.pscr);
      make_vx<T>(c, mp, np, P, lda, w.Vx, mp);
      gemm<T>(c, true, false, np, np, mp, T(1), w.Vx, mp, w.Vx, mp, T(0), w.gram, np, w.part, w.part_cap);
      larft_tri<T>(c, np, w.gram, np, w.tau, Tb, ldt);
      break;
    }
    if (!down) {
      Phase ph(h, RQR_PHASE_SKETCH, 2.0 * l * mp * (double)np);
      const T* Gi;
      if (G) {
        Gi = G + goff;
        goff += (size_t)l * mp;
      } else {
        gauss_fill_2d<T>(c, seed, (uint64_t)blk, l, mp, w.Gc, l);
        Gi = w.Gc;
      }
      mm(false, false, l, np, mp, T(1), Gi, l, P, lda, T(0), w.Y + (size_t)k0 * l, l);
    }
    // (b) pivots from the sketch, (c) swaps
    {
      Phase ph(h, RQR_PHASE_PIVOT, 4.0 * l * b * (double)np);
      if (!ypick_persist<T>(c, l, np, b, w.Y + (size_t)k0 * l, l, w.picks, w.pers))
        ypick<T>(c, l, np, b, w.Y + (size_t)k0 * l, l, w.picks, w.yscr);
    }
    {
      Phase ph(h, RQR_PHASE_SWAP, 0.0);
      apply_swaps<T>(c, b, np, w.picks, m, A, lda, k0, l, down ? w.Y : nullptr, l, k0, perm, w.swp, w.imap);
    }
    // (d) panel QR + T. With the tensor-core products (emu) V is split into
    // its unit diagonal E and strictly lower part L, V = E + L: the products
    // with L keep full precision under per-row/column scaling (the unit entry
    // would otherwise set the scale of every column of V), and the E parts are
    // exact row/column additions; so V^T V = L^T L + I + L1 + L1^T.
    {
      Phase ph(h, RQR_PHASE_PANEL, 2.0 * mp * (double)b * b - 2.0 * b * (double)b * b / 3.0);
      panel_qr<T>(c, mp, b, P, lda, w.tau, w.pscr);
      if (!emu && !w.tcg.pa) {
        make_vx<T>(c, mp, b, P, lda, w.Vx, mp);
        gemm<T>(c, true, false, b, b, mp, T(1), w.Vx, mp, w.Vx, mp, T(0), w.gram, b, w.part, w.part_cap);
      } else if (!emu) {
        // mixed modes: the Gram matrix of V stays FP64-accurate (T's accuracy
        // sets Q's orthogonality) through the FP64X digit products on V = E + L
        const Gemm<T> gram_mm{c, RQR_FP64X, w.iscr, w.part, w.part_cap, &w.tcg};
        make_vlow<T>(c, mp, b, P, lda, w.Vx, mp);
        gram_mm(true, false, b, b, mp, T(1), w.Vx, mp, w.Vx, mp, T(0), w.gram, b);
        gram_from_lower<T>(c, b, w.Vx, mp, w.gram, b);
        make_vx<T>(c, mp, b, P, lda, w.Vx, mp);
      } else {
        make_vlow<T>(c, mp, b, P, lda, w.Vx, mp);
        mm(true, false, b, b, mp, T(1), w.Vx, mp, w.Vx, mp, T(0), w.gram, b);
        gram_from_lower<T>(c, b, w.Vx, mp, w.gram, b);
      }
      larft_tri<T>(c, b, w.gram, b, w.tau, Tb, ldt);
    }
    // (e) trailing update
    const int n2 = np - b;
    T* A2 = A + k0 + (size_t)(k0 + b) * lda;
    {
      Phase ph(h, RQR_PHASE_UPDATE, 4.0 * mp * (double)n2 * b);
      if (!emu) {
        mm(true, false, b, n2, mp, T(1), w.Vx, mp, A2, lda, T(0), w.W, b);
        mm(true, false, b, n2, b, T(1), Tb, ldt, w.W, b, T(0), w.W2, b);
        mm(false, false, mp, n2, b, T(-1), w.Vx, mp, w.W2, b, T(1), A2, lda);
      } else {
        copy_mat<T>(c, b, n2, A2, lda, w.W, b);                              // E^T A2
        mm(true, false, b, n2, mp, T(1), w.Vx, mp, A2, lda, T(1), w.W, b);   // + L^T A2
        mm(true, false, b, n2, b, T(1), Tb, ldt, w.W, b, T(0), w.W2, b);     // T^T W
        mm(false, false, mp, n2, b, T(-1), w.Vx, mp, w.W2, b, T(1), A2, lda);  // - L W2
        add_mat<T>(c, b, n2, T(-1), w.W2, b, A2, lda);                         // - E W2
      }
    }
    if (down) {
      Phase ph(h, RQR_PHASE_DOWNDATE, 4.0 * l * mp * (double)b + 2.0 * l * b * (double)n2);
      T* Gk = w.Gc + (size_t)k0 * l;
      if (!emu) {
        mm(false, false, l, b, mp, T(1), Gk, l, w.Vx, mp, T(0), w.GV, l);
        mm(false, false, l, b, b, T(1), w.GV, l, Tb, ldt, T(0), w.GVT, l);
        mm(false, true, l, mp, b, T(-1), w.GVT, l, w.Vx, mp, T(1), Gk, l);
      } else {
        copy_mat<T>(c, l, b, Gk, l, w.GV, l);                                  // G E
        mm(false, false, l, b, mp, T(1), Gk, l, w.Vx, mp, T(1), w.GV, l);      // + G L
        mm(false, false, l, b, b, T(1), w.GV, l, Tb, ldt, T(0), w.GVT, l);
        mm(false, true, l, mp, b, T(-1), w.GVT, l, w.Vx, mp, T(1), Gk, l);     // - GVT L^T
        add_mat<T>(c, l, b, T(-1), w.GVT, l, Gk, l);                           // - GVT E^T
      }
      mm(false, false, l, n2, b, T(-1), Gk, l, A + k0 + (size_t)(k0 + b) * lda, lda, T(1),
         w.Y + (size_t)(k0 + b) * l, l);
    }
    k0 += b;
    ++blk;
  }
  return finish(h, info);
}

template <typename T>
int form_q_impl(rqr_handle_t h, int m, int n, int b, const T* F, int ldf, const T* Tm, int ldt, T* Q, int ldq,
                int ncols, void* work, size_t lwork) {
  using namespace rqr;
  Carver cv{static_cast<char*>(work), lwork, 0, false};
  T* Vx = cv.take<T>((size_t)std::max(m, 1) * b);
  T* W = cv.take<T>((size_t)b * std::max(ncols, 1));
  T* W2 = cv.take<T>((size_t)b * std::max(ncols, 1));
  const size_t cap = gemm_cap(h->sms);
  T* part = cv.take<T>(cap);
  if (!cv.ok()) return RQR_ERR_WORKSPACE;
  Ctx c = make_ctx(h);
  set_mat<T>(c, m, ncols, T(0), Q, ldq);
  set_mat<T>(c, 1, std::min(m, ncols), T(1), Q, ldq + 1);  // unit diagonal
  // block starts
  int nb = 0;
  for (int k0 = 0; k0 < n; k0 += (n - k0 > b ? b : n - k0)) ++nb;
  int* starts = new (std::nothrow) int[nb > 0 ? nb : 1];
  if (!starts) return RQR_ERR_CUDA;
  {
    int i = 0;
    for (int k0 = 0; k0 < n; k0 += (n - k0 > b ? b : n - k0)) starts[i++] = k0;
  }
  for (int i = nb - 1; i >= 0; --i) {
    const int k0 = starts[i], kb = std::min(b, n - k0), mp = m - k0;
    make_vx<T>(c, mp, kb, F + k0 + (size_t)k0 * ldf, ldf, Vx, mp);
    T* Qk = Q + k0;
    gemm<T>(c, true, false, kb, ncols, mp, T(1), Vx, mp, Qk, ldq, T(0), W, kb, part, cap);
    gemm<T>(c, false, false, kb, ncols, kb, T(1), Tm + (size_t)k0 * ldt, ldt, W, kb, T(0), W2, kb, part, cap);
    gemm<T>(c, false, false, mp, ncols, kb, T(-1), Vx, mp, W2, kb, T(1), Qk, ldq, part, cap);
  }
  delete[] starts;
  return finish(h, nullptr);
}


struct RurvWs {
  double *Z, *Qz, *Wm, *Qw, *Vx, *gram, *Tz, *W1, *Mj, *Jm, *Js, *sv, *Zr, *P1, *P2, *W, *W2, *tau, *part, *pscr;
  double *Vl, *Tt;  // tensor-core modes: strictly lower part of V (FP64X), transposed products
  int *order, *flags, *iscr;
  size_t part_cap;
  rqr::TcScratch tc;
};

size_t carve_rurv(rqr::Carver& cv, int m, int n, int b, int p, int sms, RurvWs& w, int tcm = 0) {
  const int l = b + p;
  const size_t mm = std::max(m, 1), nn = std::max(n, 1), mx = std::max(mm, nn);
  w.Z = cv.take<double>(nn * l);
  w.Qz = cv.take<double>(nn * l);
  w.Wm = cv.take<double>(mm * l);
  w.Qw = cv.take<double>(mm * l);
  w.Vx = cv.take<double>(mx * l);
  w.gram = cv.take<double>((size_t)l * l);
  w.Tz = cv.take<double>((size_t)l * l);
  w.W1 = cv.take<double>((size_t)l * l);
  w.Mj = cv.take<double>((size_t)l * l);
  w.Jm = cv.take<double>((size_t)l * l);
  w.Js = cv.take<double>((size_t)l * b);
  w.sv = cv.take<double>((size_t)l);
  w.Zr = cv.take<double>(nn * b);
  w.P1 = cv.take<double>(mm * b);
  w.P2 = cv.take<double>(mm * b);
  w.W = cv.take<double>((size_t)b * nn);
  w.W2 = cv.take<double>((size_t)b * nn);
  w.tau = cv.take<double>((size_t)l);
  w.part_cap = gemm_cap(sms);
  w.part = cv.take<double>(w.part_cap);
  w.pscr = cv.take<double>(rqr::panel_scratch_elems<double>((int)mx, l, sms));
  w.order = cv.take<int>((size_t)l);
  w.flags = cv.take<int>(8);
  w.Vl = w.Tt = nullptr;
  w.iscr = nullptr;
  w.tc = rqr::TcScratch{};
  if (tcm) {
    // op(A) of every tensor-core product is one of the thin factors (at most
    // max(l, b) rows or columns of length max(m, n)); the large matrix is op(B)
    const int lb = std::max(l, b);
    w.Vl = cv.take<double>(mx * b);
    w.Tt = cv.take<double>(mx * lb);
    w.iscr = cv.take<int>(rqr::ozaki_scratch_elems((int)std::max<size_t>(mx, l), (int)mx));
    const size_t pa = std::max(tc_plane_units(tcm, lb, (int)mx), tc_plane_units(tcm, (int)mx, lb));
    const size_t pb = std::max(tc_plane_units(tcm, (int)mx, lb), std::min(tc_plane_units(tcm, (int)mx, (int)mx),
                                                                         kTcPlaneBudget));
    carve_tc(cv, tcm == RQR_FP64X ? 2 * mx + lb + 64 : 1, pa, pb, w.tc);
  }
  return cv.used;
}

// Q (r x kq) = (I - V T V^T)[I_kq; 0] from a panel factored in place (r x cc).
void form_thin_q(const rqr::Ctx& c, int r, int cc, int kq, const double* F, int ldf, const double* tau, RurvWs& w,
                 double* Q, int ldq) {
  using namespace rqr;
  make_vx<double>(c, r, cc, F, ldf, w.Vx, r);
  gemm<double>(c, true, false, cc, cc, r, 1.0, w.Vx, r, w.Vx, r, 0.0, w.gram, cc, w.part, w.part_cap);
  larft_tri<double>(c, cc, w.gram, cc, tau, w.Tz, cc);
  gemm<double>(c, false, true, cc, kq, cc, 1.0, w.Tz, cc, w.Vx, r, 0.0, w.W1, cc, w.part, w.part_cap);
  set_mat<double>(c, r, kq, 0.0, Q, ldq);
  set_mat<double>(c, 1, std::min(r, kq), 1.0, Q, ldq + 1);
  gemm<double>(c, false, false, r, kq, cc, -1.0, w.Vx, r, w.W1, cc, 1.0, Q, ldq, w.part, w.part_cap);
}

int rurv_impl(rqr_handle_t h, int m, int n, double* A, int lda, int b, int p, int q, int k, uint64_t seed,
              const double* G, double* TU, int ldtu, double* WV, int ldwv, double* TV, int ldtv, double* DU, int lddu,
              double* DV, int lddv, int prec, void* work, size_t lwork, int* info) {
  using namespace rqr;
  const int l = b + p;
  const int tcm = tc_mode(prec);
  const bool emu = prec == RQR_FP64X;  // V = E + L split of the FP64X products (see rqrcp_impl)
  Carver cv{static_cast<char*>(work), lwork, 0, false};
  RurvWs w;
  carve_rurv(cv, m, n, b, p, h->sms, w, tcm);
  if (!cv.ok()) return RQR_ERR_WORKSPACE;
  Ctx c = make_ctx(h);
  const Gemm<double> mm{c, tcm, w.iscr, w.part, w.part_cap, tcm ? &w.tc : nullptr};
  // C (M x N) = op(A) op(B) with a large op(A): the tensor-core kernels need
  // op(A)'s planes whole, so they compute C^T = op(B)^T op(A)^T (the large
  // matrix becomes op(B), split in column chunks) and the result is transposed.
  auto mm_t = [&](bool ta, bool tb, int M, int N, int K, const double* Am, int ldam, const double* Bm, int ldbm,
                  double* Cm, int ldcm) {
    if (!tcm) {
      gemm<double>(c, ta, tb, M, N, K, 1.0, Am, ldam, Bm, ldbm, 0.0, Cm, ldcm, w.part, w.part_cap);
      return;
    }
    mm(!tb, !ta, N, M, K, 1.0, Bm, ldbm, Am, ldam, 0.0, w.Tt, N);
    transpose_mat<double>(c, N, M, w.Tt, N, Cm, ldcm);
  };
  cudaMemsetAsync(h->d_status, 0, sizeof(int), c.stream);
  if (n == 0) return finish(h, info);
  set_mat<double>(c, b, n, 0.0, TU, ldtu);
  set_mat<double>(c, b, n, 0.0, TV, ldtv);
  set_mat<double>(c, n, n, 0.0, WV, ldwv);
  size_t goff = 0;
  int k0 = 0, blk = 0;
  while (k0 < n) {
    const int np = n - k0, mp = m - k0, bi = std::min(b, np);
    double* X = A + k0 + (size_t)k0 * lda;
    int zc = l;
    {
      // Sec. 4.2 / 6.3: Z = X^T Omega, then q power steps with orthonormalisation
      Phase ph(h, RQR_PHASE_SKETCH, (2.0 * q + 1.0) * 2.0 * l * mp * (double)np);
      const double* Gi;
      if (G) {
        Gi = G + goff;
        goff += (size_t)l * mp;
      } else {
        gauss_fill_2d<double>(c, seed, (uint64_t)blk, l, mp, w.Qw, l);
        Gi = w.Qw;
      }
      mm_t(true, true, np, l, mp, X, lda, Gi, l, w.Z, np);
      for (int t = 0; t < q; ++t) {
        const int kz = std::min(np, zc);
        panel_qr<double>(c, np, zc, w.Z, np, w.tau, w.pscr);
        form_thin_q(c, np, zc, kz, w.Z, np, w.tau, w, w.Qz, np);
        mm_t(false, false, mp, kz, np, X, lda, w.Qz, np, w.Wm, mp);
        const int kw = std::min(mp, kz);
        panel_qr<double>(c, mp, kz, w.Wm, mp, w.tau, w.pscr);
        form_thin_q(c, mp, kz, kw, w.Wm, mp, w.tau, w, w.Qw, mp);
        mm_t(true, false, np, kw, mp, X, lda, w.Qw, mp, w.Z, np);
        zc = kw;
      }
    }
    double* TS = TV + (size_t)k0 * ldtv;
    double* Wb = WV + k0 + (size_t)k0 * ldwv;
    {
      // l -> b_i reduction through the SVD of R_z, then Householder QR of Z
      Phase ph(h, RQR_PHASE_PIVOT, 2.0 * np * (double)zc * zc + 2.0 * np * (double)bi * bi);
      double* Zb = w.Z;
      if (zc > bi) {
        const int kk = std::min(np, zc);
        panel_qr<double>(c, np, zc, w.Z, np, w.tau, w.pscr);
        form_thin_q(c, np, zc, kk, w.Z, np, w.tau, w, w.Qz, np);
        r_transpose<double>(c, kk, zc, w.Z, np, w.Mj, zc);
        jacobi_svd(c, zc, kk, w.Mj, zc, w.Jm, kk, bi, w.Js, kk, w.sv, w.order, w.flags);
        gemm<double>(c, false, false, np, bi, kk, 1.0, w.Qz, np, w.Js, kk, 0.0, w.Zr, np, w.part, w.part_cap);
        Zb = w.Zr;
      }
      panel_qr<double>(c, np, bi, Zb, np, w.tau, w.pscr);
      copy_lower<double>(c, np, bi, Zb, np, Wb, ldwv);
      make_vx<double>(c, np, bi, Zb, np, w.Vx, np);
      gemm<double>(c, true, false, bi, bi, np, 1.0, w.Vx, np, w.Vx, np, 0.0, w.gram, bi, w.part, w.part_cap);
      larft_tri<double>(c, bi, w.gram, bi, w.tau, TS, ldtv);
    }
    {
      // A(0:m, k0:n) <- A(0:m, k0:n) (I - W TS W^T), all m rows (Fig. blockRRQR)
      Phase ph(h, RQR_PHASE_RIGHT, 4.0 * m * (double)np * bi);
      double* Ak = A + (size_t)k0 * lda;
      if (!emu) {
        mm_t(false, false, m, bi, np, Ak, lda, w.Vx, np, w.P1, m);
        gemm<double>(c, false, false, m, bi, bi, 1.0, w.P1, m, TS, ldtv, 0.0, w.P2, m, w.part, w.part_cap);
        mm(false, true, m, np, bi, -1.0, w.P2, m, w.Vx, np, 1.0, Ak, lda);
      } else {
        // W = E + L (unit diagonal E = [I; 0], strictly lower L), as in the left update
        make_vlow<double>(c, np, bi, w.Vx, np, w.Vl, np);
        mm_t(false, false, m, bi, np, Ak, lda, w.Vl, np, w.P1, m);                 // A L
        add_mat<double>(c, m, bi, 1.0, Ak, lda, w.P1, m);                           // + A E
        gemm<double>(c, false, false, m, bi, bi, 1.0, w.P1, m, TS, ldtv, 0.0, w.P2, m, w.part, w.part_cap);
        mm(false, true, m, np, bi, -1.0, w.P2, m, w.Vl, np, 1.0, Ak, lda);          // - P2 L^T
        add_mat<double>(c, m, bi, -1.0, w.P2, m, Ak, lda);                          // - P2 E^T
      }
    }
    double* Tb = TU + (size_t)k0 * ldtu;
    {
      Phase ph(h, RQR_PHASE_PANEL, 2.0 * mp * (double)bi * bi - 2.0 * bi * (double)bi * bi / 3.0);
      panel_qr<double>(c, mp, bi, X, lda, w.tau, w.pscr);
      make_vx<double>(c, mp, bi, X, lda, w.Vx, mp);
      gemm<double>(c, true, false, bi, bi, mp, 1.0, w.Vx, mp, w.Vx, mp, 0.0, w.gram, bi, w.part, w.part_cap);
      larft_tri<double>(c, bi, w.gram, bi, w.tau, Tb, ldtu);
    }
    const int n2 = np - bi;
    if (n2 > 0) {
      Phase ph(h, RQR_PHASE_UPDATE, 4.0 * mp * (double)n2 * bi);
      double* A2 = A + k0 + (size_t)(k0 + bi) * lda;
      if (!emu) {
        mm(true, false, bi, n2, mp, 1.0, w.Vx, mp, A2, lda, 0.0, w.W, bi);
        mm(true, false, bi, n2, bi, 1.0, Tb, ldtu, w.W, bi, 0.0, w.W2, bi);
        mm(false, false, mp, n2, bi, -1.0, w.Vx, mp, w.W2, bi, 1.0, A2, lda);
      } else {
        make_vlow<double>(c, mp, bi, X, lda, w.Vl, mp);
        copy_mat<double>(c, bi, n2, A2, lda, w.W, bi);                             // E^T A2
        mm(true, false, bi, n2, mp, 1.0, w.Vl, mp, A2, lda, 1.0, w.W, bi);         // + L^T A2
        gemm<double>(c, true, false, bi, n2, bi, 1.0, Tb, ldtu, w.W, bi, 0.0, w.W2, bi, w.part, w.part_cap);
        mm(false, false, mp, n2, bi, -1.0, w.Vl, mp, w.W2, bi, 1.0, A2, lda);      // - L W2
        add_mat<double>(c, bi, n2, -1.0, w.W2, bi, A2, lda);                        // - E W2
      }
    }
    if (DU && DV) {
      // Sec. 6.2 (Fig. blockRRQR): R11 = U' D Vt^T; A(0:k0, block) <- A(0:k0, block) Vt,
      // R12 <- U'^T R12, R11 <- D
      Phase ph(h, RQR_PHASE_PANEL, 6.0 * bi * (double)bi * bi + 2.0 * (k0 + n2) * (double)bi * bi);
      r_transpose<double>(c, bi, bi, X, lda, w.Mj, bi);
      jacobi_svd(c, bi, bi, w.Mj, bi, w.Jm, bi, bi, w.Js, bi, w.sv, w.order, w.flags);
      double* Ub = DU + (size_t)k0 * lddu;
      double* Vb = DV + (size_t)k0 * lddv;
      diag_finish(c, bi, w.Mj, bi, w.order, w.sv, w.Js, bi, Ub, lddu, Vb, lddv, X, lda);
      if (k0 > 0) {
        double* Ab = A + (size_t)k0 * lda;
        gemm<double>(c, false, false, k0, bi, bi, 1.0, Ab, lda, Vb, lddv, 0.0, w.P1, k0, w.part, w.part_cap);
        copy_mat<double>(c, k0, bi, w.P1, k0, Ab, lda);
      }
      if (n2 > 0) {
        double* R12 = A + k0 + (size_t)(k0 + bi) * lda;
        gemm<double>(c, true, false, bi, n2, bi, 1.0, Ub, lddu, R12, lda, 0.0, w.W, bi, w.part, w.part_cap);
        copy_mat<double>(c, bi, n2, w.W, bi, R12, lda);
      }
    }
    k0 += bi;
    ++blk;
    if (k > 0 && k0 >= k) break;
  }
  return finish(h, info);
}

}  // namespace

namespace rqr {
// Stream, SM count, status word and launch counter of a live handle.
bool handle_ctx(rqr_handle_t h, Ctx* out) {
  if (!valid(h) || !out) return false;
  *out = make_ctx(h);
  return true;
}
}  // namespace rqr

extern "C" {

int rqr_create(rqr_handle_t* h, void* stream) {
  if (!h) return -1;
  *h = nullptr;
  rqr_handle_s* s = new (std::nothrow) rqr_handle_s();
  if (!s) return RQR_ERR_CUDA;
  s->magic = kMagic;
  s->nlaunch = 0;
  s->wait_ns = kDefaultWaitNs;
  s->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess ||
      cudaMalloc(&s->d_status, 64) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return RQR_ERR_CUDA;
  }
  cudaMemset(s->d_status, 0, 64);
  *h = s;
  return RQR_OK;
}

int rqr_destroy(rqr_handle_t h) {
  if (!valid(h)) return RQR_ERR_HANDLE;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->d_status);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  for (cudaEvent_t e : h->kt.pool) cudaEventDestroy(e);
  h->magic = 0;
  delete h;
  return RQR_OK;
}

int rqr_set_stream(rqr_handle_t h, void* stream) {
  if (!valid(h)) return RQR_ERR_HANDLE;
  h->stream = static_cast<cudaStream_t>(stream);
  return RQR_OK;
}

int rqr_set_wait_limit_ns(rqr_handle_t h, uint64_t ns) {
  if (!valid(h)) return -1;
  h->wait_ns = ns == 0 ? kDefaultWaitNs : (unsigned long long)ns;
  return RQR_OK;
}

int rqr_workspace_bytes(int m, int n, int b, int p, int q, int prec, int sketch, size_t* bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (b < 1 || b > 512) return -3;
  if (p < 0) return -4;
  if (!valid_prec(prec)) return -6;
  if (sketch != RQR_SKETCH_DOWNDATE && sketch != RQR_SKETCH_RESAMPLE) return -7;
  if (!bytes) return -8;
  int dev = 0, sms = rqr::kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  rqr::Carver cv{nullptr, 0, 0, true};
  if (q >= 0) {
    if (prec == RQR_FP32) return -6;
    RurvWs w;
    carve_rurv(cv, m, n, b, p, sms, w, tc_mode(prec));
  } else if (prec != RQR_FP32) {
    RqrcpWs<double> w;
    carve_rqrcp<double>(cv, m, n, b, p, sms, w, tc_mode(prec));
  } else {
    RqrcpWs<float> w;
    carve_rqrcp<float>(cv, m, n, b, p, sms, w, tc_mode(prec));
  }
  *bytes = cv.used + 256;
  return RQR_OK;
}

int rqrcp_factor(rqr_handle_t h, int m, int n, void* A, int lda, int b, int p, uint64_t seed, const void* G, int ldg,
                 void* T, int ldt, int32_t* perm, int prec, int sketch, void* work, size_t lwork, int* info) {
  if (!valid(h)) return -1;
  if (m < 0) return -2;
  if (n < 0 || n > m) return -3;
  if (!A && n > 0) return -4;
  if (lda < std::max(1, m)) return -5;
  if (b < 1 || b > 512) return -6;
  if (p < 0 || b + p > 1024) return -7;
  if (G && sketch == RQR_SKETCH_DOWNDATE && ldg < b + p) return -10;
  if (!T && n > 0) return -11;
  if (ldt < b) return -12;
  if (!perm && n > 0) return -13;
  if (!valid_prec(prec)) return -14;
  if (sketch != RQR_SKETCH_DOWNDATE && sketch != RQR_SKETCH_RESAMPLE) return -15;
  if (!work && n > 0) return -16;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return -16;
  cudaGetLastError();
  if (prec != RQR_FP32)
    return rqrcp_impl<double>(h, m, n, static_cast<double*>(A), lda, b, p, seed, static_cast<const double*>(G), ldg,
                              static_cast<double*>(T), ldt, perm, sketch, prec, work, lwork, info);
  return rqrcp_impl<float>(h, m, n, static_cast<float*>(A), lda, b, p, seed, static_cast<const float*>(G), ldg,
                           static_cast<float*>(T), ldt, perm, sketch, prec, work, lwork, info);
}

int rurv_factor(rqr_handle_t h, int m, int n, void* A, int lda, int b, int p, int q, int k, uint64_t seed,
                const void* G, void* TU, int ldtu, void* WV, int ldwv, void* TV, int ldtv, void* DU, int lddu,
                void* DV, int lddv, int prec, void* work, size_t lwork, int* info) {
  if (!valid(h)) return -1;
  if (m < 0) return -2;
  if (n < 0 || n > m) return -3;
  if (!A && n > 0) return -4;
  if (lda < std::max(1, m)) return -5;
  if (b < 1 || b > 512) return -6;
  if (p < 0 || b + p > 1024) return -7;
  if (q < 0 || q > 64) return -8;
  if (!TU && n > 0) return -12;
  if (ldtu < b) return -13;
  if (!WV && n > 0) return -14;
  if (ldwv < std::max(1, n)) return -15;
  if (!TV && n > 0) return -16;
  if (ldtv < b) return -17;
  if ((DU == nullptr) != (DV == nullptr)) return DU ? -20 : -18;
  if (DU && lddu < b) return -19;
  if (DV && lddv < b) return -21;
  if (!valid_prec(prec) || prec == RQR_FP32) return -22;
  if (!work && n > 0) return -23;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return -23;
  cudaGetLastError();
  return rurv_impl(h, m, n, static_cast<double*>(A), lda, b, p, q, k, seed, static_cast<const double*>(G),
                   static_cast<double*>(TU), ldtu, static_cast<double*>(WV), ldwv, static_cast<double*>(TV), ldtv,
                   static_cast<double*>(DU), lddu, static_cast<double*>(DV), lddv, prec, work, lwork, info);
}

int rqr_form_q(rqr_handle_t h, int m, int n, int b, const void* F, int ldf, const void* T, int ldt, void* Q, int ldq,
               int ncols, int prec, void* work, size_t lwork) {
  if (!valid(h)) return -1;
  if (m < 0) return -2;
  if (n < 0 || n > m) return -3;
  if (b < 1 || b > 512) return -4;
  if (!F && n > 0) return -5;
  if (ldf < std::max(1, m)) return -6;
  if (!T && n > 0) return -7;
  if (ldt < b) return -8;
  if (!Q) return -9;
  if (ldq < std::max(1, m)) return -10;
  if (ncols < 0 || ncols > m) return -11;
  if (prec != RQR_FP64 && prec != RQR_FP32) return -12;
  if (!work) return -13;
  cudaGetLastError();
  if (prec == RQR_FP64)
    return form_q_impl<double>(h, m, n, b, static_cast<const double*>(F), ldf, static_cast<const double*>(T), ldt,
                               static_cast<double*>(Q), ldq, ncols, work, lwork);
  return form_q_impl<float>(h, m, n, b, static_cast<const float*>(F), ldf, static_cast<const float*>(T), ldt,
                            static_cast<float*>(Q), ldq, ncols, work, lwork);
}

int rqr_gauss_fill(rqr_handle_t h, uint64_t seed, uint64_t stream, int64_t count, void* out, int prec) {
  if (!valid(h)) return -1;
  if (count < 0) return -4;
  if (!out && count > 0) return -5;
  if (prec != RQR_FP64 && prec != RQR_FP32) return -6;
  cudaGetLastError();
  rqr::Ctx c = make_ctx(h);
  if (prec == RQR_FP64) rqr::gauss_fill<double>(c, seed, stream, count, static_cast<double*>(out));
  else rqr::gauss_fill<float>(c, seed, stream, count, static_cast<float*>(out));
  return finish(h, nullptr);
}

int rqr_philox_raw(rqr_handle_t h, uint32_t ctr0, uint32_t ctr2, uint32_t ctr3, uint32_t key0, uint32_t key1,
                   int64_t count, uint32_t* out) {
  if (!valid(h)) return -1;
  if (count < 0) return -7;
  if (!out && count > 0) return -8;
  cudaGetLastError();
  rqr::Ctx c = make_ctx(h);
  rqr::philox_raw(c, ctr0, ctr2, ctr3, key0, key1, count, out);
  return finish(h, nullptr);
}

int rqr_profile_enable(rqr_handle_t h, int on) {
  if (!valid(h)) return -1;
  RqrProfile& p = h->prof;
  p.on = on ? 1 : 0;
  h->kt.on = p.on;
  h->kt.used = 0;
  h->kt.flops = 0.0;
  h->kt.bytes = 0.0;
  h->kt.launches = 0;
  p.span_phase.clear();
  for (int i = 0; i < RQR_NUM_PHASES; ++i) {
    p.flops[i] = 0.0;
    p.launches[i] = 0;
  }
  return RQR_OK;
}

int rqr_profile_read(rqr_handle_t h, double* ms, double* flops, int64_t* launches, int nphase) {
  if (!valid(h)) return -1;
  if (nphase < 0) return -5;
  RqrProfile& p = h->prof;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return RQR_ERR_CUDA;
  }
  double acc[RQR_NUM_PHASES] = {};
  for (size_t s = 0; s < p.span_phase.size(); ++s) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.pool[2 * s], p.pool[2 * s + 1]) == cudaSuccess) acc[p.span_phase[s]] += t;
    else cudaGetLastError();
  }
  const int k = std::min(nphase, (int)RQR_NUM_PHASES);
  for (int i = 0; i < k; ++i) {
    if (ms) ms[i] = acc[i];
    if (flops) flops[i] = p.flops[i];
    if (launches) launches[i] = p.launches[i];
  }
  return rqr_profile_enable(h, p.on);
}

int rqr_profile_kernel_read(rqr_handle_t h, double* ms, double* flops, double* bytes, int64_t* launches) {
  if (!valid(h)) return -1;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
    cudaGetLastError();
    return RQR_ERR_CUDA;
  }
  rqr::KernelTimer& k = h->kt;
  double acc = 0.0;
  for (size_t i = 0; i < k.used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, k.pool[2 * i], k.pool[2 * i + 1]) == cudaSuccess) acc += t;
    else cudaGetLastError();
  }
  if (ms) *ms = acc;
  if (flops) *flops = k.flops;
  if (bytes) *bytes = k.bytes;
  if (launches) *launches = k.launches;
  k.used = 0;
  k.flops = 0.0;
  k.bytes = 0.0;
  k.launches = 0;
  return RQR_OK;
}

int rqr_gemm(rqr_handle_t h, int prec, int ta, int tb, int M, int N, int K, double alpha, const void* A, int lda,
             const void* B, int ldb, double beta, void* C, int ldc, void* work, size_t lwork) {
  if (!valid(h)) return -1;
  if (!valid_prec(prec)) return -2;
  if (M < 0) return -5;
  if (N < 0) return -6;
  if (K < 0) return -7;
  const int ar = ta ? K : M, br = tb ? N : K;
  if (!A && M > 0 && K > 0) return -9;
  if (lda < std::max(1, ar)) return -10;
  if (!B && N > 0 && K > 0) return -11;
  if (ldb < std::max(1, br)) return -12;
  if (!C && M > 0 && N > 0) return -14;
  if (ldc < std::max(1, M)) return -15;
  size_t need = 0;
  rqr_gemm_workspace_bytes(prec, M, N, K, &need);
  if (lwork < need || (need > 0 && !work)) return RQR_ERR_WORKSPACE;
  cudaGetLastError();
  rqr::Ctx c = make_ctx(h);
  rqr::Carver cv{static_cast<char*>(work), lwork, 0, false};
  if (prec == RQR_FP32) {
    const size_t cap = gemm_cap(h->sms);
    float* part = cv.take<float>(cap);
    rqr::gemm<float>(c, ta != 0, tb != 0, M, N, K, (float)alpha, static_cast<const float*>(A), lda,
                     static_cast<const float*>(B), ldb, (float)beta, static_cast<float*>(C), ldc, part, cap);
  } else if (is_mixed(prec)) {
    const size_t cap = gemm_cap(h->sms);
    double* part = cv.take<double>(cap);
    rqr::TcScratch tc{};
    gemm_tc_carve(cv, prec, M, N, K, tc);
    if (M > 0 && N > 0 && K > 0 &&
        rqr::gemm_mix_tc<double>(c, prec, ta != 0, tb != 0, M, N, K, alpha, static_cast<const double*>(A), lda,
                                 static_cast<const double*>(B), ldb, beta, static_cast<double*>(C), ldc, tc.pa,
                                 2 * tc.pa_cap, tc.pb, 2 * tc.pb_cap, part, cap))
      return finish(h, nullptr);
    // no tensor-map encoder (or an empty product): the FP64 product
    rqr::gemm<double>(c, ta != 0, tb != 0, M, N, K, alpha, static_cast<const double*>(A), lda,
                      static_cast<const double*>(B), ldb, beta, static_cast<double*>(C), ldc, part, cap);
  } else {
    const size_t cap = gemm_cap(h->sms);
    double* part = cv.take<double>(cap);
    int* iscr = cv.take<int>(rqr::ozaki_scratch_elems(M, N));
    rqr::TcScratch tc{};
    if (prec == RQR_FP64X) gemm_tc_carve(cv, prec, M, N, K, tc);
    const Gemm<double> mm{c, prec == RQR_FP64X ? RQR_FP64X : 0, iscr, part, cap, prec == RQR_FP64X ? &tc : nullptr};
    if (prec == RQR_FP64X && M > 0 && N > 0 && K > 0) {
      if (!rqr::gemm_f64x_tc(c, ta != 0, tb != 0, M, N, K, alpha, static_cast<const double*>(A), lda,
                             static_cast<const double*>(B), ldb, beta, static_cast<double*>(C), ldc, tc.emax, tc.pa,
                             tc.pa_cap, tc.pb, tc.pb_cap, part, cap))
        rqr::gemm_f64x(c, ta != 0, tb != 0, M, N, K, alpha, static_cast<const double*>(A), lda,
                       static_cast<const double*>(B), ldb, beta, static_cast<double*>(C), ldc, iscr, part, cap);
    } else
      mm(ta != 0, tb != 0, M, N, K, alpha, static_cast<const double*>(A), lda, static_cast<const double*>(B), ldb,
         beta, static_cast<double*>(C), ldc);
  }
  return finish(h, nullptr);
}

int rqr_gemm_workspace_bytes(int prec, int M, int N, int K, size_t* bytes) {
  if (!bytes) return -5;
  if (!valid_prec(prec)) return -1;
  int dev = 0, sms = rqr::kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  rqr::Carver cv{nullptr, 0, 0, true};
  if (prec == RQR_FP32) cv.take<float>(gemm_cap(sms));
  else if (is_mixed(prec)) {
    cv.take<double>(gemm_cap(sms));
    rqr::TcScratch tc{};
    gemm_tc_carve(cv, prec, M, N, K, tc);
  } else {
    cv.take<double>(gemm_cap(sms));
    cv.take<int>(rqr::ozaki_scratch_elems(std::max(M, 0), std::max(N, 0)));
    if (prec == RQR_FP64X) {
      rqr::TcScratch tc{};
      gemm_tc_carve(cv, prec, M, N, K, tc);
    }
  }
  *bytes = cv.used;
  return RQR_OK;
}

int rqr_qr_adjoint_workspace_bytes(int m, int n, int k, size_t* bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (k < 0 || k > n) return -3;
  if (!bytes) return -4;
  int dev = 0, sms = rqr::kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  *bytes = sizeof(double) * rqr::qr_adjoint_work_elems(m, n, k, sms) + 256;
  return RQR_OK;
}

int rqr_qr_adjoint(rqr_handle_t h, int m, int n, int k, const void* Q, int ldq, const void* F, int ldf, const void* A,
                   int lda, const int32_t* perm, const void* X2, int ldx2, const void* Qbar, int ldqb, const void* Rbar,
                   int ldrb, void* Abar, int ldab, void* work, size_t lwork, int* info) {
  if (!valid(h)) return -1;
  if (m < 0) return -2;
  if (n < 1 || n > m) return -3;
  if (k < 1 || k > n) return -4;
  if (!Q) return -5;
  if (ldq < std::max(1, m)) return -6;
  if (!F) return -7;
  if (ldf < std::max(1, m)) return -8;
  if (perm && k < n && !A) return -9;
  if (perm && k < n && lda < std::max(1, m)) return -10;
  if (!perm && k < n && !X2) return -12;
  if (!perm && k < n && ldx2 < std::max(1, m)) return -13;
  if (!Qbar) return -14;
  if (ldqb < std::max(1, m)) return -15;
  if (!Rbar) return -16;
  if (ldrb < k) return -17;
  if (!Abar) return -18;
  if (ldab < std::max(1, m)) return -19;
  if (!work) return -20;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return -20;
  if (lwork < sizeof(double) * rqr::qr_adjoint_work_elems(m, n, k, h->sms)) return RQR_ERR_WORKSPACE;
  cudaGetLastError();
  rqr::Ctx c = make_ctx(h);
  cudaMemsetAsync(h->d_status, 0, sizeof(int), c.stream);
  rqr::qr_adjoint(c, m, n, k, static_cast<const double*>(Q), ldq, static_cast<const double*>(F), ldf,
                  static_cast<const double*>(A), lda, perm, static_cast<const double*>(X2), ldx2,
                  static_cast<const double*>(Qbar), ldqb, static_cast<const double*>(Rbar), ldrb,
                  static_cast<double*>(Abar), ldab, static_cast<double*>(work));
  return finish(h, info);
}

int rqr_copy_r(rqr_handle_t h, int k, int n, const void* F, int ldf, void* R, int ldr) {
  if (!valid(h)) return -1;
  if (k < 0) return -2;
  if (n < 0) return -3;
  if (!F && k > 0 && n > 0) return -4;
  if (ldf < std::max(1, k)) return -5;
  if (!R && k > 0 && n > 0) return -6;
  if (ldr < std::max(1, k)) return -7;
  cudaGetLastError();
  rqr::Ctx c = make_ctx(h);
  rqr::copy_upper(c, k, n, static_cast<const double*>(F), ldf, static_cast<double*>(R), ldr);
  return finish(h, nullptr);
}

int rqr_batched_workspace_bytes(int method, int count, int max_m, int max_n, int max_b, int p, size_t* bytes) {
  if (method != RQR_BATCH_QRCP && method != RQR_BATCH_URV) return -1;
  if (count < 0) return -2;
  if (max_m < 1 || max_m > 1024) return -3;
  if (max_n < 1 || max_n > max_m || max_n > 512) return -4;
  if (max_b < 1 || max_b > 32) return -5;
  if (p < 0 || max_b + p > 64 || (method == RQR_BATCH_URV && p != 0)) return -6;
  if (!bytes) return -7;
  int dev = 0, sms = rqr::kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  *bytes = rqr::batched_workspace_bytes(method, count, max_m, max_n, max_b, p, sms);
  return RQR_OK;
}

int rqr_batched_factor(rqr_handle_t h, int method, int count, const int64_t* desc, const int32_t* order, float* A,
                       float* T, int32_t* perm, float* WV, float* TV, const float* G, int p, int q, uint64_t seed,
                       int max_m, int max_n, int max_b, void* work, size_t lwork, int* info) {
  if (!valid(h)) return -1;
  if (method != RQR_BATCH_QRCP && method != RQR_BATCH_URV) return -2;
  if (count < 0) return -3;
  if (!desc && count > 0) return -4;
  if (!A && count > 0) return -6;
  if (!T && count > 0) return -7;
  if (method == RQR_BATCH_QRCP && !perm && count > 0) return -8;
  if (method == RQR_BATCH_URV && !WV && count > 0) return -9;
  if (method == RQR_BATCH_URV && !TV && count > 0) return -10;
  if (p < 0 || max_b + p > 64 || (method == RQR_BATCH_URV && p != 0)) return -12;
  if (q < 0 || q > 64) return -13;
  if (max_m < 1 || max_m > 1024) return -15;
  if (max_n < 1 || max_n > max_m || max_n > 512) return -16;
  if (max_b < 1 || max_b > 32) return -17;
  if (!work && count > 0) return -18;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return -18;
  cudaGetLastError();
  rqr::Ctx c = make_ctx(h);
  cudaMemsetAsync(h->d_status, 0, sizeof(int), c.stream);
  const int rc = rqr::batched_factor(c, method, count, reinterpret_cast<const long long*>(desc), order, A, T, perm, WV,
                                     TV, G, p, q, seed, max_m, max_n, max_b, work, lwork);
  if (rc != RQR_OK) return rc;
  return finish(h, info);
}

const char* rqr_version(void) { return "rqr-gb300 0.1 (sm_103a)"; }

}  // extern "C"
