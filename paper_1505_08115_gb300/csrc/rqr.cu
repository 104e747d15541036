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
  RqrProfile prof;
};

namespace {

constexpr unsigned kMagic = 0x52515231u;  // "RQR1"

bool valid(rqr_handle_t h) { return h && h->magic == kMagic; }

rqr::Ctx make_ctx(rqr_handle_t h) { return rqr::Ctx{h->stream, h->sms, h->d_status, &h->nlaunch}; }

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
  int *picks, *imap;
  size_t part_cap;
};

template <typename T>
size_t carve_rqrcp(rqr::Carver& cv, int m, int n, int b, int p, int sms, RqrcpWs<T>& w) {
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
               int ldt, int32_t* perm, int sketch, void* work, size_t lwork, int* info) {
  using namespace rqr;
  const int l = b + p;
  Carver cv{static_cast<char*>(work), lwork, 0, false};
  RqrcpWs<T> w;
  carve_rqrcp<T>(cv, m, n, b, p, h->sms, w);
  if (!cv.ok()) return RQR_ERR_WORKSPACE;
  Ctx c = make_ctx(h);
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
      gemm<T>(c, false, false, l, n, m, T(1), w.Gc, l, A, lda, T(0), w.Y, l, w.part, w.part_cap);
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
      gemm<T>(c, false, false, l, np, mp, T(1), Gi, l, P, lda, T(0), w.Y + (size_t)k0 * l, l, w.part, w.part_cap);
    }
    // (b) pivots from the sketch, (c) swaps
    {
      Phase ph(h, RQR_PHASE_PIVOT, 4.0 * l * b * (double)np);
      ypick<T>(c, l, np, b, w.Y + (size_t)k0 * l, l, w.picks, w.yscr);
    }
    {
      Phase ph(h, RQR_PHASE_SWAP, 0.0);
      apply_swaps<T>(c, b, w.picks, m, A, lda, k0, l, down ? w.Y : nullptr, l, k0, perm, w.swp, w.imap);
    }
    // (d) panel QR + T
    {
      Phase ph(h, RQR_PHASE_PANEL, 2.0 * mp * (double)b * b - 2.0 * b * (double)b * b / 3.0);
      panel_qr<T>(c, mp, b, P, lda, w.tau, w.pscr);
      make_vx<T>(c, mp, b, P, lda, w.Vx, mp);
      gemm<T>(c, true, false, b, b, mp, T(1), w.Vx, mp, w.Vx, mp, T(0), w.gram, b, w.part, w.part_cap);
      larft_tri<T>(c, b, w.gram, b, w.tau, Tb, ldt);
    }
    // (e) trailing update
    const int n2 = np - b;
    T* A2 = A + k0 + (size_t)(k0 + b) * lda;
    {
      Phase ph(h, RQR_PHASE_UPDATE, 4.0 * mp * (double)n2 * b);
      gemm<T>(c, true, false, b, n2, mp, T(1), w.Vx, mp, A2, lda, T(0), w.W, b, w.part, w.part_cap);
      gemm<T>(c, true, false, b, n2, b, T(1), Tb, ldt, w.W, b, T(0), w.W2, b, w.part, w.part_cap);
      gemm<T>(c, false, false, mp, n2, b, T(-1), w.Vx, mp, w.W2, b, T(1), A2, lda, w.part, w.part_cap);
    }
    if (down) {
      Phase ph(h, RQR_PHASE_DOWNDATE, 4.0 * l * mp * (double)b + 2.0 * l * b * (double)n2);
      T* Gk = w.Gc + (size_t)k0 * l;
      gemm<T>(c, false, false, l, b, mp, T(1), Gk, l, w.Vx, mp, T(0), w.GV, l, w.part, w.part_cap);
      gemm<T>(c, false, false, l, b, b, T(1), w.GV, l, Tb, ldt, T(0), w.GVT, l, w.part, w.part_cap);
      gemm<T>(c, false, true, l, mp, b, T(-1), w.GVT, l, w.Vx, mp, T(1), Gk, l, w.part, w.part_cap);
      gemm<T>(c, false, false, l, n2, b, T(-1), Gk, l, A + k0 + (size_t)(k0 + b) * lda, lda, T(1),
              w.Y + (size_t)(k0 + b) * l, l, w.part, w.part_cap);
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

}  // namespace

extern "C" {

int rqr_create(rqr_handle_t* h, void* stream) {
  if (!h) return -1;
  *h = nullptr;
  rqr_handle_s* s = new (std::nothrow) rqr_handle_s();
  if (!s) return RQR_ERR_CUDA;
  s->magic = kMagic;
  s->nlaunch = 0;
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
  h->magic = 0;
  delete h;
  return RQR_OK;
}

int rqr_set_stream(rqr_handle_t h, void* stream) {
  if (!valid(h)) return RQR_ERR_HANDLE;
  h->stream = static_cast<cudaStream_t>(stream);
  return RQR_OK;
}

int rqr_workspace_bytes(int m, int n, int b, int p, int q, int prec, int sketch, size_t* bytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (b < 1 || b > 512) return -3;
  if (p < 0) return -4;
  if (prec != RQR_FP64 && prec != RQR_FP32) return -6;
  if (sketch != RQR_SKETCH_DOWNDATE && sketch != RQR_SKETCH_RESAMPLE) return -7;
  if (!bytes) return -8;
  int dev = 0, sms = rqr::kNumSMs;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  rqr::Carver cv{nullptr, 0, 0, true};
  if (prec == RQR_FP64) {
    RqrcpWs<double> w;
    carve_rqrcp<double>(cv, m, n, b, p, sms, w);
  } else {
    RqrcpWs<float> w;
    carve_rqrcp<float>(cv, m, n, b, p, sms, w);
  }
  (void)q;
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
  if (prec != RQR_FP64 && prec != RQR_FP32) return -14;
  if (sketch != RQR_SKETCH_DOWNDATE && sketch != RQR_SKETCH_RESAMPLE) return -15;
  if (!work && n > 0) return -16;
  if (reinterpret_cast<uintptr_t>(work) % 256 != 0) return -16;
  cudaGetLastError();
  if (prec == RQR_FP64)
    return rqrcp_impl<double>(h, m, n, static_cast<double*>(A), lda, b, p, seed, static_cast<const double*>(G), ldg,
                              static_cast<double*>(T), ldt, perm, sketch, work, lwork, info);
  return rqrcp_impl<float>(h, m, n, static_cast<float*>(A), lda, b, p, seed, static_cast<const float*>(G), ldg,
                           static_cast<float*>(T), ldt, perm, sketch, work, lwork, info);
}

int rurv_factor(rqr_handle_t h, int m, int n, void* A, int lda, int b, int p, int q, int k, uint64_t seed,
                const void* G, void* TU, int ldtu, void* WV, int ldwv, void* TV, int ldtv, int prec, void* work,
                size_t lwork, int* info) {
  (void)h; (void)m; (void)n; (void)A; (void)lda; (void)b; (void)p; (void)q; (void)k; (void)seed; (void)G;
  (void)TU; (void)ldtu; (void)WV; (void)ldwv; (void)TV; (void)ldtv; (void)prec; (void)work; (void)lwork;
  if (info) *info = RQR_ERR_UNSUPPORTED;
  return RQR_ERR_UNSUPPORTED;
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

const char* rqr_version(void) { return "rqr-gb300 0.1 (sm_103a)"; }

}  // extern "C"
