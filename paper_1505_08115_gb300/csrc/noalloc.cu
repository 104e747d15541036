// noalloc.cu -- rqr_form_q_noalloc: forming Q from the block reflectors
// without any caller-provided workspace.
//
// Who needs this: code that runs where it cannot allocate device memory --
// inside a CUDA-graph capture that must not call cudaMalloc, from a
// real-time or signal-safe context, or a host plugin whose host application
// owns every allocation and hands out only the input and output buffers. Such
// callers can still pass A/F, T and Q; the scratch that the regular
// rqr_form_q takes from `work` lives here in one file-scope device array.
//
// The array is static device memory of every GPU that loads this library, and
// stays resident until the process exits. Its size bounds the problems this
// entry point accepts (RQR_FORM_Q_NOALLOC_MAX_BYTES); larger ones get
// RQR_ERR_SIZE. All calls share the array: two calls whose work overlaps on
// the GPU (different streams, or different handles on one device) race on it.
// Every value the kernels read from it is written earlier in the same call, so
// nothing needs clearing between calls.
//
// Set-up: host code cannot use the array's name as a device address (in host
// code it is a stand-in object). The first call with a handle of a given
// device looks up that device's copy of the array with cudaGetSymbolAddress,
// with the handle's device made current for the lookup (the caller's current
// device is restored afterwards), and caches it per device; that first call
// therefore must not happen while the stream is being captured into a CUDA
// graph. The cache assumes the device's primary context lives as long as the
// process: after cudaDeviceReset the cached address is stale, so a process
// that resets a device must not call this entry point on it again.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"


namespace {

constexpr size_t kNoAllocScratchBytes = RQR_FORM_Q_NOALLOC_MAX_BYTES;  // 8 MiB per device
constexpr size_t kScratchDoubles = kNoAllocScratchBytes / sizeof(double);

static __device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the static scratch on device `dev` (the handle's device,
// whose stream runs the kernels), looked up once per device with that device
// current; the caller's current device is restored.
int scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return RQR_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) {
      cudaGetLastError();
      return RQR_ERR_CUDA;
    }
    if (cur != dev && cudaSetDevice(dev) != cudaSuccess) {
      cudaGetLastError();
      return RQR_ERR_CUDA;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (cur != dev) cudaSetDevice(cur);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return RQR_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return RQR_OK;
}

size_t round256(size_t elems, size_t esz) { return ((elems * esz + 255) / 256) * 256; }

// Scratch layout (bytes): Vx (m x b), W (b x ncols), W2 (b x ncols), split-K partials.
template <typename T>
bool layout(int m, int b, int ncols, size_t& off_w, size_t& off_w2, size_t& off_part, size_t& part_cap) {
  const size_t vx = round256((size_t)std::max(m, 1) * b, sizeof(T));
  const size_t wv = round256((size_t)b * std::max(ncols, 1), sizeof(T));
  off_w = vx;
  off_w2 = vx + wv;
  off_part = vx + 2 * wv;
  if (off_part > kNoAllocScratchBytes) return false;
  part_cap = (kNoAllocScratchBytes - off_part) / sizeof(T);
  return true;
}

template <typename T>
int form_q_static(rqr::Ctx c, int m, int n, int b, const T* F, int ldf, const T* Tm, int ldt, T* Q, int ldq,
                  int ncols, char* base) {
  using namespace rqr;
  size_t ow, ow2, op, cap;
  if (!layout<T>(m, b, ncols, ow, ow2, op, cap)) return RQR_ERR_SIZE;
  T* Vx = reinterpret_cast<T*>(base);
  T* W = reinterpret_cast<T*>(base + ow);
  T* W2 = reinterpret_cast<T*>(base + ow2);
  T* part = reinterpret_cast<T*>(base + op);
  set_mat<T>(c, m, ncols, T(0), Q, ldq);
  set_mat<T>(c, 1, std::min(m, ncols), T(1), Q, ldq + 1);
  if (n == 0) return RQR_OK;
  // Q = Q_0 Q_1 ... applied to [I; 0], last block first; block i starts at i*b
  for (int i = (n - 1) / b; i >= 0; --i) {
    const int k0 = i * b, kb = std::min(b, n - k0), mp = m - k0;
    make_vx<T>(c, mp, kb, F + k0 + (size_t)k0 * ldf, ldf, Vx, mp);
    T* Qk = Q + k0;
    gemm<T>(c, true, false, kb, ncols, mp, T(1), Vx, mp, Qk, ldq, T(0), W, kb, part, cap);
    gemm<T>(c, false, false, kb, ncols, kb, T(1), Tm + (size_t)k0 * ldt, ldt, W, kb, T(0), W2, kb, part, cap);
    gemm<T>(c, false, false, mp, ncols, kb, T(-1), Vx, mp, W2, kb, T(1), Qk, ldq, part, cap);
  }
  return RQR_OK;
}

}  // namespace

extern "C" {

int rqr_form_q_noalloc(rqr_handle_t h, int m, int n, int b, const void* F, int ldf, const void* T, int ldt, void* Q,
                       int ldq, int ncols, int prec) {
  rqr::Ctx c{};
  if (!rqr::handle_ctx(h, &c)) return -1;
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
  size_t ow, ow2, op, cap;
  const bool fits = prec == RQR_FP64 ? layout<double>(m, b, ncols, ow, ow2, op, cap)
                                     : layout<float>(m, b, ncols, ow, ow2, op, cap);
  if (!fits) return RQR_ERR_SIZE;
  void* base = nullptr;
  const int rc = scratch_address(c.device, &base);
  if (rc != RQR_OK) return rc;
  cudaGetLastError();
  const int st = prec == RQR_FP64
                     ? form_q_static<double>(c, m, n, b, static_cast<const double*>(F), ldf,
                                             static_cast<const double*>(T), ldt, static_cast<double*>(Q), ldq, ncols,
                                             static_cast<char*>(base))
                     : form_q_static<float>(c, m, n, b, static_cast<const float*>(F), ldf,
                                            static_cast<const float*>(T), ldt, static_cast<float*>(Q), ldq, ncols,
                                            static_cast<char*>(base));
  if (st != RQR_OK) return st;
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();
    return RQR_ERR_CUDA;
  }
  return RQR_OK;
}

}  // extern "C"
