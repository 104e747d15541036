// gemm.cu -- dense contractions of the method (sketch Y = G A, trailing
// update A22 <- A22 - V (T^T (V^T A22)), sketch downdate, Gram V^T V).
//
// FP64: the contraction runs on the FP64 matrix pipe with
// mma.sync.m8n8k4.f64 (GB300 has no tcgen05 kind for FP64; its FP64 rate is
// about 1.06 TFLOP/s whether issued as DMMA or DFMA, so the kernel only has to
// keep that pipe busy: 64x64 CTA tiles, 2x2 warps of 32x32, K staged through
// shared memory in steps of 16, several CTAs per SM, split-K when the output
// is too small to fill 152 SMs).
// FP32: register-tiled FFMA kernel of the same tiling.
#include "common.cuh"

namespace rqr {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, PAD = 8;

__device__ __forceinline__ void dmma884(double (&c)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(c[0]), "+d"(c[1])
               : "d"(a), "d"(b));
}

// Loads the BM x BK tile of op(A) starting at (m0, k0) into As[k][i] and the
// BK x BN tile of op(B) at (k0, n0) into Bs[k][j]; out-of-range entries are 0.
template <typename T, bool TA, bool TB, int NT>
__device__ __forceinline__ void load_tiles(T (*As)[BM + PAD], T (*Bs)[BN + PAD], const T* __restrict__ A, int lda,
                                           const T* __restrict__ B, int ldb, int M, int N, int m0, int n0, int k0,
                                           int ke, int tid) {
  constexpr int PER = BM * BK / NT;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int i, k;
    if (!TA) {
      i = tid % BM;
      k = tid / BM + (NT / BM) * q;
    } else {
      k = tid % BK;
      i = tid / BK + (NT / BK) * q;
    }
    const int gi = m0 + i, gk = k0 + k;
    T v = T(0);
    if (gi < M && gk < ke) v = TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda];
    As[k][i] = v;
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    int j, k;
    if (!TB) {
      k = tid % BK;
      j = tid / BK + (NT / BK) * q;
    } else {
      j = tid % BN;
      k = tid / BN + (NT / BN) * q;
    }
    const int gj = n0 + j, gk = k0 + k;
    T v = T(0);
    if (gj < N && gk < ke) v = TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb];
    Bs[k][j] = v;
  }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128) k_dgemm(int M, int N, int K, int kchunk, double alpha,
                                               const double* __restrict__ A, int lda,
                                               const double* __restrict__ B, int ldb, double beta, double* C,
                                               int ldc, double* part) {
  __shared__ double As[BK][BM + PAD];
  __shared__ double Bs[BK][BN + PAD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 1, wn = warp >> 1;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  double acc[4][4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q][0] = acc[r][q][1] = 0.0;

  for (int k0 = kb; k0 < ke; k0 += BK) {
    load_tiles<double, TA, TB, 128>(As, Bs, A, lda, B, ldb, M, N, m0, n0, k0, ke, tid);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < BK / 4; ++s) {
      double a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[s * 4 + t][wm * 32 + r * 8 + g];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[s * 4 + t][wn * 32 + q * 8 + g];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) dmma884(acc[r][q], a[r], b[q]);
    }
    __syncthreads();
  }
  // C fragment: (row g, cols 2t, 2t+1) of each 8x8 sub-tile
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = m0 + wm * 32 + r * 8 + g;
        const int j = n0 + wn * 32 + q * 8 + 2 * t + h;
        if (i < M && j < N) {
          if (part) {
            part[(size_t)blockIdx.z * M * N + i + (size_t)j * M] = acc[r][q][h];
          } else {
            double* cp = C + i + (size_t)j * ldc;
            *cp = beta == 0.0 ? alpha * acc[r][q][h] : alpha * acc[r][q][h] + beta * *cp;
          }
        }
      }
}

// FP32: 256 threads, each computes a 4x4 micro-tile of the 64x64 CTA tile.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, int kchunk, float alpha,
                                               const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float beta, float* C,
                                               int ldc, float* part) {
  __shared__ float As[BK][BM + PAD];
  __shared__ float Bs[BK][BN + PAD];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  float acc[4][4] = {};
  for (int k0 = kb; k0 < ke; k0 += BK) {
    load_tiles<float, TA, TB, 256>(As, Bs, A, lda, B, ldb, M, N, m0, n0, k0, ke, tid);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[k][tx + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = Bs[k][ty + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = fmaf(a[r], b[q], acc[r][q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + tx + 16 * r, j = n0 + ty + 16 * q;
      if (i < M && j < N) {
        if (part) {
          part[(size_t)blockIdx.z * M * N + i + (size_t)j * M] = acc[r][q];
        } else {
          float* cp = C + i + (size_t)j * ldc;
          *cp = beta == 0.f ? alpha * acc[r][q] : alpha * acc[r][q] + beta * *cp;
        }
      }
    }
}

template <typename T>
__global__ void k_splitk_reduce(int M, int N, int S, T alpha, const T* __restrict__ part, T beta, T* C, int ldc) {
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    T s = T(0);
    for (int z = 0; z < S; ++z) s += part[z * MN + e];
    const int i = (int)(e % M), j = (int)(e / M);
    T* cp = C + i + (size_t)j * ldc;
    *cp = beta == T(0) ? alpha * s : alpha * s + beta * *cp;
  }
}

// Split count: enough CTAs for ~3 waves of 152 SMs, at least 128 of K per split.
int choose_splits(int M, int N, int K, int sms, size_t cap) {
  const int tiles = ceil_div(M, BM) * ceil_div(N, BN);
  int s = 1;
  while (tiles * s < 3 * sms && K / (2 * s) >= 128 && (size_t)(2 * s) * M * N <= cap) s *= 2;
  return s;
}

}  // namespace

size_t gemm_part_elems(int M, int N, int K, int sms) {
  const int tiles = ceil_div(M, BM) * ceil_div(N, BN);
  int s = 1;
  while (tiles * s < 3 * sms && K / (2 * s) >= 128) s *= 2;
  return s > 1 ? (size_t)s * M * N : 0;
}

template <typename T>
void gemm(const Ctx& c, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda, const T* B, int ldb,
          T beta, T* C, int ldc, T* part, size_t part_cap) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    // C = beta C
    if (beta == T(0)) {
      set_mat<T>(c, M, N, T(0), C, ldc);
    } else if (beta != T(1)) {
      // scaling through the split-K reduce with S = 0 partials
      const size_t MN = (size_t)M * N;
      int blocks = (int)std::min<size_t>((MN + 255) / 256, (size_t)c.sms * 8);
      k_splitk_reduce<T><<<blocks, 256, 0, c.stream>>>(M, N, 0, alpha, part, beta, C, ldc);
      note_launch(c);
    }
    return;
  }
  const int S = part ? choose_splits(M, N, K, c.sms, part_cap) : 1;
  int kchunk = ceil_div(K, S);
  kchunk = ceil_div(kchunk, BK) * BK;
  const int Sz = ceil_div(K, kchunk);
  dim3 grid(ceil_div(M, BM), ceil_div(N, BN), Sz);
  T* pp = Sz > 1 ? part : nullptr;
  if constexpr (sizeof(T) == 8) {
    auto launch = [&](auto kern) {
      kern<<<grid, 128, 0, c.stream>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, pp);
    };
    if (!ta && !tb) launch(k_dgemm<false, false>);
    else if (ta && !tb) launch(k_dgemm<true, false>);
    else if (!ta && tb) launch(k_dgemm<false, true>);
    else launch(k_dgemm<true, true>);
  } else {
    auto launch = [&](auto kern) {
      kern<<<grid, 256, 0, c.stream>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, pp);
    };
    if (!ta && !tb) launch(k_sgemm<false, false>);
    else if (ta && !tb) launch(k_sgemm<true, false>);
    else if (!ta && tb) launch(k_sgemm<false, true>);
    else launch(k_sgemm<true, true>);
  }
  note_launch(c);
  if (Sz > 1) {
    const size_t MN = (size_t)M * N;
    int blocks = (int)std::min<size_t>((MN + 255) / 256, (size_t)c.sms * 8);
    k_splitk_reduce<T><<<blocks, 256, 0, c.stream>>>(M, N, Sz, alpha, part, beta, C, ldc);
    note_launch(c);
  }
}

template void gemm<double>(const Ctx&, bool, bool, int, int, int, double, const double*, int, const double*, int,
                           double, double*, int, double*, size_t);
template void gemm<float>(const Ctx&, bool, bool, int, int, int, float, const float*, int, const float*, int, float,
                          float*, int, float*, size_t);

}  // namespace rqr
