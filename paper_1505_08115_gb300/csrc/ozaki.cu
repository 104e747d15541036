// ozaki.cu -- FP64-accurate matrix products on the bf16 tensor cores by
// error-free splitting (Ozaki, Ogita, Oishi, "Error-free transformations of
// matrix multiplication by using fast routines of matrix multiplication and
// its applications", Numer. Algorithms 59, 2012; Ootomo, Ozaki, Yokota, IJHPCA
// 2024). Used for the dense contractions of the method (trailing update,
// sketch, sketch downdate) where GB300's FP64 rate (~1.06 TFLOP/s) is the
// bound.
//
// Scheme. Row i of op(A) is scaled by 2^-e_i with |a_ik| < 2^e_i, column j of
// op(B) by 2^-f_j; each scaled value becomes 8 signed 7-bit digits
//   a_ik = 2^e_i * sum_p d_p(a_ik) 2^(-7p),   |d_p| <= 127,  p = 1..8
// (56 bits, three more than FP64 carries; the digits are taken from the FP64
// bit pattern with integer shifts). Then
//   (AB)_ij = 2^(e_i + f_j) * sum_g 2^(-7g) S_g(i,j),
//   S_g = sum_k sum_{p+q=g} d_p(a_ik) d_q(b_kj),   g = 2..9 (36 pairs p+q <= 9).
// Digits are exact in bf16; every product d_p d_q <= 127^2 is exact, and over
// a K chunk of 128 a group holds at most 8 pairs: |S_g| <= 8*128*127^2 < 2^24,
// so the tensor core's FP32 accumulation of a group is exact. After each
// chunk the eight group sums are added exactly into two 64-bit integer
// accumulators (shifted by their relative scales), converted to FP64 once at
// the end; the dropped pairs (p+q >= 10) and digits (below 2^-56 of the
// row/column maximum) are far below FP64 rounding for the norm-wise error of
// the product.
//
// Kernel. CTA tile 64 x 32, eight warps of 16 x 16, K staged 32 at a time:
// the FP64 tiles are loaded, split into digits and stored as bf16 slices
// (k contiguous, rows padded to 40 for conflict-free fragment loads); each warp
// keeps its eight A-slice fragments in registers and runs the 36 pairs x 2
// n8 tiles = 72 mma.sync.m16n8k16 per k16 step into eight FP32 group
// accumulators; the integer accumulators live in shared memory.
#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"

namespace rqr {

namespace {

constexpr int OBM = 64, OBN = 32, OBK = 32, OKP = 40, ONS = 8, OKC = 128, OT = 256;

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Scale exponent e with |x| < 2^e for every x of a row whose largest
// magnitude has biased exponent emax (0 for an all-zero row).
__device__ __forceinline__ int scale_exp(int emax) { return emax == 0 ? -1022 : emax - 1022; }

// 56-bit magnitude N = trunc(|x| 2^(56-e)) from the bit pattern (|x| < 2^e).
__device__ __forceinline__ unsigned long long fixed56(double x, int e, bool& neg) {
  const long long bits = __double_as_longlong(x);
  neg = bits < 0;
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0) return 0ull;
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1019 - e;
  if (sh >= 0) return mant << sh;  // sh <= 3 because |x| < 2^e
  if (sh <= -64) return 0ull;
  return mant >> (-sh);
}

__device__ __forceinline__ void store_digits(__nv_bfloat16* base, size_t stride, double x, int e) {
  bool neg;
  const unsigned long long N = fixed56(x, e, neg);
#pragma unroll
  for (int p = 0; p < ONS; ++p) {
    const int d = (int)((N >> (49 - 7 * p)) & 127ull);
    base[p * stride] = __float2bfloat16_rn(neg ? -(float)d : (float)d);
  }
}

// Biased exponent of the largest |value| along rows (dir = 0: of op(A), over k)
// or columns (of op(B)). One warp per row/column.
__device__ __forceinline__ int biased_exp(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7ff); }

template <bool TA>
__global__ void k_row_exp(int M, int K, const double* __restrict__ A, int lda, int* ea) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= M) return;
  int emax = 0;
  for (int k = lane; k < K; k += 32) {
    const double v = TA ? A[k + (size_t)i * lda] : A[i + (size_t)k * lda];
    emax = max(emax, biased_exp(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if (lane == 0) ea[i] = scale_exp(emax);
}

// Column scale of op(A) read column-major when !TA: threads over rows instead.
__global__ void k_row_exp_colmajor(int M, int K, const double* __restrict__ A, int lda, int* ea) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  int emax = 0;
  for (int k = 0; k < K; ++k) emax = max(emax, biased_exp(A[i + (size_t)k * lda]));
  ea[i] = scale_exp(emax);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(OT, 2) k_ozgemm(int M, int N, int K, int kchunk, double alpha,
                                                   const double* __restrict__ A, int lda,
                                                   const double* __restrict__ B, int ldb, double beta, double* C,
                                                   int ldc, const int* __restrict__ ea, const int* __restrict__ eb,
                                                   double* part) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);          // [ONS][OBM][OKP]
  __nv_bfloat16* Bs = As + ONS * OBM * OKP;                             // [ONS][OBN][OKP]
  long long* accH = reinterpret_cast<long long*>(Bs + ONS * OBN * OKP);  // [OBN][OBM]
  long long* accL = accH + OBM * OBN;                                     // [OBN][OBM]
  __shared__ int sea[OBM], seb[OBN];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int wm = warp & 3, wn = warp >> 2;
  const int m0 = blockIdx.x * OBM, n0 = blockIdx.y * OBN;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  for (int e = tid; e < OBM * OBN; e += OT) accH[e] = accL[e] = 0;
  if (tid < OBM) sea[tid] = (m0 + tid < M) ? ea[m0 + tid] : 0;
  if (tid < OBN) seb[tid] = (n0 + tid < N) ? eb[n0 + tid] : 0;
  float S[8][2][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 4; ++c) S[a][b][c] = 0.f;
  __syncthreads();
  int kin = 0;  // K consumed since the last flush
  for (int k0 = kb; k0 < ke; k0 += OBK) {
    // ---- stage and split the FP64 tiles
#pragma unroll
    for (int q = 0; q < OBM * OBK / OT; ++q) {
      int i, k;
      if (!TA) {
        i = tid % OBM;
        k = tid / OBM + (OT / OBM) * q;
      } else {
        k = tid % OBK;
        i = tid / OBK + (OT / OBK) * q;
      }
      const int gi = m0 + i, gk = k0 + k;
      double v = 0.0;
      if (gi < M && gk < ke) v = TA ? A[gk + (size_t)gi * lda] : A[gi + (size_t)gk * lda];
      store_digits(As + i * OKP + k, (size_t)OBM * OKP, v, sea[i]);
    }
#pragma unroll
    for (int q = 0; q < OBN * OBK / OT; ++q) {
      int j, k;
      if (!TB) {
        k = tid % OBK;
        j = tid / OBK + (OT / OBK) * q;
      } else {
        j = tid % OBN;
        k = tid / OBN + (OT / OBN) * q;
      }
      const int gj = n0 + j, gk = k0 + k;
      double v = 0.0;
      if (gj < N && gk < ke) v = TB ? B[gj + (size_t)gk * ldb] : B[gk + (size_t)gj * ldb];
      store_digits(Bs + j * OKP + k, (size_t)OBN * OKP, v, seb[j]);
    }
    __syncthreads();
    // ---- 36 digit pairs per k16 step
#pragma unroll
    for (int kk = 0; kk < OBK; kk += 16) {
      uint32_t af[ONS][4];
#pragma unroll
      for (int p = 0; p < ONS; ++p) {
        const __nv_bfloat16* ap = As + p * OBM * OKP + (wm * 16) * OKP + kk;
        af[p][0] = *reinterpret_cast<const uint32_t*>(ap + g * OKP + 2 * t);
        af[p][1] = *reinterpret_cast<const uint32_t*>(ap + (g + 8) * OKP + 2 * t);
        af[p][2] = *reinterpret_cast<const uint32_t*>(ap + g * OKP + 2 * t + 8);
        af[p][3] = *reinterpret_cast<const uint32_t*>(ap + (g + 8) * OKP + 2 * t + 8);
      }
#pragma unroll
      for (int q = 0; q < ONS; ++q) {
        uint32_t bf[2][2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const __nv_bfloat16* bp = Bs + q * OBN * OKP + (wn * 16 + h * 8 + g) * OKP + kk;
          bf[h][0] = *reinterpret_cast<const uint32_t*>(bp + 2 * t);
          bf[h][1] = *reinterpret_cast<const uint32_t*>(bp + 2 * t + 8);
        }
#pragma unroll
        for (int p = 0; p < ONS; ++p) {
          if (p + q <= ONS - 1) {  // digit indices p+1, q+1 with (p+1)+(q+1) <= 9
            mma_bf16(S[p + q][0], af[p], bf[0][0], bf[0][1]);
            mma_bf16(S[p + q][1], af[p], bf[1][0], bf[1][1]);
          }
        }
      }
    }
    __syncthreads();
    kin += OBK;
    if (kin >= OKC || k0 + OBK >= ke) {
      // flush the exact group sums (integers below 2^24) into two 64-bit
      // integer accumulators: H collects groups a = 0..3 (scale 2^(-7(a+2)))
      // as sum S_a 2^(7(3-a)), L groups 4..7 as sum S_a 2^(7(7-a)); so
      // H 2^-35 + L 2^-63 is the chunk's value, and no rounding happens before
      // the final conversion
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int r = wm * 16 + g + (c >> 1) * 8;
          const int col = wn * 16 + h * 8 + 2 * t + (c & 1);
          long long hi = 0, lo = 0;
#pragma unroll
          for (int a = 0; a < 4; ++a) hi += (long long)__float2int_rn(S[a][h][c]) << (7 * (3 - a));
#pragma unroll
          for (int a = 4; a < 8; ++a) lo += (long long)__float2int_rn(S[a][h][c]) << (7 * (7 - a));
          accH[col * OBM + r] += hi;
          accL[col * OBM + r] += lo;
#pragma unroll
          for (int a = 0; a < 8; ++a) S[a][h][c] = 0.f;
        }
      kin = 0;
    }
  }
  __syncthreads();
  for (int e = tid; e < OBM * OBN; e += OT) {
    const int r = e % OBM, col = e / OBM;
    const int i = m0 + r, j = n0 + col;
    if (i < M && j < N) {
      const double v =
          ldexp(fma((double)accH[col * OBM + r], 0x1p-35, (double)accL[col * OBM + r] * 0x1p-63), sea[r] + seb[col]);
      if (part) {
        part[(size_t)blockIdx.z * M * N + i + (size_t)j * M] = v;
      } else {
        double* cp = C + i + (size_t)j * ldc;
        *cp = beta == 0.0 ? alpha * v : alpha * v + beta * *cp;
      }
    }
  }
}

__global__ void k_ozreduce(int M, int N, int S, double alpha, const double* __restrict__ part, double beta, double* C,
                           int ldc) {
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int z = 0; z < S; ++z) s += part[z * MN + e];
    const int i = (int)(e % M), j = (int)(e / M);
    double* cp = C + i + (size_t)j * ldc;
    *cp = beta == 0.0 ? alpha * s : alpha * s + beta * *cp;
  }
}

constexpr size_t kOzSmem = sizeof(__nv_bfloat16) * ONS * (OBM + OBN) * OKP + 2 * sizeof(long long) * OBM * OBN;

}  // namespace

size_t ozaki_scratch_elems(int M, int N) { return (size_t)M + N + 64; }

// C = alpha op(A) op(B) + beta C with FP64 accuracy on the bf16 tensor cores.
// iscr: M + N ints of scratch for the scale exponents; part/part_cap as gemm().
void gemm_f64x(const Ctx& c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
               const double* B, int ldb, double beta, double* C, int ldc, int* iscr, double* part, size_t part_cap) {
  if (M <= 0 || N <= 0) return;
  if (K <= 0) {
    gemm<double>(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, part, part_cap);
    return;
  }
  int* ea = iscr;
  int* eb = iscr + M;
  // scales: rows of op(A) over K, columns of op(B) over K
  if (ta) k_row_exp<true><<<ceil_div(M, 8), 256, 0, c.stream>>>(M, K, A, lda, ea);
  else k_row_exp_colmajor<<<ceil_div(M, 128), 128, 0, c.stream>>>(M, K, A, lda, ea);
  if (!tb) k_row_exp<true><<<ceil_div(N, 8), 256, 0, c.stream>>>(N, K, B, ldb, eb);
  else k_row_exp_colmajor<<<ceil_div(N, 128), 128, 0, c.stream>>>(N, K, B, ldb, eb);
  note_launch(c, 2);
  const int tiles = ceil_div(M, OBM) * ceil_div(N, OBN);
  int S = 1;
  while (part && tiles * S < 2 * c.sms && K / (2 * S) >= 256 && (size_t)(2 * S) * M * N <= part_cap) S *= 2;
  int kchunk = ceil_div(ceil_div(K, S), OKC) * OKC;
  const int Sz = ceil_div(K, kchunk);
  dim3 grid(ceil_div(M, OBM), ceil_div(N, OBN), Sz);
  double* pp = Sz > 1 ? part : nullptr;
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOzSmem);
    kern<<<grid, OT, kOzSmem, c.stream>>>(M, N, K, kchunk, alpha, A, lda, B, ldb, beta, C, ldc, ea, eb, pp);
  };
  if (!ta && !tb) launch(k_ozgemm<false, false>);
  else if (ta && !tb) launch(k_ozgemm<true, false>);
  else if (!ta && tb) launch(k_ozgemm<false, true>);
  else launch(k_ozgemm<true, true>);
  note_launch(c);
  if (Sz > 1) {
    const size_t MN = (size_t)M * N;
    const int blocks = (int)std::min<size_t>((MN + 255) / 256, (size_t)c.sms * 8);
    k_ozreduce<<<blocks, 256, 0, c.stream>>>(M, N, Sz, alpha, part, beta, C, ldc);
    note_launch(c);
  }
}

}  // namespace rqr
