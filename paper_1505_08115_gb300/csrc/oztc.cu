// oztc.cu -- FP64-accurate matrix products on the fifth-generation tensor
// cores of sm_103a (tcgen05.mma with TMEM accumulators, operands staged by
// TMA). Same error-free splitting as ozaki.cu (Ozaki, Ogita, Oishi 2012;
// Ootomo, Ozaki, Yokota 2024), laid out for the tcgen05 pipeline:
//
// 1. Splitting (k_split_*). Row r of op(A) (or of op(B)^T) is scaled by 2^-e_r,
//    |x| < 2^e_r, and becomes 8 signed 7-bit digits d_p, p = 0..7,
//      x = 2^(e_r - 7) sum_p d_p 2^(-7p).
//    Plane p stores d_p 2^(-7p) in bf16 (exact: at most 7 significant bits),
//    K-contiguous: planes[p][r][k], row stride kld.
// 2. Products (k_oztc). A 128 x 64 output tile, K consumed 16 at a time.
//    For each k16 step all 36 digit pairs p + q <= 7 are multiplied into
//    eight TMEM slots of 64 columns, slot a = p + q. Since the B planes sit
//    next to each other in shared memory and the slots next to each other in
//    TMEM, the pairs (p, q0..q0+3) are ONE tcgen05.mma.kind::f16 with M = 128,
//    N = 256 (A plane p against B planes q0..q0+3 into slots p+q0..p+q0+3):
//    12 MMAs per k16 step, and each A plane is read from shared memory 1 or 2
//    times instead of 8 - p. Pairs of slot a carry the common factor 2^(-7a);
//    with |d| <= 127 and at most a + 1 pairs per slot, a slot's sum over a
//    window of 128 K is below (a + 1) 128 127^2 2^(-7a) < 2^(24 - 7a), so every
//    slot holds an exact integer S_a 2^(-7a) in FP32.
// 3. Drain (epilogue warps), once per window of 128 K: slots 0..5 are
//    converted to integers, paired in 32 bits (S_2k 2^7 + S_2k+1 < 2^31) and
//    added into H = sum_{a<=5} S_a 2^(7(5-a))
//    (int64; below 2^57 per window, at most 64 windows per tile), slots 6 and 7
//    (weights 2^-42 and below relative to the leading term) into a float M6,
//    whose rounding stays below 2^-58 of the product's scale. At the end of
//    the tile the value
//      (AB)_ij = 2^(e_i + f_j - 63) (H 2^14 + M6 2^49)
//    is rounded once to FP64 with integer operations (GB300 runs FP64 at
//    about two operations per clock per SM, so the epilogue avoids FP64
//    conversions) and combined with C by one FP64 add or multiply-add.
//
// Warp roles of the persistent kernel (one CTA per SM, 576 threads):
// warps 0-15 drain TMEM (warp w: lanes 32 (w % 4).., columns 16 (w / 4)..),
// warp 16 issues TMA loads (one 3-D box per operand per stage: 8 planes x rows x 16 K),
// warp 17 allocates TMEM and issues the MMAs from one thread.
// Every wait is bounded (about two seconds); on a timeout the kernel records
// RQR_ERR_TIMEOUT, lets its in-flight copies and MMAs finish, frees TMEM
// and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace rqr {

namespace {

using namespace tcp;

constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 16, TC_ND = 8, TC_NS = 4, TC_WIN = 8;
// 18 warps: 16 epilogue warps (4 per TMEM lane quadrant, 16 columns each),
// one TMA producer warp, one MMA warp.
constexpr int TC_EPI_WARPS = 16, TC_PROD_WARP = 16, TC_MMA_WARP = 17, TC_THREADS = 576;
constexpr int TC_EPI_COLS = TC_BN / (TC_EPI_WARPS / 4);  // 16 columns per epilogue warp
constexpr int TC_CCH = 4;                                 // C values loaded together in the epilogue
constexpr uint32_t TC_A_BYTES = TC_ND * TC_BM * TC_BK * 2;    // 32 KB
constexpr uint32_t TC_B_BYTES = TC_ND * TC_BN * TC_BK * 2;    // 16 KB
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;  // 48 KB
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr size_t TC_SMEM = (size_t)TC_NS * TC_STAGE_BYTES + 1024 + 256;

// Instruction descriptor of kind::f16: bf16 x bf16 -> FP32, A and B K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

// ------------------------------------------------------------------ digits
// Scale exponent e with |x| < 2^e for every x of a row whose largest
// magnitude has biased exponent emax (an all-zero row gets the smallest).
__device__ __forceinline__ int scale_exp_tc(int emax) { return emax == 0 ? -1022 : emax - 1022; }

// 56-bit magnitude trunc(|x| 2^(56-e)) from the bit pattern (|x| < 2^e).
__device__ __forceinline__ unsigned long long fixed56_tc(double x, int e, bool& neg) {
  const long long bits = __double_as_longlong(x);
  neg = bits < 0;
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0) return 0ull;
  const unsigned long long mant = (bits & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1019 - e;
  if (sh >= 0) return mant << sh;
  if (sh <= -64) return 0ull;
  return mant >> (-sh);
}

// bf16 bit pattern of +-d 2^(-7p) for an integer digit 0 <= d <= 127.
__device__ __forceinline__ uint32_t digit_bf16(unsigned d, int p, bool neg) {
  const float f = (__uint_as_float(0x4B000000u | d) - 8388608.0f) * __uint_as_float((uint32_t)(127 - 7 * p) << 23);
  return (__float_as_uint(f) >> 16) | (neg ? 0x8000u : 0u);
}

__device__ __forceinline__ void store_digit_pair(uint32_t* planes, size_t pstride, size_t off, double x0, double x1,
                                                 int e) {
  bool n0, n1;
  const unsigned long long N0 = fixed56_tc(x0, e, n0), N1 = fixed56_tc(x1, e, n1);
#pragma unroll
  for (int p = 0; p < TC_ND; ++p) {
    const unsigned d0 = (unsigned)((N0 >> (49 - 7 * p)) & 127ull);
    const unsigned d1 = (unsigned)((N1 >> (49 - 7 * p)) & 127ull);
    planes[p * pstride + off] = digit_bf16(d0, p, n0) | (digit_bf16(d1, p, n1) << 16);
  }
}

__device__ __forceinline__ int biased_exp_tc(double v) { return (int)((__double_as_longlong(v) >> 52) & 0x7ff); }

// Largest biased exponent of each row r of the R x K operand X, where
// element (r, k) sits at X[k + r ld] (contig) or X[r + k ld] (!contig).
// emax must be zeroed before; blocks cover rows x K-chunks and combine with atomicMax.
template <bool CONTIG>
__global__ void k_plane_exp(int R, int K, int kchunk, const double* __restrict__ X, int ld, int* emax) {
  const int k0 = blockIdx.y * kchunk, k1 = min(K, k0 + kchunk);
  if (CONTIG) {
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= R) return;
    int e = 0;
    for (int k = k0 + lane; k < k1; k += 32) e = max(e, biased_exp_tc(X[k + (size_t)r * ld]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0 && e > 0) atomicMax(emax + r, e);
  } else {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    int e = 0;
    for (int k = k0; k < k1; ++k) e = max(e, biased_exp_tc(X[r + (size_t)k * ld]));
    if (e > 0) atomicMax(emax + r, e);
  }
}

// Digit planes of rows with contiguous K: one warp per row, two K per lane.
__global__ void k_split_contig(int R, int K, const double* __restrict__ X, int ld, const int* __restrict__ emax,
                               uint32_t* planes, int kld) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= R) return;
  const int e = scale_exp_tc(emax[r]);
  const size_t pstride = (size_t)R * kld / 2;
  const double* x = X + (size_t)r * ld;
  for (int k = 2 * lane; k < K; k += 64) {
    const double x0 = x[k];
    const double x1 = k + 1 < K ? x[k + 1] : 0.0;
    store_digit_pair(planes, pstride, ((size_t)r * kld + k) / 2, x0, x1, e);
  }
}

// Digit planes of long contiguous rows (element (r, k) at X[k + r ld]) with
// the row exponent computed in the same launch: one CTA per row, a first pass
// for the largest exponent (block max), a second pass (served mostly from L2)
// that writes the digits; four 16-byte loads in flight per thread.
constexpr int SPLIT_T = 256;
__global__ void __launch_bounds__(SPLIT_T) k_split_rows(int R, int K, const double* __restrict__ X, int ld,
                                                        int* emax_out, uint32_t* planes, int kld) {
  __shared__ int wmax[SPLIT_T / 32];
  const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double* x = X + (size_t)r * ld;
  // pass 1: largest biased exponent of the row
  int e = 0;
  const bool al16 = ((reinterpret_cast<uintptr_t>(x) & 15) == 0);
  if (al16) {
    const double2* x2 = reinterpret_cast<const double2*>(x);
    const int K2 = K / 2;
    for (int k = tid; k < K2; k += 4 * SPLIT_T) {
      double2 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = (k + u * SPLIT_T < K2) ? x2[k + u * SPLIT_T] : make_double2(0.0, 0.0);
#pragma unroll
      for (int u = 0; u < 4; ++u) e = max(e, max(biased_exp_tc(v[u].x), biased_exp_tc(v[u].y)));
    }
    if ((K & 1) && tid == 0) e = max(e, biased_exp_tc(x[K - 1]));
  } else {
    for (int k = tid; k < K; k += SPLIT_T) e = max(e, biased_exp_tc(x[k]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (lane == 0) wmax[warp] = e;
  __syncthreads();
  int emx = 0;
#pragma unroll
  for (int w = 0; w < SPLIT_T / 32; ++w) emx = max(emx, wmax[w]);
  if (tid == 0) emax_out[r] = emx;
  const int sc = scale_exp_tc(emx);
  // pass 2: digits, two values per thread and step (one 32-bit word per plane)
  const size_t pstride = (size_t)R * kld / 2;
  const size_t rbase = (size_t)r * kld / 2;
  for (int kp = tid; 2 * kp < K; kp += 2 * SPLIT_T) {
    double a0[2], a1[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int k = 2 * (kp + u * SPLIT_T);
      a0[u] = k < K ? x[k] : 0.0;
      a1[u] = k + 1 < K ? x[k + 1] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int k = 2 * (kp + u * SPLIT_T);
      if (k < K) store_digit_pair(planes, pstride, rbase + k / 2, a0[u], a1[u], sc);
    }
  }
}

// Digit planes of rows stored with stride (element (r, k) at X[r + k ld]):
// 32 x 64 tiles transposed through shared memory.
__global__ void __launch_bounds__(256) k_split_strided(int R, int K, const double* __restrict__ X, int ld,
                                                        const int* __restrict__ emax, uint32_t* planes, int kld) {
  __shared__ double tile[64][33];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + (t & 31), k = k0 + (t >> 5) + 8 * i;
    tile[(t >> 5) + 8 * i][t & 31] = (r < R && k < K) ? X[r + (size_t)k * ld] : 0.0;
  }
  __syncthreads();
  const int rr = t >> 3, r = r0 + rr;
  if (r >= R) return;
  const int e = scale_exp_tc(emax[r]);
  const size_t pstride = (size_t)R * kld / 2;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int kp = (t & 7) + 8 * j, k = k0 + 2 * kp;
    if (k < K) store_digit_pair(planes, pstride, ((size_t)r * kld + k) / 2, tile[2 * kp][rr], tile[2 * kp + 1][rr], e);
  }
}

// ------------------------------------------------------------------ epilogue arithmetic
// Integer value of an integer-valued float with |v| < 2^22 (one FADD).
__device__ __forceinline__ int small_float_to_int(float v) {
  return (int)(__float_as_uint(v + 12582912.0f) - 0x4B400000u);
}

// trunc(m6 2^49) for the float slot-6 sum (integer operations only).
__device__ __forceinline__ long long m6_fixed(float m6) {
  const uint32_t b = __float_as_uint(m6);
  const int E = (int)((b >> 23) & 0xff);
  if (E == 0) return 0;
  const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
  const int sh = E - 101;  // m 2^(E - 150) 2^49 = m 2^(E - 101)
  long long v;
  if (sh >= 0) v = sh < 40 ? (m << sh) : 0;  // |m6| < 2^-17 by the digit bounds
  else v = sh > -32 ? (m >> (-sh)) : 0;
  return (b >> 31) ? -v : v;
}

// FP64 value nearest to (H 2^14 + R) 2^(ex - 63), using integer operations
// (a second rounding only for results that leave the normal range).
__device__ __forceinline__ double z_to_double(long long H, long long R, int ex) {
  const long long zh = H + (R >> 14);
  const unsigned long long zl = (unsigned long long)(R & ((1ll << 14) - 1));
  if (zh == 0 && zl == 0) return 0.0;
  const bool neg = zh < 0;
  unsigned long long mh, ml;  // |Z| = mh 2^14 + ml, 0 <= ml < 2^14
  if (!neg) {
    mh = (unsigned long long)zh;
    ml = zl;
  } else if (zl == 0) {
    mh = (unsigned long long)(-zh);
    ml = 0;
  } else {
    mh = (unsigned long long)(-zh) - 1ull;
    ml = (1ull << 14) - zl;
  }
  const unsigned long long hi = mh >> 50, lo = (mh << 14) | ml;
  const int lz = hi ? __clzll((long long)hi) : 64 + __clzll((long long)lo);
  unsigned long long nh, nl;
  if (lz >= 64) {
    nh = lo << (lz - 64);
    nl = 0;
  } else if (lz == 0) {
    nh = hi;
    nl = lo;
  } else {
    nh = (hi << lz) | (lo >> (64 - lz));
    nl = lo << lz;
  }
  unsigned long long mant = nh >> 11;
  const unsigned rb = (unsigned)(nh & 0x7FFull);
  if (rb > 0x400u || (rb == 0x400u && (nl != 0 || (mant & 1ull)))) ++mant;
  int e2 = 127 - lz;
  if (mant >> 53) {
    mant >>= 1;
    ++e2;
  }
  const int be = e2 - 63 + ex + 1023;
  if (be >= 1 && be <= 2046)
    return __longlong_as_double(
        (long long)(((unsigned long long)neg << 63) | ((unsigned long long)be << 52) | (mant & 0xFFFFFFFFFFFFFull)));
  const double v = ldexp((double)mant, e2 - 52 - 63 + ex);
  return neg ? -v : v;
}

// ------------------------------------------------------------------ product kernel
struct TcArgs {
  int M, N, K;       // op(A) is M x K, op(B) is K x N
  int mt, nt, S;     // tiles along M and N, K splits
  int kchunk;        // K per split, a multiple of 128
  double alpha, beta;
  double* C;
  int ldc;
  double* part;      // S > 1: partial products part[z][i + j M]
  const int* emaxA;  // biased exponent maxima of the rows of op(A)
  const int* emaxB;  // ... of the columns of op(B)
  int* status;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_oztc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + TC_NS * TC_STAGE_BYTES);
  // bars: full[NS], empty[NS], tfull, tempty, done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TC_NS + 3);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (TC_NS + s); };
  const uint32_t tfull = bar0 + 8u * (2 * TC_NS), tempty = tfull + 8u, done = tfull + 16u;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, TC_EPI_WARPS);
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == TC_PROD_WARP && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == TC_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int ntiles = a.mt * a.nt * a.S;
  auto tile_of = [&](int t, int& m0, int& n0, int& kb, int& ke) {
    const int z = t % a.S, mn = t / a.S;
    m0 = (mn % a.mt) * TC_BM;
    n0 = (mn / a.mt) * TC_BN;
    kb = z * a.kchunk;
    ke = min(a.K, kb + a.kchunk);
  };

  if (warp == TC_PROD_WARP) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0, kb, ke;
        tile_of(t, m0, n0, kb, ke);
        for (int k = kb; k < ke; k += TC_BK, ++it) {
          const int s = it % TC_NS;
          const uint32_t r = it / TC_NS;
          if (!mbar_wait(empty(s), (r & 1) ^ 1, abort, a.status)) {
            ok = false;
            break;
          }
          const uint32_t sa = sbase + s * TC_STAGE_BYTES;
          mbar_expect_tx(full(s), TC_STAGE_BYTES);
          tma_load_3d(sa, &tmA, full(s), k, m0, 0);
          tma_load_3d(sa + TC_A_BYTES, &tmB, full(s), k, n0, 0);
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA's memory goes away
        const uint32_t first = it > (uint32_t)TC_NS ? it - TC_NS : 0;
        for (uint32_t j = first; j < it; ++j) mbar_wait_quiet(full(j % TC_NS), (j / TC_NS) & 1);
      }
    }
  } else if (warp == TC_MMA_WARP) {
    if (lane == 0) {
      uint32_t it = 0, win = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0, kb, ke;
        tile_of(t, m0, n0, kb, ke);
        for (int w0 = kb; w0 < ke && ok; w0 += TC_BK * TC_WIN, ++win) {
          if (!mbar_wait(tempty, (win & 1) ^ 1, abort, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int w1 = min(ke, w0 + TC_BK * TC_WIN);
          for (int k = w0; k < w1; k += TC_BK, ++it) {
            const int s = it % TC_NS;
            const uint32_t r = it / TC_NS;
            if (!mbar_wait(full(s), r & 1, abort, a.status)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sa = sbase + s * TC_STAGE_BYTES, sb = sa + TC_A_BYTES;
            // the first k-step of a window overwrites every slot with plane
            // p = 0 (it reaches slots 0..7); everything else accumulates
#pragma unroll
            for (int p = 0; p < TC_ND; ++p) {
              const uint64_t ad = sdesc_sw32(sa + p * (TC_BM * TC_BK * 2));
              const uint32_t acc = (k == w0 && p == 0) ? 0u : 1u;
#pragma unroll
              for (int q0 = 0; q0 < TC_ND - p; q0 += 4) {
                const int nq = TC_ND - p - q0 < 4 ? TC_ND - p - q0 : 4;
                const uint64_t bd = sdesc_sw32(sb + q0 * (TC_BN * TC_BK * 2));
                tc_mma(tmem + (p + q0) * TC_BN, ad, bd, idesc_n(TC_BN * nq), acc);
              }
            }
            tc_commit(empty(s));
          }
          if (ok) tc_commit(tfull);
        }
      }
      // every MMA issued by this thread has completed once `done` fires
      tc_commit(done);
      mbar_wait_quiet(done, 0);
    }
  } else {
    // ---- epilogue warps
    const int quad = warp & 3, cg = warp >> 2;
    const int row = quad * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + cg * TC_EPI_COLS;
    // how the product meets C (uniform over the kernel, decided once):
    // 0 partial store, 1 C = v, 2 C = -v, 3 C += v, 4 C -= v, 5 C = alpha v, 6 general
    const int mode = a.S > 1 ? 0
                     : a.beta == 0.0 ? (a.alpha == 1.0 ? 1 : a.alpha == -1.0 ? 2 : 5)
                     : a.beta == 1.0 ? (a.alpha == 1.0 ? 3 : a.alpha == -1.0 ? 4 : 6)
                                     : 6;
    uint32_t win = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int m0, n0, kb, ke;
      tile_of(t, m0, n0, kb, ke);
      long long H[TC_EPI_COLS];
      float M6[TC_EPI_COLS];
#pragma unroll
      for (int c = 0; c < TC_EPI_COLS; ++c) {
        H[c] = 0;
        M6[c] = 0.f;
      }
      for (int w0 = kb; w0 < ke; w0 += TC_BK * TC_WIN, ++win) {
        // every lane waits; the warp continues only together (tcgen05.ld is warp-wide)
        const bool got = mbar_wait(tfull, win & 1, abort, a.status);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc_fence_after();
        uint32_t v[TC_EPI_COLS];
        // slots 0, 1: |S| < 2^22 (one FADD each); slots 2..5: |S| < 2^24. Slots
        // (2k, 2k+1) are first combined in 32 bits, S_2k 2^7 + S_2k+1 < 2^31, so
        // H takes three 64-bit shift-adds per window instead of six
#pragma unroll
        for (int s = 0; s < 6; s += 2) {
          int P[TC_EPI_COLS];
          tc_ld16(tbase + s * TC_BN, v);
          tc_wait_ld();
          const float up0 = __uint_as_float((uint32_t)(127 + 7 * s) << 23);  // S_a = slot a x 2^(7a), exact
#pragma unroll
          for (int c = 0; c < TC_EPI_COLS; ++c) {
            const float f = __uint_as_float(v[c]) * up0;
            P[c] = (s < 2 ? small_float_to_int(f) : __float2int_rn(f)) << 7;
          }
          tc_ld16(tbase + (s + 1) * TC_BN, v);
          tc_wait_ld();
          const float up1 = __uint_as_float((uint32_t)(127 + 7 * (s + 1)) << 23);
#pragma unroll
          for (int c = 0; c < TC_EPI_COLS; ++c) {
            const float f = __uint_as_float(v[c]) * up1;
            P[c] += s < 2 ? small_float_to_int(f) : __float2int_rn(f);
            H[c] += (long long)P[c] << (7 * (4 - s));
          }
        }
#pragma unroll
        for (int s = 6; s < 8; ++s) {
          tc_ld16(tbase + s * TC_BN, v);
          tc_wait_ld();
#pragma unroll
          for (int c = 0; c < TC_EPI_COLS; ++c) M6[c] += __uint_as_float(v[c]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty);
      }
      if (!ok) break;
      const int i = m0 + row;
      if (i < a.M) {
        const int ei = scale_exp_tc(a.emaxA[i]);
        const bool needc = mode == 3 || mode == 4 || mode == 6;
        // chunks of TC_CCH columns: the C loads of a chunk are issued together
        // (one memory latency per chunk instead of one per element)
#pragma unroll
        for (int h = 0; h < TC_EPI_COLS; h += TC_CCH) {
          double cold[TC_CCH];
#pragma unroll
          for (int c = 0; c < TC_CCH; ++c) {
            const int j = n0 + cg * TC_EPI_COLS + h + c;
            cold[c] = (needc && j < a.N) ? a.C[i + (size_t)j * a.ldc] : 0.0;
          }
#pragma unroll
          for (int c = 0; c < TC_CCH; ++c) {
            const int j = n0 + cg * TC_EPI_COLS + h + c;
            if (j >= a.N) continue;
            const double v = z_to_double(H[h + c], m6_fixed(M6[h + c]), ei + scale_exp_tc(a.emaxB[j]));
            const double nv = __longlong_as_double(__double_as_longlong(v) ^ (1ll << 63));  // -v, exact
            double* cp = a.C + i + (size_t)j * a.ldc;
            switch (mode) {
              case 0: a.part[(size_t)(t % a.S) * a.M * a.N + i + (size_t)j * a.M] = v; break;
              case 1: *cp = v; break;
              case 2: *cp = nv; break;
              case 3: *cp = cold[c] + v; break;
              case 4: *cp = cold[c] + nv; break;
              case 5: *cp = a.alpha * v; break;
              default: *cp = fma(a.alpha, v, a.beta * cold[c]); break;
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == TC_MMA_WARP) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

__global__ void k_oztc_reduce(int M, int N, int S, double alpha, const double* __restrict__ part, double beta,
                              double* C, int ldc) {
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    double s = part[e];
    for (int z = 1; z < S; ++z) s += part[z * MN + e];
    const int i = (int)(e % M), j = (int)(e / M);
    double* cp = C + i + (size_t)j * ldc;
    *cp = beta == 0.0 ? alpha * s : fma(alpha, s, beta * *cp);
  }
}

// ------------------------------------------------------------------ host side
// 3-D map over digit planes [8][rows][kld] (bf16), box 16 x box_rows x 8.
bool plane_map(CUtensorMap* map, const void* planes, int rows, int K, int kld, int box_rows) {
  return plane_map_3d(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, planes, TC_ND, rows, K, kld, box_rows);
}

inline int kld_of(int K) { return (K + 7) & ~7; }

// Exponents and digit planes of the R x K operand (contig: element (r, k) at
// X[k + r ld]; else at X[r + k ld]).
void split_operand(const Ctx& c, bool contig, int R, int K, const double* X, int ld, int* emax, uint16_t* planes) {
  const int kld = kld_of(K);
  if (contig && K >= 2048) {
    // long rows: exponent and digits in one launch, one CTA per row
    k_split_rows<<<R, SPLIT_T, 0, c.stream>>>(R, K, X, ld, emax, reinterpret_cast<uint32_t*>(planes), kld);
    note_launch(c);
    return;
  }
  cudaMemsetAsync(emax, 0, sizeof(int) * R, c.stream);
  const int kch = 4096;
  dim3 ge(contig ? ceil_div(R, 8) : ceil_div(R, 128), ceil_div(K, kch));
  if (contig) k_plane_exp<true><<<ge, 256, 0, c.stream>>>(R, K, kch, X, ld, emax);
  else k_plane_exp<false><<<ge, 128, 0, c.stream>>>(R, K, kch, X, ld, emax);
  if (contig) {
    k_split_contig<<<ceil_div(R, 8), 256, 0, c.stream>>>(R, K, X, ld, emax, reinterpret_cast<uint32_t*>(planes), kld);
  } else {
    dim3 g(ceil_div(R, 32), ceil_div(K, 64));
    k_split_strided<<<g, 256, 0, c.stream>>>(R, K, X, ld, emax, reinterpret_cast<uint32_t*>(planes), kld);
  }
  note_launch(c, 2);
}

}  // namespace

size_t oztc_plane_elems(int rows, int K) { return (size_t)TC_ND * rows * kld_of(K) + 128; }

bool oztc_available() { return encoder() != nullptr; }

// C = alpha op(A) op(B) + beta C on the tcgen05 tensor cores with FP64
// accuracy. Scratch: emax (M + N ints), planes of op(A) (pa_cap bf16) and of
// op(B) (pb_cap bf16; op(B) is processed in column chunks that fit), split-K
// partials (part_cap doubles). Returns false (nothing queued) when the
// tensor-map encoder is unavailable or the A planes do not fit.
bool gemm_f64x_tc(const Ctx& c, bool ta, bool tb, int M, int N, int K, double alpha, const double* A, int lda,
                  const double* B, int ldb, double beta, double* C, int ldc, int* emax, uint16_t* pa, size_t pa_cap,
                  uint16_t* pb, size_t pb_cap, double* part, size_t part_cap) {
  if (M <= 0 || N <= 0 || K <= 0) return false;
  if (!oztc_available()) return false;
  const int kld = kld_of(K);
  if ((size_t)TC_ND * M * kld > pa_cap) return false;
  const size_t col_elems = (size_t)TC_ND * kld;
  int nc = (int)std::min<size_t>((size_t)N, pb_cap / col_elems);
  if (nc < N) nc = nc / TC_BN * TC_BN;
  if (nc <= 0) return false;
  const int nlast = N - (ceil_div(N, nc) - 1) * nc;
  // tensor maps first, so that a failure queues nothing
  CUtensorMap mapA, mapB, mapBlast;
  if (!plane_map(&mapA, pa, M, K, kld, TC_BM) || !plane_map(&mapB, pb, nc, K, kld, TC_BN) ||
      !plane_map(&mapBlast, pb, nlast, K, kld, TC_BN))
    return false;
  if (cudaFuncSetAttribute(k_oztc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int* emaxA = emax;
  int* emaxB = emax + M;
  // op(A) rows are contiguous when op(A) = A^T
  split_operand(c, ta, M, K, A, lda, emaxA, pa);
  const int kwin = ceil_div(K, TC_BK * TC_WIN);
  for (int j0 = 0; j0 < N; j0 += nc) {
    const int nn = std::min(nc, N - j0);
    // columns j0.. of op(B): contiguous when op(B) = B (column-major K x N)
    const double* Bj = tb ? B + j0 : B + (size_t)j0 * ldb;
    split_operand(c, !tb, nn, K, Bj, ldb, emaxB + j0, pb);
    TcArgs a{};
    a.M = M;
    a.N = nn;
    a.K = K;
    a.mt = ceil_div(M, TC_BM);
    a.nt = ceil_div(nn, TC_BN);
    // K splits: fill the machine in whole waves; each split keeps at least 4
    // windows and at most 64 (H stays below 2^63)
    const int mn = a.mt * a.nt;
    int S = 0;
    double best = 1e30;
    for (int s = 1; s <= 64; ++s) {
      if (s > 1 && (kwin / s < 4 || (size_t)s * M * nn > part_cap)) break;
      if (ceil_div(kwin, s) > 64) continue;
      const double waves = (double)mn * s / c.sms;
      const double cost = std::ceil(waves) / s + 0.02 * s;
      if (cost < best - 1e-9) {
        best = cost;
        S = s;
      }
    }
    if (S == 0) S = ceil_div(kwin, 64);  // very long K with little partial space
    a.kchunk = ceil_div(kwin, S) * TC_BK * TC_WIN;
    a.S = ceil_div(K, a.kchunk);
    if (a.S > 1 && (size_t)a.S * M * nn > part_cap) {
      // no room for the partial products: fall back for this chunk
      gemm_f64x(c, ta, tb, M, nn, K, alpha, A, lda, Bj, ldb, beta, C + (size_t)j0 * ldc, ldc, emax, part, part_cap);
      continue;
    }
    a.alpha = alpha;
    a.beta = beta;
    a.C = C + (size_t)j0 * ldc;
    a.ldc = ldc;
    a.part = part;
    a.emaxA = emaxA;
    a.emaxB = emaxB + j0;
    a.status = c.status;
    const int tiles = mn * a.S;
    const int grid = std::min(tiles, c.sms);
    const bool timed = c.kt && c.kt->start(c.stream);
    k_oztc<<<grid, TC_THREADS, TC_SMEM, c.stream>>>(mapA, nn == nc ? mapB : mapBlast, a);
    if (timed) {
      // 36 digit-pair products; bytes: both operands' digit planes once (16 B per
      // element) and C read (beta != 0) and written, or the split-K partials written
      const double planes = 16.0 * ((double)M + nn) * K;
      const double cbytes = a.S > 1 ? 8.0 * a.S * M * nn : 8.0 * M * nn * (beta != 0.0 ? 2.0 : 1.0);
      c.kt->stop(c.stream, 36.0 * 2.0 * (double)M * nn * K, planes + cbytes);
    }
    note_launch(c);
    if (a.S > 1) {
      const size_t MN = (size_t)M * nn;
      const int blocks = (int)std::min<size_t>((MN + 255) / 256, (size_t)c.sms * 8);
      k_oztc_reduce<<<blocks, 256, 0, c.stream>>>(M, nn, a.S, alpha, part, beta, a.C, ldc);
      note_launch(c);
    }
  }
  return true;
}

}  // namespace rqr
