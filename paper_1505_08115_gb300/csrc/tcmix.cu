// tcmix.cu -- the products of the mixed-precision modes on the fifth-
// generation tensor cores (tcgen05.mma, accumulators in TMEM, operands staged
// by TMA): C = alpha op(A) op(B) + beta C with op(A), op(B) rounded to
//   TF32   one TF32 plane per operand (10 explicit significand bits);
//   3xTF32 big + small TF32 planes, x ~ big + small to about 22 bits, and
//          the three products big.big + big.small + small.big;
//   3xBF16 hi + lo bf16 planes (about 16 bits) and hi.hi + hi.lo + lo.hi;
// all accumulated in FP32 over the whole K range (modes the paper does not
// have: its Sec. 2 cost model only requires the products to be matrix-matrix
// multiplications).
//
// 1. Splitting (k_mix_split_*): row r of op(A) (or of op(B)^T) becomes NP
//    planes planes[p][r][k], K contiguous, row stride kld (a multiple of 8).
// 2. Products (k_tcmix): persistent, one CTA per SM, 128 x 256 output tiles,
//    K consumed 32 bytes per stage (8 TF32 or 16 bf16). One thread issues the
//    1 or 3 MMAs of a stage (M = 128, N = 256) into one of two TMEM buffers of
//    256 FP32 columns, so the drain of one tile overlaps the MMAs of the next.
// 3. Drain: 16 epilogue warps (warp w: TMEM lanes 32 (w % 4).., 64 columns
//    from 64 (w / 4)) read their accumulators 16 columns at a time, combine
//    them with C in C's precision (or store split-K partials; 8 C loads of a
//    thread in flight together) and release the buffer once the tile is
//    written. Measured on the 16384^2 trailing update and not kept: a
//    prefetch of the next tile's C into L2 (+5 ms, more DRAM re-reads), 16
//    loads in flight (+22 ms), 8 epilogue warps with 32 loads each (+25 ms).
// Waits are bounded (2 s); on a timeout the CTA records RQR_ERR_TIMEOUT,
// lets its copies and MMAs land, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace rqr {

namespace {

using namespace tcp;

constexpr int MX_BM = 128, MX_BN = 256, MX_NS = 6;
constexpr int MX_EPI_WARPS = 16, MX_PROD_WARP = 16, MX_MMA_WARP = 17, MX_THREADS = 576;
constexpr int MX_EPI_COLS = MX_BN / (MX_EPI_WARPS / 4);  // 64 columns per epilogue warp
constexpr int MX_CCH = 16;                                // accumulator columns per TMEM load
constexpr int MX_CLD = 8;                                 // C values loaded together
constexpr uint32_t MX_TMEM_COLS = 512;                    // two accumulator buffers of 256 columns

// Operand format of each mode: planes per operand, bytes per element, K per stage.
template <int MODE>
struct Mix;
template <>
struct Mix<RQR_TF32> {
  static constexpr int NP = 1, ESZ = 4, KS = 8;
};
template <>
struct Mix<RQR_3XTF32> {
  static constexpr int NP = 2, ESZ = 4, KS = 8;
};
template <>
struct Mix<RQR_3XBF16> {
  static constexpr int NP = 2, ESZ = 2, KS = 16;
};

template <int MODE>
constexpr uint32_t a_bytes() { return Mix<MODE>::NP * MX_BM * 32; }
template <int MODE>
constexpr uint32_t b_bytes() { return Mix<MODE>::NP * MX_BN * 32; }
template <int MODE>
constexpr uint32_t stage_bytes() { return a_bytes<MODE>() + b_bytes<MODE>(); }
template <int MODE>
constexpr size_t mix_smem() { return (size_t)MX_NS * stage_bytes<MODE>() + 1024 + 256; }

// Instruction descriptor: D FP32, A and B K-major of format fmt (kind::f16:
// 1 = bf16; kind::tf32: 2 = TF32), M = 128, N = 256.
__host__ __device__ constexpr uint32_t mix_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(MX_BN >> 3) << 17) | ((uint32_t)(MX_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

template <int MODE>
__device__ __forceinline__ void mma_mode(uint32_t d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  if constexpr (MODE == RQR_3XBF16) tc_mma(d, adesc, bdesc, mix_idesc(1u), acc);
  else mma_tf32(d, adesc, bdesc, mix_idesc(2u), acc);
}

// ------------------------------------------------------------------ splitting
// TF32 nearest to an FP32 value (ties away from zero), in an FP32 container
// whose low 13 bits are zero: the tensor core reads only the top 19 bits.
__device__ __forceinline__ uint32_t tf32_rn(float f) {
  uint32_t u = __float_as_uint(f);
  if ((u & 0x7f800000u) != 0x7f800000u) u += 0x1000u;
  return u & 0xffffe000u;
}

// An FP64 value as two FP32 values, x = hi + lo + d with |d| <= 2^-47 |x|:
// hi = the leading 24 significand bits (truncated), lo = the next 24 of the
// remaining 29, both from the bit pattern with integer operations (GB300
// runs FP64 arithmetic and conversions on its narrow FP64 pipe, which would
// bound the splitting). Values outside FP32's normal range give hi = +-0 (below
// 2^-126) or +-inf (at or above 2^128).
__device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(bits >> 32) & 0x80000000u;
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;  // x = 1.f 2^e
  hi = lo = __uint_as_float(sign);
  if (e < -126) return;
  if (e > 127) {
    hi = __uint_as_float(sign | 0x7f800000u);
    return;
  }
  const unsigned long long f = bits & 0xFFFFFFFFFFFFFull;  // 52 fraction bits
  hi = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(f >> 29));
  const uint32_t rem = (uint32_t)(f & 0x1FFFFFFFu);  // value rem 2^(e - 52)
  if (rem == 0) return;
  const int msb = 31 - __clz(rem);                   // rem in [2^msb, 2^(msb+1))
  const int ef = e - 52 + msb + 127;
  if (ef <= 0) return;
  const uint32_t frac = msb >= 23 ? rem >> (msb - 23) : rem << (23 - msb);
  lo = __uint_as_float(sign | ((uint32_t)ef << 23) | (frac & 0x7FFFFFu));
}

// The planes of one value: x ~ sum_p plane_p (MODE's split), written at
// element `off` of each plane (planes pstride elements apart). FP32 and
// integer operations only.
template <int MODE, typename IT>
__device__ __forceinline__ void put_planes(void* planes, size_t pstride, size_t off, IT x) {
  float hi, lo;
  if constexpr (sizeof(IT) == 8) {
    split_f64(x, hi, lo);
  } else {
    hi = x;
    lo = 0.f;
  }
  if constexpr (MODE == RQR_3XBF16) {
    uint16_t* P = static_cast<uint16_t*>(planes);
    const __nv_bfloat16 h16 = __float2bfloat16_rn(hi);
    // hi - h16 is exact in FP32 (h16 is hi rounded to fewer bits)
    const __nv_bfloat16 l16 = __float2bfloat16_rn((hi - __bfloat162float(h16)) + lo);
    P[off] = __bfloat16_as_ushort(h16);
    P[pstride + off] = __bfloat16_as_ushort(l16);
  } else {
    uint32_t* P = static_cast<uint32_t*>(planes);
    const uint32_t big = tf32_rn(hi);
    P[off] = big;
    if constexpr (MODE == RQR_3XTF32) {
      // hi - big is exact in FP32 (big is hi rounded to fewer bits)
      P[pstride + off] = tf32_rn((hi - __uint_as_float(big)) + lo);
    }
  }
}

// Rows with contiguous K (element (r, k) at X[k + r ld]): one warp per row.
template <int MODE, typename IT>
__global__ void k_mix_split_contig(int R, int K, const IT* __restrict__ X, int ld, void* planes, int kld) {
  const int lane = threadIdx.x & 31;
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= R) return;
  const size_t pstride = (size_t)R * kld;
  const IT* x = X + (size_t)r * ld;
  for (int k = lane; k < K; k += 32) put_planes<MODE, IT>(planes, pstride, (size_t)r * kld + k, x[k]);
}

// Rows stored with stride (element (r, k) at X[r + k ld]): 32 x 64 tiles
// transposed through shared memory.
template <int MODE, typename IT>
__global__ void __launch_bounds__(256) k_mix_split_strided(int R, int K, const IT* __restrict__ X, int ld,
                                                            void* planes, int kld) {
  __shared__ IT tile[64][33];
  const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 64;
  const int t = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int r = r0 + (t & 31), k = k0 + (t >> 5) + 8 * i;
    tile[(t >> 5) + 8 * i][t & 31] = (r < R && k < K) ? X[r + (size_t)k * ld] : IT(0);
  }
  __syncthreads();
  const size_t pstride = (size_t)R * kld;
  // thread t writes row r0 + t / 8, K positions (t % 8) + 8 j: each group of 8
  // threads covers 8 consecutive K of one row per step
  const int rr = t >> 3, r = r0 + rr;
  if (r >= R) return;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int kk = (t & 7) + 8 * j, k = k0 + kk;
    if (k < K) put_planes<MODE, IT>(planes, pstride, (size_t)r * kld + k, tile[kk][rr]);
  }
}

// ------------------------------------------------------------------ epilogue arithmetic
// The FP64 value of an FP32 accumulator, from its bit pattern with integer
// operations (exact, subnormals included): GB300 runs the FP32 -> FP64
// conversion on its narrow FP64 pipe, where it doubled the epilogue's FP64
// work (measured: FP64 pipe 79% busy in the trailing update).
__device__ __forceinline__ double f32_to_f64(uint32_t u) {
  const unsigned long long s = (unsigned long long)(u >> 31) << 63;
  const uint32_t e = (u >> 23) & 0xFFu, m = u & 0x7FFFFFu;
  unsigned long long bits;
  if (e == 0xFFu) {
    bits = s | (0x7FFull << 52) | ((unsigned long long)m << 29);
  } else if (e != 0) {
    bits = s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
  } else if (m == 0) {
    bits = s;
  } else {
    const int sh = __clz(m) - 8;  // m << sh has its leading bit at position 23
    bits = s | ((unsigned long long)(897 - sh) << 52) | ((unsigned long long)((m << sh) & 0x7FFFFFu) << 29);
  }
  return __longlong_as_double((long long)bits);
}

template <typename CT>
__device__ __forceinline__ CT acc_value(uint32_t u) {
  if constexpr (sizeof(CT) == 8) return f32_to_f64(u);
  else return __uint_as_float(u);
}

// -x by flipping the sign bit (an integer operation, exact)
template <typename CT>
__device__ __forceinline__ CT neg_value(CT x) {
  if constexpr (sizeof(CT) == 8) return __longlong_as_double(__double_as_longlong(x) ^ (1ll << 63));
  else return __int_as_float(__float_as_int(x) ^ (int)0x80000000u);
}

// ------------------------------------------------------------------ product kernel
template <typename CT>
struct MixArgs {
  int M, N, K;      // op(A) is M x K, op(B) is K x N
  int mt, nt, S;    // tiles along M and N, K splits
  int kchunk;       // K per split, a multiple of the stage's K
  CT alpha, beta;
  CT* C;
  int ldc;
  CT* part;         // S > 1: partial products part[z][i + j M]
  int* status;
};

template <int MODE, typename CT>
__global__ void __launch_bounds__(MX_THREADS, 1)
    k_tcmix(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const MixArgs<CT> a) {
  constexpr int KS = Mix<MODE>::KS;
  constexpr uint32_t SB = stage_bytes<MODE>(), AB = a_bytes<MODE>();
  extern __shared__ unsigned char mx_smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)mx_smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + MX_NS * SB);
  // bars: full[NS], empty[NS], tfull[2], tempty[2], done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * MX_NS + 5);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t sbase = smem_u32(smem);
  const uint32_t bar0 = smem_u32(bars);
  auto full = [&](int s) { return bar0 + 8u * s; };
  auto empty = [&](int s) { return bar0 + 8u * (MX_NS + s); };
  auto tfull = [&](int b) { return bar0 + 8u * (2 * MX_NS + b); };
  auto tempty = [&](int b) { return bar0 + 8u * (2 * MX_NS + 2 + b); };
  const uint32_t done = bar0 + 8u * (2 * MX_NS + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < MX_NS; ++s) {
      mbar_init(full(s), 1);
      mbar_init(empty(s), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(tfull(b), 1);
      mbar_init(tempty(b), MX_EPI_WARPS);
    }
    mbar_init(done, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == MX_PROD_WARP && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == MX_MMA_WARP) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(MX_TMEM_COLS)
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
    m0 = (mn % a.mt) * MX_BM;
    n0 = (mn / a.mt) * MX_BN;
    kb = z * a.kchunk;
    ke = min(a.K, kb + a.kchunk);
  };

  if (warp == MX_PROD_WARP) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int m0, n0, kb, ke;
        tile_of(t, m0, n0, kb, ke);
        for (int k = kb; k < ke; k += KS, ++it) {
          const int s = it % MX_NS;
          const uint32_t r = it / MX_NS;
          if (!mbar_wait(empty(s), (r & 1) ^ 1, abort, a.status)) {
            ok = false;
            break;
          }
          const uint32_t sa = sbase + s * SB;
          mbar_expect_tx(full(s), SB);
          tma_load_3d(sa, &tmA, full(s), k, m0, 0);
          tma_load_3d(sa + AB, &tmB, full(s), k, n0, 0);
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA's memory goes away
        const uint32_t first = it > (uint32_t)MX_NS ? it - MX_NS : 0;
        for (uint32_t j = first; j < it; ++j) mbar_wait_quiet(full(j % MX_NS), (j / MX_NS) & 1);
      }
    }
  } else if (warp == MX_MMA_WARP) {
    if (lane == 0) {
      uint32_t it = 0, tl = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        int m0, n0, kb, ke;
        tile_of(t, m0, n0, kb, ke);
        const int bf = tl & 1;
        const uint32_t use = tl >> 1;  // how often buffer bf was used before
        if (!mbar_wait(tempty(bf), (use & 1) ^ 1, abort, a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + bf * MX_BN;
        for (int k = kb; k < ke; k += KS, ++it) {
          const int s = it % MX_NS;
          const uint32_t r = it / MX_NS;
          if (!mbar_wait(full(s), r & 1, abort, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = sbase + s * SB, sb = sa + AB;
          const uint32_t first = k == kb ? 0u : 1u;
          mma_mode<MODE>(d, sdesc_sw32(sa), sdesc_sw32(sb), first);
          if constexpr (Mix<MODE>::NP == 2) {
            // the two cross products of the split operands into the same accumulator
            mma_mode<MODE>(d, sdesc_sw32(sa), sdesc_sw32(sb + MX_BN * 32), 1u);
            mma_mode<MODE>(d, sdesc_sw32(sa + MX_BM * 32), sdesc_sw32(sb), 1u);
          }
          tc_commit(empty(s));
        }
        if (ok) tc_commit(tfull(bf));
      }
      // every MMA issued by this thread has completed once `done` fires
      tc_commit(done);
      mbar_wait_quiet(done, 0);
    }
  } else {
    // ---- epilogue warps
    const int quad = warp & 3, cg = warp >> 2;
    const int row = quad * 32 + lane;
    // how the product meets C (uniform over the kernel):
    // 0 partial store, 1 C = v, 2 C = -v, 3 C += v, 4 C -= v, 5 C = alpha v, 6 general
    const int mode = a.S > 1 ? 0
                     : a.beta == CT(0) ? (a.alpha == CT(1) ? 1 : a.alpha == CT(-1) ? 2 : 5)
                     : a.beta == CT(1) ? (a.alpha == CT(1) ? 3 : a.alpha == CT(-1) ? 4 : 6)
                                       : 6;
    uint32_t tl = 0;
    const bool needc = mode == 3 || mode == 4 || mode == 6;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      int m0, n0, kb, ke;
      tile_of(t, m0, n0, kb, ke);
      const int bf = tl & 1;
      const int i = m0 + row;
      const bool got = mbar_wait(tfull(bf), (tl >> 1) & 1, abort, a.status);
      if (!__all_sync(0xffffffffu, got)) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + bf * MX_BN + cg * MX_EPI_COLS;
      // 16 columns at a time: the buffer stays ours until the whole tile is
      // written (the MMA warp needs it again only two tiles later)
#pragma unroll 1
      for (int h = 0; h < MX_EPI_COLS; h += MX_CCH) {
        uint32_t v[MX_CCH];
        __syncwarp();  // tcgen05.ld is warp-wide: every lane takes part, rows past M included
        tc_ld16(taddr + h, v);
        tc_wait_ld();
        if (i < a.M) {
#pragma unroll
          for (int g = 0; g < MX_CCH; g += MX_CLD) {
            const int jb = n0 + cg * MX_EPI_COLS + h + g;
            CT cold[MX_CLD];
#pragma unroll
            for (int c = 0; c < MX_CLD; ++c)
              cold[c] = (needc && jb + c < a.N) ? a.C[i + (size_t)(jb + c) * a.ldc] : CT(0);
#pragma unroll
            for (int c = 0; c < MX_CLD; ++c) {
              const int j = jb + c;
              if (j >= a.N) continue;
              const CT x = acc_value<CT>(v[g + c]);
              CT* cp = a.C + i + (size_t)j * a.ldc;
              switch (mode) {
                case 0: a.part[(size_t)(t % a.S) * a.M * a.N + i + (size_t)j * a.M] = x; break;
                case 1: *cp = x; break;
                case 2: *cp = neg_value<CT>(x); break;
                case 3: *cp = cold[c] + x; break;
                case 4: *cp = cold[c] - x; break;
                case 5: *cp = a.alpha * x; break;
                default: *cp = a.alpha * x + a.beta * cold[c]; break;
              }
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty(bf));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MX_MMA_WARP) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MX_TMEM_COLS) : "memory");
  }
}

template <typename CT>
__global__ void k_tcmix_reduce(int M, int N, int S, CT alpha, const CT* __restrict__ part, CT beta, CT* C, int ldc) {
  const size_t MN = (size_t)M * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    CT s = part[e];
    for (int z = 1; z < S; ++z) s += part[z * MN + e];
    const int i = (int)(e % M), j = (int)(e / M);
    CT* cp = C + i + (size_t)j * ldc;
    *cp = beta == CT(0) ? alpha * s : alpha * s + beta * *cp;
  }
}

inline int mix_kld(int K) { return (K + 7) & ~7; }

template <int MODE, typename IT>
void split_mix(const Ctx& c, bool contig, int R, int K, const IT* X, int ld, void* planes) {
  const int kld = mix_kld(K);
  if (contig) {
    k_mix_split_contig<MODE, IT><<<ceil_div(R, 8), 256, 0, c.stream>>>(R, K, X, ld, planes, kld);
  } else {
    dim3 g(ceil_div(R, 32), ceil_div(K, 64));
    k_mix_split_strided<MODE, IT><<<g, 256, 0, c.stream>>>(R, K, X, ld, planes, kld);
  }
  note_launch(c);
}

template <int MODE, typename IT>
bool mix_tc_impl(const Ctx& c, bool ta, bool tb, int M, int N, int K, IT alpha, const IT* A, int lda, const IT* B,
                 int ldb, IT beta, IT* C, int ldc, void* pa, size_t pa_bytes, void* pb, size_t pb_bytes, IT* part,
                 size_t part_cap) {
  using MX = Mix<MODE>;
  if (M <= 0 || N <= 0 || K <= 0) return false;
  const int kld = mix_kld(K);
  const size_t row_bytes = (size_t)MX::NP * kld * MX::ESZ;
  if (row_bytes * M > pa_bytes) return false;
  int nc = (int)std::min<size_t>((size_t)N, pb_bytes / row_bytes);
  if (nc < N) nc = nc / MX_BN * MX_BN;
  if (nc <= 0) return false;
  const int nlast = N - (ceil_div(N, nc) - 1) * nc;
  const CUtensorMapDataType dt = MX::ESZ == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  CUtensorMap mapA, mapB, mapBlast;
  if (!plane_map_3d(&mapA, dt, MX::ESZ, pa, MX::NP, M, K, kld, MX_BM) ||
      !plane_map_3d(&mapB, dt, MX::ESZ, pb, MX::NP, nc, K, kld, MX_BN) ||
      !plane_map_3d(&mapBlast, dt, MX::ESZ, pb, MX::NP, nlast, K, kld, MX_BN))
    return false;
  if (cudaFuncSetAttribute(k_tcmix<MODE, IT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mix_smem<MODE>()) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  // op(A) rows are contiguous when op(A) = A^T
  split_mix<MODE, IT>(c, ta, M, K, A, lda, pa);
  const int ksteps = ceil_div(K, MX::KS);
  for (int j0 = 0; j0 < N; j0 += nc) {
    const int nn = std::min(nc, N - j0);
    const IT* Bj = tb ? B + j0 : B + (size_t)j0 * ldb;
    split_mix<MODE, IT>(c, !tb, nn, K, Bj, ldb, pb);
    MixArgs<IT> a{};
    a.M = M;
    a.N = nn;
    a.K = K;
    a.mt = ceil_div(M, MX_BM);
    a.nt = ceil_div(nn, MX_BN);
    // K splits: fill the machine in whole waves, each split keeping at least
    // 64 stages of K, as long as the partial products fit
    const int mn = a.mt * a.nt;
    int S = 1;
    double best = 1e30;
    for (int s = 1; s <= 32; ++s) {
      if (s > 1 && (ksteps / s < 64 || (size_t)s * M * nn > part_cap)) break;
      const double cost = std::ceil((double)mn * s / c.sms) / s + 0.02 * s;
      if (cost < best - 1e-9) {
        best = cost;
        S = s;
      }
    }
    a.kchunk = ceil_div(ksteps, S) * MX::KS;
    a.S = ceil_div(K, a.kchunk);
    a.alpha = alpha;
    a.beta = beta;
    a.C = C + (size_t)j0 * ldc;
    a.ldc = ldc;
    a.part = part;
    a.status = c.status;
    const int grid = std::min(mn * a.S, c.sms);
    const bool timed = c.kt && c.kt->start(c.stream);
    k_tcmix<MODE, IT><<<grid, MX_THREADS, mix_smem<MODE>(), c.stream>>>(mapA, nn == nc ? mapB : mapBlast, a);
    if (timed) {
      // flops: the 1 or 3 operand-plane products, 2 M N K each; bytes: both
      // operands' planes read once, C read (beta != 0) and written, or the
      // split-K partials written
      const double planes = (double)MX::NP * MX::ESZ * ((double)M + nn) * K;
      const double cbytes = a.S > 1 ? (double)sizeof(IT) * a.S * M * nn
                                    : (double)sizeof(IT) * M * nn * (beta != IT(0) ? 2.0 : 1.0);
      c.kt->stop(c.stream, (MX::NP == 2 ? 3.0 : 1.0) * 2.0 * (double)M * nn * K, planes + cbytes);
    }
    note_launch(c);
    if (a.S > 1) {
      const size_t MN = (size_t)M * nn;
      const int blocks = (int)std::min<size_t>((MN + 255) / 256, (size_t)c.sms * 8);
      k_tcmix_reduce<IT><<<blocks, 256, 0, c.stream>>>(M, nn, a.S, alpha, part, beta, a.C, ldc);
      note_launch(c);
    }
  }
  return true;
}

}  // namespace

size_t mix_plane_bytes(int mode, int rows, int K) {
  const int np = mode == RQR_TF32 ? 1 : 2, esz = mode == RQR_3XBF16 ? 2 : 4;
  return (size_t)np * esz * std::max(rows, 1) * mix_kld(std::max(K, 1)) + 256;
}

template <typename T>
bool gemm_mix_tc(const Ctx& c, int mode, bool ta, bool tb, int M, int N, int K, T alpha, const T* A, int lda,
                 const T* B, int ldb, T beta, T* C, int ldc, void* pa, size_t pa_bytes, void* pb, size_t pb_bytes,
                 T* part, size_t part_cap) {
  if (!encoder()) return false;
  switch (mode) {
    case RQR_TF32:
      return mix_tc_impl<RQR_TF32, T>(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, pa, pa_bytes, pb,
                                      pb_bytes, part, part_cap);
    case RQR_3XTF32:
      return mix_tc_impl<RQR_3XTF32, T>(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, pa, pa_bytes, pb,
                                        pb_bytes, part, part_cap);
    case RQR_3XBF16:
      return mix_tc_impl<RQR_3XBF16, T>(c, ta, tb, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, pa, pa_bytes, pb,
                                        pb_bytes, part, part_cap);
    default:
      return false;
  }
}

template bool gemm_mix_tc<double>(const Ctx&, int, bool, bool, int, int, int, double, const double*, int,
                                  const double*, int, double, double*, int, void*, size_t, void*, size_t, double*,
                                  size_t);
template bool gemm_mix_tc<float>(const Ctx&, int, bool, bool, int, int, int, float, const float*, int, const float*,
                                 int, float, float*, int, void*, size_t, void*, size_t, float*, size_t);

}  // namespace rqr
