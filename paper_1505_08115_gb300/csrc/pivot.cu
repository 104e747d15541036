// pivot.cu -- block pivot selection from the sketch (Sec. 4.1 with the
// over-sampling of Sec. 4.3): the first b steps of classical Householder QR
// with column pivoting (Fig. QR) on the l x n' sketch Y, and the application
// of the chosen swaps to the matrix, the sketch and the permutation.
//
// The working copy of Y lives in two ping-pong buffers (l x n' FP64 each,
// L2-resident at n' = 16384). One launch per pivot step: every CTA owns a
// fixed range of column positions; it reads the source column of each of its
// positions from the input buffer (the swap of positions j and c* is a change
// of source, so no CTA writes what another reads), applies the reflector of
// step j, recomputes the squared norm of the remaining rows, and writes the
// output buffer. The last CTA to finish (fence + atomic ticket, no waiting)
// picks the largest norm (lowest position on ties) and builds the next
// reflector.
#include <algorithm>

#include "common.cuh"

namespace rqr {

namespace {

constexpr int YT = 256;  // threads per CTA
constexpr int NW = YT / 32;

struct YArgs {
  int l, np, per;  // rows, positions, positions per CTA
};

__device__ bool y_last_cta(int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Per-CTA best (norm2, pos) from per-warp candidates in shared memory.
template <typename T>
__device__ void cta_best(T wn, int wp, T* shn, int* shp, T& bn, int& bp) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    shn[warp] = wn;
    shp[warp] = wp;
  }
  __syncthreads();
  bn = T(-1);
  bp = 0x7fffffff;
  for (int w = 0; w < NW; ++w)
    if (shn[w] > bn || (shn[w] == bn && shp[w] < bp)) {
      bn = shn[w];
      bp = shp[w];
    }
}

// Last CTA: global argmax over the CTA candidates (every thread scans a few,
// then a fixed-order reduction in shared memory; largest norm, lowest position
// on ties), record the pick, and build the reflector of the picked column
// (rows j..l-1 of buffer Yw, column pick).
template <typename T>
__device__ void pick_and_reflect(int j, const YArgs& a, const T* cand_n, const int* cand_p, const T* Yw, int* picks,
                                 T* vbuf, int* counter) {
  __shared__ T sn[YT];
  __shared__ int sp[YT];
  const int tid = threadIdx.x, lane = tid & 31;
  T bn = T(-1);
  int bp = 0x7fffffff;
  for (int q = tid; q < (int)gridDim.x; q += YT) {
    const T n = __ldcg(cand_n + q);
    const int p = __ldcg(cand_p + q);
    if (n > bn || (n == bn && p < bp)) {
      bn = n;
      bp = p;
    }
  }
  sn[tid] = bn;
  sp[tid] = bp;
  __syncthreads();
  for (int half = YT / 2; half > 0; half >>= 1) {
    if (tid < half) {
      const T on = sn[tid + half];
      const int op = sp[tid + half];
      if (on > sn[tid] || (on == sn[tid] && op < sp[tid])) {
        sn[tid] = on;
        sp[tid] = op;
      }
    }
    __syncthreads();
  }
  const int pick = sp[0];
  if (tid == 0) picks[j] = pick;
  // reflector of Yw(j:l, pick): alpha, norm, v = y / (alpha - beta), tau
  if (tid < 32) {
    const T* y = Yw + (size_t)pick * a.l;
    const int L = a.l - j;
    T s = T(0);
    for (int r = lane; r < L; r += 32) {
      const T x = __ldcg(y + j + r);
      s += x * x;
    }
    s = warp_sum(s);
    const T alpha = __ldcg(y + j);
    T tau = T(0), d = T(1);
    if (L >= 2 && s > T(0)) {
      const T beta = -sgn0(alpha) * sqrt(s);
      d = alpha - beta;
      tau = (beta - alpha) / beta;
    }
    for (int r = 1 + lane; r < L; r += 32) vbuf[1 + r] = tau == T(0) ? T(0) : __ldcg(y + j + r) / d;
    if (lane == 0) {
      vbuf[0] = tau;
      vbuf[1] = T(1);
      *counter = 0;
    }
  }
}

// Copies Y into Yw0, computes full column norms, CTA candidates; last CTA picks
// position 0's pivot and builds reflector 0.
template <typename T>
__global__ void __launch_bounds__(YT) k_ypick_init(YArgs a, const T* __restrict__ Y, int ldy, T* Yw0, T* cand_n,
                                                   int* cand_p, int* picks, T* vbuf, int* counter) {
  __shared__ T shn[NW];
  __shared__ int shp[NW];
  const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int lo = q * a.per, hi = min(a.np, lo + a.per);
  T wn = T(-1);
  int wp = 0x7fffffff;
  for (int pos = lo + warp; pos < hi; pos += NW) {
    const T* y = Y + (size_t)pos * ldy;
    T* o = Yw0 + (size_t)pos * a.l;
    T s = T(0);
    for (int r = lane; r < a.l; r += 32) {
      const T x = y[r];
      o[r] = x;
      s += x * x;
    }
    s = warp_sum(s);
    if (s > wn || (s == wn && pos < wp)) {
      wn = s;
      wp = pos;
    }
  }
  T bn;
  int bp;
  cta_best(wn, wp, shn, shp, bn, bp);
  if (threadIdx.x == 0) {
    cand_n[q] = bn;
    cand_p[q] = bp;
  }
  if (y_last_cta(counter)) pick_and_reflect<T>(0, a, cand_n, cand_p, Yw0, picks, vbuf, counter);
}

// Step j: positions j and picks[j] swap; every active position pos > j takes
// source column (pos == pick ? j : pos) of Yin, gets H_j applied on rows
// j..l-1, and rows j+1.. go to Yout with their squared norm.
template <typename T>
__global__ void __launch_bounds__(YT) k_ypick_step(int j, YArgs a, const T* __restrict__ Yin, T* __restrict__ Yout,
                                                   const T* vin, T* vout, T* cand_n, int* cand_p, int* picks,
                                                   int* counter) {
  extern __shared__ unsigned char smem_raw[];
  T* v = reinterpret_cast<T*>(smem_raw);  // [l]
  __shared__ T shn[NW];
  __shared__ int shp[NW];
  const int q = blockIdx.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int L = a.l - j;
  for (int r = threadIdx.x; r < L; r += YT) v[r] = vin[1 + r];
  const T tau = vin[0];
  const int pj = picks[j];
  __syncthreads();
  const int lo = max(q * a.per, j + 1), hi = min(a.np, q * a.per + a.per);
  T wn = T(-1);
  int wp = 0x7fffffff;
  for (int pos = lo + warp; pos < hi; pos += NW) {
    const int src = pos == pj ? j : pos;
    const T* y = Yin + (size_t)src * a.l + j;
    T* o = Yout + (size_t)pos * a.l + j;
    T x[5];
    T dot = T(0);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const int r = lane + 32 * t;
      x[t] = r < L ? y[r] : T(0);
      dot += r < L ? v[r] * x[t] : T(0);
    }
    for (int r = lane + 160; r < L; r += 32) dot += v[r] * y[r];  // l > 160
    dot = warp_sum(dot) * tau;
    T s = T(0);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const int r = lane + 32 * t;
      if (r < L) {
        const T nx = x[t] - dot * v[r];
        if (r >= 1) {
          o[r] = nx;
          s += nx * nx;
        }
      }
    }
    for (int r = lane + 160; r < L; r += 32) {
      const T nx = y[r] - dot * v[r];
      o[r] = nx;
      s += nx * nx;
    }
    s = warp_sum(s);
    if (s > wn || (s == wn && pos < wp)) {
      wn = s;
      wp = pos;
    }
  }
  T bn;
  int bp;
  cta_best(wn, wp, shn, shp, bn, bp);
  if (threadIdx.x == 0) {
    cand_n[q] = bn;
    cand_p[q] = bp;
  }
  if (y_last_cta(counter)) pick_and_reflect<T>(j + 1, a, cand_n, cand_p, Yout, picks, vout, counter);
}

// ------------------------------------------------------------ swaps
// Replays the swaps (j, picks[j]), j = 0..kb-1, on the touched positions and
// emits (dst, src) pairs of the net permutation: imap[0] = count, then pairs.
// Positions below kb map to their own slot; the at most kb others go through
// an open-addressing hash table in shared memory, so the replay is O(kb).
// When the status word is already set (a pivot step gave up, so picks may be
// stale) or a pick lies outside [j, np), no swap is made: imap[0] = 0.
constexpr int kMapHash = 2048;  // >= 4 kb for kb <= 512
__global__ void k_build_map(int kb, int np, const int* picks, int* imap, int* status) {
  extern __shared__ int sh[];
  const bool failed = *(volatile int*)status != 0;  // set by an earlier kernel of the stream
  int bad = 0;
  for (int j = threadIdx.x; j < kb; j += blockDim.x)
    if (picks[j] < j || picks[j] >= np) bad = 1;
  bad = __syncthreads_or(bad);
  if (failed || bad) {
    if (threadIdx.x == 0) {
      imap[0] = 0;
      if (!failed) atomicCAS(status, 0, RQR_ERR_CUDA);
    }
    return;
  }
  int* cont = sh;               // [kb] content of positions 0..kb-1
  int* hkey = sh + kb;          // [kMapHash] position, -1 = empty
  int* hval = hkey + kMapHash;  // [kMapHash] content
  for (int e = threadIdx.x; e < kb; e += blockDim.x) cont[e] = e;
  for (int e = threadIdx.x; e < kMapHash; e += blockDim.x) hkey[e] = -1;
  __syncthreads();
  auto slot = [&](int p) -> int* {
    if (p < kb) return cont + p;
    unsigned h = ((unsigned)p * 2654435761u) & (kMapHash - 1);
    while (hkey[h] != -1 && hkey[h] != p) h = (h + 1) & (kMapHash - 1);
    if (hkey[h] == -1) {
      hkey[h] = p;
      hval[h] = p;
    }
    return hval + h;
  };
  if (threadIdx.x == 0)
    for (int j = 0; j < kb; ++j) {
      const int pk = picks[j];
      if (pk == j) continue;
      int* a = slot(j);
      int* b = slot(pk);
      const int t = *a;
      *a = *b;
      *b = t;
    }
  __syncthreads();
  // emit the moved positions with all threads (the pairs are independent, so
  // their order in imap does not matter)
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (int e = threadIdx.x; e < kb; e += blockDim.x)
    if (cont[e] != e) {
      const int t = atomicAdd(&s_n, 1);
      imap[1 + 2 * t] = e;
      imap[2 + 2 * t] = cont[e];
    }
  for (int h = threadIdx.x; h < kMapHash; h += blockDim.x)
    if (hkey[h] != -1 && hval[h] != hkey[h]) {
      const int t = atomicAdd(&s_n, 1);
      imap[1 + 2 * t] = hkey[h];
      imap[2 + 2 * t] = hval[h];
    }
  __syncthreads();
  if (threadIdx.x == 0) imap[0] = s_n;
}

template <typename T>
__global__ void k_gather(const int* imap, int m, const T* A, int lda, int k0, int l, const T* Y, int ldy, int y0,
                         const int32_t* perm, T* tmpA, T* tmpY, int32_t* tmpP) {
  const int t = blockIdx.y;
  if (t >= imap[0]) return;
  const int src = imap[2 + 2 * t];
  const T* a = A + (size_t)(k0 + src) * lda;
  T* o = tmpA + (size_t)t * m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) o[i] = a[i];
  if (Y && blockIdx.x == 0) {
    const T* y = Y + (size_t)(y0 + src) * ldy;
    for (int i = threadIdx.x; i < l; i += blockDim.x) tmpY[(size_t)t * l + i] = y[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) tmpP[t] = perm[k0 + src];
}

template <typename T>
__global__ void k_scatter(const int* imap, int m, T* A, int lda, int k0, int l, T* Y, int ldy, int y0, int32_t* perm,
                          const T* tmpA, const T* tmpY, const int32_t* tmpP) {
  const int t = blockIdx.y;
  if (t >= imap[0]) return;
  const int dst = imap[1 + 2 * t];
  T* a = A + (size_t)(k0 + dst) * lda;
  const T* s = tmpA + (size_t)t * m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) a[i] = s[i];
  if (Y && blockIdx.x == 0) {
    T* y = Y + (size_t)(y0 + dst) * ldy;
    for (int i = threadIdx.x; i < l; i += blockDim.x) y[i] = tmpY[(size_t)t * l + i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) perm[k0 + dst] = tmpP[t];
}

// Four CTAs per SM: each warp then handles only a few positions per step, so
// the chain of dependent L2 round trips inside a step stays short.
void ygeometry(int np, int sms, int& C, int& per) {
  C = std::max(1, std::min(4 * sms, ceil_div(np, 8)));
  per = ceil_div(std::max(np, 1), C);
  C = ceil_div(std::max(np, 1), per);
}

}  // namespace

template <typename T>
size_t ypick_scratch_elems(int l, int np, int b, int sms) {
  int C, per;
  ygeometry(np, sms, C, per);
  // Yw ping/pong, 2 vbufs, cand_n, cand_p (as T), counter
  return 2 * (size_t)l * np + 2 * (size_t)(l + 2) + 2 * (size_t)C + 64;
}

template <typename T>
void ypick(const Ctx& c, int l, int np, int bsteps, const T* Y, int ldy, int* picks, T* scratch) {
  if (bsteps <= 0 || np <= 0) return;
  int C, per;
  ygeometry(np, c.sms, C, per);
  T* yw0 = scratch;
  T* yw1 = yw0 + (size_t)l * np;
  T* vb0 = yw1 + (size_t)l * np;
  T* vb1 = vb0 + (l + 2);
  T* cand_n = vb1 + (l + 2);
  int* cand_p = reinterpret_cast<int*>(cand_n + C);
  int* counter = cand_p + C + 2;
  counter = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(counter) + 15) & ~uintptr_t(15));
  cudaMemsetAsync(counter, 0, sizeof(int), c.stream);
  YArgs a{l, np, per};
  k_ypick_init<T><<<C, YT, 0, c.stream>>>(a, Y, ldy, yw0, cand_n, cand_p, picks, vb0, counter);
  note_launch(c, bsteps);
  for (int j = 0; j + 1 < bsteps; ++j) {
    const T* yin = (j & 1) ? yw1 : yw0;
    T* yout = (j & 1) ? yw0 : yw1;
    const T* vin = (j & 1) ? vb1 : vb0;
    T* vout = (j & 1) ? vb0 : vb1;
    k_ypick_step<T><<<C, YT, sizeof(T) * l, c.stream>>>(j, a, yin, yout, vin, vout, cand_n, cand_p, picks, counter);
  }
}

template <typename T>
void apply_swaps(const Ctx& c, int kb, int np, const int* picks, int m, T* A, int lda, int k0, int l, T* Y, int ldy,
                 int y0, int32_t* perm, T* tmp, int* imap) {
  if (kb <= 0) return;
  k_build_map<<<1, 256, sizeof(int) * ((size_t)kb + 2 * kMapHash), c.stream>>>(kb, np, picks, imap, c.status);
  T* tmpA = tmp;
  T* tmpY = tmpA + (size_t)m * 2 * kb;
  int32_t* tmpP = reinterpret_cast<int32_t*>(tmpY + (size_t)l * 2 * kb);
  dim3 grid(std::max(1, std::min(ceil_div(m, 256), 16)), 2 * kb);
  k_gather<T><<<grid, 256, 0, c.stream>>>(imap, m, A, lda, k0, l, Y, ldy, y0, perm, tmpA, tmpY, tmpP);
  k_scatter<T><<<grid, 256, 0, c.stream>>>(imap, m, A, lda, k0, l, Y, ldy, y0, perm, tmpA, tmpY, tmpP);
  note_launch(c, 3);
}

#define RQR_INST(T)                                                                                      \
  template size_t ypick_scratch_elems<T>(int, int, int, int);                                           \
  template void ypick<T>(const Ctx&, int, int, int, const T*, int, int*, T*);                             \
  template void apply_swaps<T>(const Ctx&, int, int, const int*, int, T*, int, int, int, T*, int, int, int32_t*, \
                               T*, int*);
RQR_INST(double)
RQR_INST(float)
#undef RQR_INST

}  // namespace rqr
