// persist.cu -- the b pivot steps of the sketch (Sec. 4.1 with the
// over-sampling of Sec. 4.3: first b steps of Fig. QR on the l x n' sketch) as
// ONE cooperative launch instead of one launch per step.
//
// Every CTA keeps the sketch columns of its fixed range of positions resident
// in shared memory for all b steps (l x ~108 FP64 values per SM at n' = 16384),
// so a step reads no global memory except the reflector and the column that
// the swap brings in. Steps are separated by a grid barrier: the last CTA to
// arrive picks the largest remaining norm (lowest position on ties), builds
// the next reflector from the candidate column the winning CTA published, and
// releases the others. Waiting CTAs spin with a bounded count; a wait that
// runs out sets RQR_ERR_TIMEOUT in the status word and every CTA returns at
// the next barrier (co-residency is guaranteed by the cooperative launch, so
// this only guards against a defect).
#include <algorithm>

#include "common.cuh"
#include "panel_common.cuh"

namespace rqr {

namespace {

constexpr int PT = 256, PNW = PT / 32;
constexpr unsigned kMaxSpins = 1u << 24;  // x ~100 ns sleep: ~2 s

struct GridSync {
  unsigned count, gen;
  int err, pad;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Arrive; returns true in the last CTA to arrive (the caller then does the
// step's serial work and calls grid_release). Others wait for the release.
__device__ bool grid_arrive(GridSync* gs, unsigned& gen_seen) {
  __shared__ int s_last;
  __shared__ unsigned s_gen;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = ld_acquire(&gs->gen);
    __threadfence();
    const unsigned t = atomicAdd(&gs->count, 1u);
    s_last = (t == gridDim.x - 1) ? 1 : 0;
    s_gen = g;
  }
  __syncthreads();
  gen_seen = s_gen;
  if (s_last) __threadfence();
  return s_last != 0;
}

__device__ void grid_release(GridSync* gs, unsigned gen_seen) {
  __syncthreads();
  if (threadIdx.x == 0) {
    gs->count = 0;
    __threadfence();
    st_release(&gs->gen, gen_seen + 1);
  }
}

// Waits for the release of generation gen_seen; false when the wait ran out
// or another CTA reported one.
__device__ bool grid_wait(GridSync* gs, unsigned gen_seen, int* status) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    unsigned spins = 0;
    int ok = 1;
    while (ld_acquire(&gs->gen) == gen_seen) {
      if (++spins > kMaxSpins || *(volatile int*)&gs->err) {
        atomicExch(&gs->err, 1);
        atomicCAS(status, 0, RQR_ERR_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(100);
    }
    if (*(volatile int*)&gs->err) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename T>
struct PArgs {
  int l, np, per, bsteps;
  const T* Y;
  int ldy;
  int* picks;
  T* cand_n;
  int* cand_p;
  T* candcol;  // [C][l]
  T* vbuf;     // [l + 2]
  T* colbuf;   // [2][l]
  GridSync* gs;
  int* status;
};

// Last CTA: global best over the CTA candidates, pick, and the reflector of
// rows j..l-1 of the winner's published column.
template <typename T>
__device__ void reduce_pick(int j, const PArgs<T>& a) {
  __shared__ T sn[PT];
  __shared__ int sp[PT], sq[PT];
  const int tid = threadIdx.x, lane = tid & 31;
  T bn = T(-1);
  int bp = 0x7fffffff, bq = 0;
  for (int q = tid; q < (int)gridDim.x; q += PT) {
    const T n = __ldcg(a.cand_n + q);
    const int p = __ldcg(a.cand_p + q);
    if (n > bn || (n == bn && p < bp)) {
      bn = n;
      bp = p;
      bq = q;
    }
  }
  sn[tid] = bn;
  sp[tid] = bp;
  sq[tid] = bq;
  __syncthreads();
  for (int half = PT / 2; half > 0; half >>= 1) {
    if (tid < half && (sn[tid + half] > sn[tid] || (sn[tid + half] == sn[tid] && sp[tid + half] < sp[tid]))) {
      sn[tid] = sn[tid + half];
      sp[tid] = sp[tid + half];
      sq[tid] = sq[tid + half];
    }
    __syncthreads();
  }
  if (tid < 32) {
    const T* y = a.candcol + (size_t)sq[0] * a.l;
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
    for (int r = 1 + lane; r < L; r += 32) a.vbuf[1 + r] = tau == T(0) ? T(0) : __ldcg(y + j + r) / d;
    if (lane == 0) {
      a.vbuf[0] = tau;
      a.vbuf[1] = T(1);
      a.picks[j] = sp[0];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(PT) k_ypick_persist(PArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = a.l;
  T* tile = reinterpret_cast<T*>(smem_raw);  // [per][l]
  T* v = tile + (size_t)a.per * l;            // [l]
  __shared__ T shn[PNW];
  __shared__ int shp[PNW];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int lo = q * a.per, hi = min(a.np, lo + a.per), cnt = max(0, hi - lo);
  for (int e = tid; e < cnt * l; e += PT) {
    const int pl = e / l, r = e % l;
    tile[e] = a.Y[(size_t)(lo + pl) * a.ldy + r];
  }
  __syncthreads();
  // full column norms, CTA candidate
  T wn = T(-1);
  int wp = 0x7fffffff;
  for (int pl = warp; pl < cnt; pl += PNW) {
    const T* y = tile + (size_t)pl * l;
    T s = T(0);
    for (int r = lane; r < l; r += 32) s += y[r] * y[r];
    s = warp_sum(s);
    if (s > wn || (s == wn && lo + pl < wp)) {
      wn = s;
      wp = lo + pl;
    }
  }
  int j = -1;
  for (;;) {
    // ---- publish this CTA's candidate (value, position, column rows j+1..)
    if (lane == 0) {
      shn[warp] = wn;
      shp[warp] = wp;
    }
    __syncthreads();
    T bn = T(-1);
    int bp = 0x7fffffff;
    for (int w = 0; w < PNW; ++w)
      if (shn[w] > bn || (shn[w] == bn && shp[w] < bp)) {
        bn = shn[w];
        bp = shp[w];
      }
    if (tid == 0) {
      a.cand_n[q] = bn;
      a.cand_p[q] = bp;
    }
    if (bp >= lo && bp < hi)
      for (int r = j + 1 + tid; r < l; r += PT) a.candcol[(size_t)q * l + r] = tile[(size_t)(bp - lo) * l + r];
    // the content of position j+1 moves to the next pivot's position: publish it
    if (j + 2 < a.bsteps + 1 && j + 1 >= lo && j + 1 < hi)
      for (int r = j + 1 + tid; r < l; r += PT)
        a.colbuf[(size_t)((j + 1) & 1) * l + r] = tile[(size_t)(j + 1 - lo) * l + r];
    unsigned gen;
    if (grid_arrive(a.gs, gen)) {
      reduce_pick<T>(j + 1, a);
      grid_release(a.gs, gen);
    } else if (!grid_wait(a.gs, gen, a.status)) {
      return;
    }
    ++j;  // now step j: positions j and picks[j] swap, reflector j applies
    if (j + 1 >= a.bsteps) break;
    // ---- step j
    const int pj = __ldcg(a.picks + j);
    const int L = l - j;
    for (int r = tid; r < L; r += PT) v[r] = __ldcg(a.vbuf + 1 + r);
    const T tau = __ldcg(a.vbuf);
    if (pj != j && pj >= lo && pj < hi)
      for (int r = j + tid; r < l; r += PT) tile[(size_t)(pj - lo) * l + r] = __ldcg(a.colbuf + (size_t)(j & 1) * l + r);
    __syncthreads();
    wn = T(-1);
    wp = 0x7fffffff;
    for (int pl = max(0, j + 1 - lo) + warp; pl < cnt; pl += PNW) {
      T* y = tile + (size_t)pl * l + j;
      T dot = T(0);
      for (int r = lane; r < L; r += 32) dot += v[r] * y[r];
      dot = warp_sum(dot) * tau;
      T s = T(0);
      for (int r = lane; r < L; r += 32) {
        const T nx = y[r] - dot * v[r];
        y[r] = nx;
        if (r >= 1) s += nx * nx;
      }
      s = warp_sum(s);
      if (s > wn || (s == wn && lo + pl < wp)) {
        wn = s;
        wp = lo + pl;
      }
    }
  }
}

// ------------------------------------------------------------ panel
// Householder QR of an mp x nc panel (Sec. 3.2) as one cooperative launch:
// each CTA keeps its rows of all nc columns in shared memory for the whole
// panel; per column the same fused update / next-column partial sums as the
// multi-launch k_panel_step (panel.cu), separated by the grid barrier, whose
// last arriver prepares the next column's coefficients.
template <typename T>
struct QArgs {
  int mp, nc, R;
  T* P;
  int ldp;
  T* tau;
  T* part;    // [C][nc + 1]
  T* rowbuf;  // [2][nc]
  T* coef;    // [2][NCOEF + nc]
  GridSync* gs;
  int* status;
};

template <typename T>
__global__ void __launch_bounds__(pnl::PT) k_panel_persist(QArgs<T> a) {
  using namespace pnl;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nc = a.nc, R = a.R;
  T* w = reinterpret_cast<T*>(smem_raw);  // [nc]
  T* tile = w + nc;                       // [nc][R]: tile[c * R + rr] = P(r0 + rr, c)
  __shared__ T wsum[PT / 32];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = q * R, r1 = min(a.mp, r0 + R), nr = max(0, r1 - r0);
  const PanelArgs pa{a.mp, nc, R, a.ldp};
  for (int e = tid; e < nr * nc; e += PT) {
    const int rr = e % nr, cc = e / nr;
    tile[cc * R + rr] = a.P[r0 + rr + (size_t)cc * a.ldp];
  }
  __syncthreads();
  // partials of column 0 (below the diagonal) and row 0
  {
    T* myp = a.part + (size_t)q * (nc + 1);
    T s = T(0);
    for (int rr = tid; rr < nr; rr += PT)
      if (r0 + rr > 0) s += tile[rr] * tile[rr];
    s = block_sum(s, wsum);
    if (tid == 0) myp[0] = s;
    for (int c = 1 + warp; c < nc; c += PT / 32) {
      T acc = T(0);
      for (int rr = lane; rr < nr; rr += 32)
        if (r0 + rr > 0) acc += tile[rr] * tile[(size_t)c * R + rr];
      acc = warp_sum(acc);
      if (lane == 0) myp[1 + c] = acc;
    }
    if (r0 == 0 && nr > 0)
      for (int c = tid; c < nc; c += PT) a.rowbuf[c] = tile[(size_t)c * R];
    unsigned gen;
    if (grid_arrive(a.gs, gen)) {
      finish_coef<T>(0, pa, a.part, a.rowbuf, a.coef, a.tau, a.status, w);
      grid_release(a.gs, gen);
    } else if (!grid_wait(a.gs, gen, a.status)) {
      return;
    }
  }
  for (int j = 0; j < nc; ++j) {
    const T* cin = a.coef + (size_t)(j & 1) * (NCOEF + nc);
    for (int c = tid; c < nc; c += PT) w[c] = c > j ? __ldcg(cin + NCOEF + c) : T(0);
    const T tauj = __ldcg(cin), beta = __ldcg(cin + 1), d = __ldcg(cin + 2);
    const bool has = __ldcg(cin + 3) != T(0);
    const int lo = min(nr, max(0, j - r0));
    T* tj = tile + (size_t)j * R;
    __syncthreads();
    for (int rr = lo + tid; rr < nr; rr += PT) {
      const int i = r0 + rr;
      if (i > j) {
        if (has) tj[rr] = tauj == T(0) ? T(0) : tj[rr] / d;
      } else if (has) {
        tj[rr] = beta;
      }
    }
    __syncthreads();
    if (j + 1 >= nc) break;
    T* t1 = tile + (size_t)(j + 1) * R;
    const T w1 = w[j + 1];
    for (int rr = lo + tid; rr < nr; rr += PT) {
      const int i = r0 + rr;
      t1[rr] -= w1 * (i == j ? T(1) : tj[rr]);
    }
    __syncthreads();
    T* myp = a.part + (size_t)q * (nc + 1);
    T s = T(0);
    for (int rr = lo + tid; rr < nr; rr += PT)
      if (r0 + rr > j + 1) s += t1[rr] * t1[rr];
    s = block_sum(s, wsum);
    if (tid == 0) myp[0] = s;
    for (int c = j + 2 + warp; c < nc; c += PT / 32) {
      T* x = tile + (size_t)c * R;
      const T wc = w[c];
      T acc = T(0);
      for (int rr = lo + lane; rr < nr; rr += 32) {
        const int i = r0 + rr;
        const T xv = x[rr] - wc * (i == j ? T(1) : tj[rr]);
        x[rr] = xv;
        if (i > j + 1) acc += t1[rr] * xv;
      }
      acc = warp_sum(acc);
      if (lane == 0) myp[1 + c] = acc;
    }
    __syncthreads();
    T* rb = a.rowbuf + (size_t)((j + 1) & 1) * nc;
    if (j + 1 >= r0 && j + 1 < r1)
      for (int c = j + 1 + tid; c < nc; c += PT) rb[c] = tile[(size_t)c * R + (j + 1 - r0)];
    unsigned gen;
    if (grid_arrive(a.gs, gen)) {
      finish_coef<T>(j + 1, pa, a.part, rb, a.coef + (size_t)((j + 1) & 1) * (NCOEF + nc), a.tau, a.status, w);
      grid_release(a.gs, gen);
    } else if (!grid_wait(a.gs, gen, a.status)) {
      return;
    }
  }
  __syncthreads();
  for (int e = tid; e < nr * nc; e += PT) {
    const int rr = e % nr, cc = e / nr;
    a.P[r0 + rr + (size_t)cc * a.ldp] = tile[cc * R + rr];
  }
}

}  // namespace

// Householder QR of the mp x nc panel as one cooperative launch; false (and
// nothing queued) when the rows of one CTA do not fit in shared memory or the
// grid cannot be co-scheduled. scratch: the panel scratch of panel.cu.
template <typename T>
bool panel_qr_persist(const Ctx& c, int mp, int nc, T* P, int ldp, T* tau, T* scratch, int C, int R) {
  if (mp <= 0 || nc <= 0) return true;
  const size_t smem = sizeof(T) * ((size_t)nc + (size_t)nc * R);
  if (smem > 200 * 1024 || C > c.sms) return false;
  static int attr_set = 0;
  if (!attr_set) {
    cudaFuncSetAttribute(k_panel_persist<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_panel_persist<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_panel_persist<T>, pnl::PT, smem) != cudaSuccess ||
      per_sm * c.sms < C) {
    cudaGetLastError();
    return false;
  }
  T* part = scratch;
  T* rowbuf = part + (size_t)C * (nc + 1);
  T* coef = rowbuf + 2 * (size_t)nc;
  T* tail = coef + 2 * (size_t)(pnl::NCOEF + nc);
  GridSync* gs = reinterpret_cast<GridSync*>((reinterpret_cast<uintptr_t>(tail) + 15) & ~uintptr_t(15));
  cudaMemsetAsync(gs, 0, sizeof(GridSync), c.stream);
  QArgs<T> a{mp, nc, R, P, ldp, tau, part, rowbuf, coef, gs, c.status};
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)k_panel_persist<T>, dim3(C), dim3(pnl::PT), args, smem, c.stream) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  note_launch(c);
  return true;
}

template bool panel_qr_persist<double>(const Ctx&, int, int, double*, int, double*, double*, int, int);
template bool panel_qr_persist<float>(const Ctx&, int, int, float*, int, float*, float*, int, int);

// Shared memory per CTA for n' positions spread over `sms` CTAs.
static size_t persist_smem(int l, int np, int sms, int& C, int& per) {
  C = std::max(1, std::min(sms, ceil_div(np, 8)));
  per = ceil_div(std::max(np, 1), C);
  C = ceil_div(std::max(np, 1), per);
  return sizeof(double) * ((size_t)per * l + l);
}

size_t ypick_persist_scratch_bytes(int l, int np, int sms) {
  int C, per;
  persist_smem(l, np, sms, C, per);
  return 64 + sizeof(double) * ((size_t)C * (l + 1) + 3 * (size_t)l + 16) + sizeof(int) * (size_t)C + 256;
}

// Returns false (and queues nothing) when the sketch slice does not fit in
// shared memory or the device cannot co-schedule the grid.
template <typename T>
bool ypick_persist(const Ctx& c, int l, int np, int bsteps, const T* Y, int ldy, int* picks, void* scratch) {
  if (bsteps <= 0 || np <= 0) return true;
  int C, per;
  const size_t smem = persist_smem(l, np, c.sms, C, per) / sizeof(double) * sizeof(T);
  if (smem > 200 * 1024) return false;
  static int attr_set = 0;
  if (!attr_set) {
    cudaFuncSetAttribute(k_ypick_persist<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_ypick_persist<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ypick_persist<T>, PT, smem) != cudaSuccess ||
      per_sm * c.sms < C) {
    cudaGetLastError();
    return false;
  }
  char* p = static_cast<char*>(scratch);
  GridSync* gs = reinterpret_cast<GridSync*>(p);
  p += 64;
  T* cand_n = reinterpret_cast<T*>(p);
  T* candcol = cand_n + C;
  T* vbuf = candcol + (size_t)C * l;
  T* colbuf = vbuf + l + 2;
  int* cand_p = reinterpret_cast<int*>(colbuf + 2 * (size_t)l + 8);
  cudaMemsetAsync(gs, 0, sizeof(GridSync), c.stream);
  PArgs<T> a{l, np, per, bsteps, Y, ldy, picks, cand_n, cand_p, candcol, vbuf, colbuf, gs, c.status};
  void* args[] = {&a};
  if (cudaLaunchCooperativeKernel((const void*)k_ypick_persist<T>, dim3(C), dim3(PT), args, smem, c.stream) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  note_launch(c);
  return true;
}

template bool ypick_persist<double>(const Ctx&, int, int, int, const double*, int, int*, void*);
template bool ypick_persist<float>(const Ctx&, int, int, int, const float*, int, int*, void*);

}  // namespace rqr
