// persist.cu -- the two latency-bound steps of every block as single
// cooperative launches: the b pivot steps on the sketch (Sec. 4.1 with the
// over-sampling of Sec. 4.3: first b steps of Fig. QR on the l x n' sketch)
// and the Householder QR of the m' x b panel (Sec. 3.2).
//
// Each CTA keeps its slice resident in shared memory for all steps (sketch
// columns of a fixed range of positions; panel rows of a fixed range), so a
// step reads no global memory except the few values the CTAs exchange. The
// values are exchanged as flagged 8-byte words (32 data bits and the step's
// tag), so a reader waits for exactly the words it needs, with no grid
// barrier or fence; they are reduced by every CTA (pivot winner) or by one CTA
// per entry (panel sums) in a fixed order, so results do not depend on timing.
// Waits are bounded by the handle's wait limit (2 s of global time unless the
// caller sets another); a wait that runs out sets RQR_ERR_TIMEOUT in the
// status word and every CTA returns (co-residency is guaranteed by the
// cooperative launch, so with the default limit this only guards against a
// defect). A kernel launched after the status word was set returns at once:
// the picks and panel values of an aborted step are never used.
#include <algorithm>

#include "common.cuh"
#include "panel_common.cuh"

namespace rqr {

namespace {

constexpr int PT = 256, PNW = PT / 32;
constexpr double kRecompute = 1.0 / 1024.0;  // pivot norms: recompute below this fraction of the last exact one

__device__ __forceinline__ uint64_t gtime_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ------------------------------------------------------------ flagged words
// The pivot kernel exchanges its values as 8-byte words that carry 32 bits of
// data and a 32-bit tag (the step + 1): one 64-bit store is seen whole or not
// at all, so a reader that finds the step's tag in a word has that word's
// data, without a fence or an arrival counter. A double takes two words
// (low, high half), a float one. The words are zeroed before every launch, so
// no stale word carries a tag of the launch.
typedef unsigned long long llw;

__device__ __forceinline__ void ll_store(llw* w, uint32_t data, uint32_t tag) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(w), "l"(((llw)tag << 32) | data) : "memory");
}
__device__ __forceinline__ llw ll_load(const llw* w) {
  llw v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
  return v;
}
// Waits until the word carries `tag`; false when the wait limit ran out or
// the CTA was told to give up (*fail set by another thread).
__device__ __forceinline__ bool ll_wait(const llw* w, uint32_t tag, uint32_t& data, unsigned long long limit_ns,
                                        volatile int* fail) {
  llw v = ll_load(w);
  if ((uint32_t)(v >> 32) != tag) {
    const uint64_t t0 = gtime_ns();
    while ((uint32_t)((v = ll_load(w)) >> 32) != tag) {
      if (*fail || gtime_ns() - t0 > limit_ns) {
        *fail = 1;
        return false;
      }
    }
  }
  data = (uint32_t)v;
  return true;
}

// Two adjacent words (16-byte aligned) with one vector load: the two halves
// arrive together instead of one L2 round trip after the other.
__device__ __forceinline__ void ll_load2(const llw* w, llw& x, llw& y) {
  asm volatile("ld.volatile.global.v2.u64 {%0, %1}, [%2];" : "=l"(x), "=l"(y) : "l"(w) : "memory");
}
// Waits until both words at w (16-byte aligned) carry `tag`.
__device__ __forceinline__ bool ll_wait2(const llw* w, uint32_t tag, uint32_t& d0, uint32_t& d1,
                                         unsigned long long limit_ns, volatile int* fail) {
  llw x, y;
  ll_load2(w, x, y);
  if ((uint32_t)(x >> 32) != tag || (uint32_t)(y >> 32) != tag) {
    const uint64_t t0 = gtime_ns();
    while (true) {
      ll_load2(w, x, y);
      if ((uint32_t)(x >> 32) == tag && (uint32_t)(y >> 32) == tag) break;
      if (*fail || gtime_ns() - t0 > limit_ns) {
        *fail = 1;
        return false;
      }
    }
  }
  d0 = (uint32_t)x;
  d1 = (uint32_t)y;
  return true;
}

// Waits until the four words of a 32-byte slot carry `tag` (two vector loads
// issued together per try).
__device__ __forceinline__ bool ll_wait4(const llw* w, uint32_t tag, uint32_t d[4], unsigned long long limit_ns,
                                         volatile int* fail) {
  llw x[4];
  auto ready = [&]() {
    ll_load2(w, x[0], x[1]);
    ll_load2(w + 2, x[2], x[3]);
    return (uint32_t)(x[0] >> 32) == tag && (uint32_t)(x[1] >> 32) == tag && (uint32_t)(x[2] >> 32) == tag &&
           (uint32_t)(x[3] >> 32) == tag;
  };
  if (!ready()) {
    const uint64_t t0 = gtime_ns();
    while (!ready()) {
      if (*fail || gtime_ns() - t0 > limit_ns) {
        *fail = 1;
        return false;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) d[i] = (uint32_t)x[i];
  return true;
}

template <typename T>
__device__ __forceinline__ void ll_put(llw* w, T x, uint32_t tag) {
  if constexpr (sizeof(T) == 8) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    ll_store(w, (uint32_t)b, tag);
    ll_store(w + 1, (uint32_t)(b >> 32), tag);
  } else {
    ll_store(w, __float_as_uint(x), tag);
  }
}
template <typename T>
__device__ __forceinline__ bool ll_get(const llw* w, uint32_t tag, T& x, unsigned long long limit_ns,
                                       volatile int* fail) {
  uint32_t lo = 0, hi = 0;
  if constexpr (sizeof(T) == 8) {
    if (!ll_wait2(w, tag, lo, hi, limit_ns, fail)) return false;
    x = __longlong_as_double((long long)(((unsigned long long)hi << 32) | lo));
  } else {
    if (!ll_wait(w, tag, lo, limit_ns, fail)) return false;
    x = __uint_as_float(lo);
  }
  return true;
}

template <typename T>
struct PArgs {
  int l, np, per, bsteps;
  const T* Y;
  int ldy;
  int* picks;
  llw* slots;   // [2][C][4] per CTA and step parity: key low, key high, position (flagged words)
  llw* col;     // [2][C][2 l] each CTA's candidate column, rows s.. (flagged words)
  llw* colbuf;  // [2][2 (l + 2)] the column leaving the pivot position, its norm and reference norm
  int* status;
  unsigned long long wait_ns;  // limit of each wait for another CTA's words
};

// Candidates compare by key: the bit pattern of a squared norm (>= 0) as a
// signed integer orders like the norm itself, and anything else (the empty
// candidate, NaN) gets -1. The comparisons then run on the integer pipe; as
// FP64 compares, every thread of every CTA spent ~20 clocks of the SM's FP64
// pipe on each of them per step.
// (-0.0 gets the key of +0.0.)
__device__ __forceinline__ long long norm_key(double n) {
  return n >= 0.0 ? (__double_as_longlong(n) & 0x7fffffffffffffffll) : -1ll;
}
__device__ __forceinline__ long long norm_key(float n) { return n >= 0.f ? (long long)(__float_as_int(n) & 0x7fffffff) : -1ll; }

// Better candidate: larger squared norm, lower position on ties.
__device__ __forceinline__ bool better(long long k, int p, long long bk, int bp) {
  return k > bk || (k == bk && p < bp);
}

// b steps of Fig. QR on the sketch. Per step s every CTA publishes its best
// remaining column (squared norm of rows s.., position, values) as flagged
// words, waits for the C published candidates (one thread per CTA slot), picks
// the global winner itself (same data and order in every CTA, so the same
// winner), reads the winner's values, builds the reflector and applies it to
// its own columns. Two L2 round trips per step (the slots, then the winner's
// column), no grid barrier, no fence, and no serial phase in a single CTA.
// The squared norms of rows s+1.. are downdated from those of rows s..
// (the reflector keeps the norm of rows s..: |y(s+1:)|^2 = |y(s:)|^2 - y_s^2,
// y_s after the update) and recomputed exactly from the column whenever the
// downdated value has fallen below kRecompute of the last exact one, which
// bounds the downdate's relative error by about u / kRecompute per step.
template <typename T>
__global__ void __launch_bounds__(PT) k_ypick_persist(PArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l = a.l, C = gridDim.x;
  const int LS = l | 1;                       // odd column stride: a thread per column reads without bank conflicts
  T* tile = reinterpret_cast<T*>(smem_raw);  // [per][LS]
  T* v = tile + (size_t)a.per * LS;           // [l]
  T* nrm = v + l;                             // [per] squared norm of rows s.. of each column
  T* ref = nrm + a.per;                       // [per] the last exactly computed squared norm
  T* dsh = ref + a.per;                       // [per] phase-A dot products of a step
  T* wsh = dsh + a.per;                       // [per] w_c rd of the last step for rows > s; 0 once applied
  const int LB = l + 2;                       // colbuf stride: values, norm, reference
  __shared__ long long shn[PNW];
  __shared__ int shp[PNW], shq[PNW];
  __shared__ T s_tau, s_rd;
  __shared__ int s_win, s_pos;
  __shared__ volatile int s_fail;  // a wait of this CTA gave up: the others stop waiting too
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // an earlier step of this call failed: nothing here may be trusted (every
  // CTA reads the same word before any of them can change it)
  if (*(volatile int*)a.status != 0) return;
  if (tid == 0) s_fail = 0;
  const int lo = q * a.per, hi = min(a.np, lo + a.per), cnt = max(0, hi - lo);
  for (int e = tid; e < cnt * l; e += PT) {
    const int pl = e / l, r = e % l;
    tile[(size_t)pl * LS + r] = a.Y[(size_t)(lo + pl) * a.ldy + r];
  }
  __syncthreads();
  // full column norms, warp candidates
  long long wn = -1;
  int wp = 0x7fffffff;
  for (int pl = warp; pl < cnt; pl += PNW) {
    const T* y = tile + (size_t)pl * LS;
    T ss = T(0);
    for (int r = lane; r < l; r += 32) ss += y[r] * y[r];
    ss = warp_sum(ss);
    if (lane == 0) {
      nrm[pl] = ss;
      ref[pl] = ss;
    }
    if (better(norm_key(ss), lo + pl, wn, wp)) {
      wn = norm_key(ss);
      wp = lo + pl;
    }
  }
  for (int s = 0; s < a.bsteps; ++s) {
    const int par = s & 1;
    // ---- publish the CTA candidate and, if owned, the column at position s
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long n2 = __shfl_xor_sync(0xffffffffu, wn, o);
      const int p2 = __shfl_xor_sync(0xffffffffu, wp, o);
      if (better(n2, p2, wn, wp)) {
        wn = n2;
        wp = p2;
      }
    }
    if (lane == 0) {
      shn[warp] = wn;
      shp[warp] = wp;
    }
    __syncthreads();
    long long bn = -1;
    int bp = 0x7fffffff;
    for (int w = 0; w < PNW; ++w)
      if (better(shn[w], shp[w], bn, bp)) {
        bn = shn[w];
        bp = shp[w];
      }
    const uint32_t tag = (uint32_t)s + 1u;
    // The last step's reflector has been applied to row s-1 of every column
    // only (phase B); the rest of each column follows while this step's
    // candidates travel. The two columns published now (the CTA candidate and
    // the column at position s) get their rows s.. first.
    const int Lp = l - s + 1;  // rows s-1.. of the last step's reflector
    if (s > 0) {
      const int pc = warp == 0 ? bp : warp == 1 && s != bp ? s : -1;
      if (pc >= lo && pc < hi) {
        T* y = tile + (size_t)(pc - lo) * LS + (s - 1);
        const T wr = wsh[pc - lo];
        if (wr != T(0))
          for (int r = 1 + lane; r < Lp; r += 32) y[r] -= wr * v[r];
        __syncwarp();
        if (lane == 0) wsh[pc - lo] = T(0);
      }
      __syncthreads();
    }
    if (tid == 0) {
      llw* sl = a.slots + ((size_t)par * C + q) * 4;
      ll_store(sl, (uint32_t)(unsigned long long)bn, tag);
      ll_store(sl + 1, (uint32_t)((unsigned long long)bn >> 32), tag);
      ll_store(sl + 2, (uint32_t)bp, tag);
      ll_store(sl + 3, 0u, tag);
    }
    if (bp >= lo && bp < hi)
      for (int r = s + tid; r < l; r += PT)
        ll_put<T>(a.col + ((size_t)par * C + q) * 2 * l + 2 * r, tile[(size_t)(bp - lo) * LS + r], tag);
    if (s >= lo && s < hi) {
      llw* cb = a.colbuf + (size_t)par * 2 * LB;
      for (int r = s + tid; r < l; r += PT) ll_put<T>(cb + 2 * r, tile[(size_t)(s - lo) * LS + r], tag);
      if (tid == 0) {
        ll_put<T>(cb + 2 * l, nrm[s - lo], tag);
        ll_put<T>(cb + 2 * (l + 1), ref[s - lo], tag);
      }
    }
    // the last step's reflector on rows s.. of the remaining columns (the
    // winner of this step overwrites v only after the waits below), g threads
    // per column over all warps; not needed after the last pick
    if (s > 0 && s + 1 < a.bsteps) {
      const int firstp = max(0, s - lo);
      const int ncolp = cnt - firstp;
      int gp = 1;
      while (gp < 32 && ncolp * (2 * gp) <= PT) gp *= 2;
      const int lgp = __ffs(gp) - 1, kp = tid & (gp - 1);
      for (int base = firstp; base < cnt; base += PT >> lgp) {
        const int pl = base + (tid >> lgp);
        if (pl < cnt) {
          const T wr = wsh[pl];
          if (wr != T(0)) {
            T* y = tile + (size_t)pl * LS + (s - 1);
            for (int r = 1 + kp; r < Lp; r += gp) y[r] -= wr * v[r];
          }
        }
      }
    }
    // ---- global winner (every CTA, identical order): thread t waits for CTA
    // t's slot words of this step; no barrier, no fence, no counter
    long long cn = -1;
    int cp = 0x7fffffff, cq = 0;
    bool bad = false;
    for (int t = tid; t < C && !bad; t += PT) {
      const llw* sl = a.slots + ((size_t)par * C + t) * 4;
      // key halves and position in one 32-byte slot: two vector loads in flight together
      uint32_t d[4];
      if (!ll_wait4(sl, tag, d, a.wait_ns, &s_fail)) {
        bad = true;
        break;
      }
      const uint32_t k0 = d[0], k1 = d[1], pp = d[2];
      const long long n = (long long)(((unsigned long long)k1 << 32) | k0);
      if (better(n, (int)pp, cn, cp)) {
        cn = n;
        cp = (int)pp;
        cq = t;
      }
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) atomicCAS(a.status, 0, RQR_ERR_TIMEOUT);
      return;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long n2 = __shfl_xor_sync(0xffffffffu, cn, o);
      const int p2 = __shfl_xor_sync(0xffffffffu, cp, o);
      const int q2 = __shfl_xor_sync(0xffffffffu, cq, o);
      if (better(n2, p2, cn, cp)) {
        cn = n2;
        cp = p2;
        cq = q2;
      }
    }
    if (lane == 0) {
      shn[warp] = cn;
      shp[warp] = cp;
      shq[warp] = cq;
    }
    __syncthreads();
    if (tid == 0) {
      long long gn = shn[0];
      int gp = shp[0], gq = shq[0];
      for (int w = 1; w < PNW; ++w)
        if (better(shn[w], shp[w], gn, gp)) {
          gn = shn[w];
          gp = shp[w];
          gq = shq[w];
        }
      s_win = gq;
      s_pos = gp;
      if (q == 0) a.picks[s] = gp;
    }
    __syncthreads();
    const int qj = s_win, pw = s_pos;  // winning CTA and position (the same in every CTA)
    const llw* ycol = a.col + ((size_t)par * C + qj) * 2 * l;
    const int L = l - s;
    // the winner's rows s.. into v, and the column leaving position s into the
    // winner's position when this CTA owns it
    for (int r = tid; r < L && !bad; r += PT) {
      T x;
      if (!ll_get<T>(ycol + 2 * (s + r), tag, x, a.wait_ns, &s_fail)) bad = true;
      else v[r] = x;
    }
    if (pw != s && pw >= lo && pw < hi) {
      const llw* cb = a.colbuf + (size_t)par * 2 * LB;
      for (int r = s + tid; r < l && !bad; r += PT) {
        T x;
        if (!ll_get<T>(cb + 2 * r, tag, x, a.wait_ns, &s_fail)) bad = true;
        else tile[(size_t)(pw - lo) * LS + r] = x;
      }
      if (tid == 0 && !bad) {
        T x1, x2;
        if (ll_get<T>(cb + 2 * l, tag, x1, a.wait_ns, &s_fail) && ll_get<T>(cb + 2 * (l + 1), tag, x2, a.wait_ns, &s_fail)) {
          nrm[pw - lo] = x1;
          ref[pw - lo] = x2;
        } else {
          bad = true;
        }
      }
    }
    if (__syncthreads_or(bad)) {
      if (tid == 0) atomicCAS(a.status, 0, RQR_ERR_TIMEOUT);
      return;
    }
    if (s + 1 >= a.bsteps) break;  // the last pick needs no reflector
    // ---- reflector of rows s.. of the winner (Sec. 3.1, sign(0) = +1) and its
    // application to the remaining columns, in two phases, so that the scalar
    // chain of the reflector (a square root and two divisions, slow on GB300's
    // FP64 pipe) in the last warp overlaps the dot products in the others:
    //   A: d_c = sum_{r >= 1} x_r y_c(r), x = the winner's rows s.. as read;
    //   B: with v = (1, rd x_1, rd x_2, ...) and rd = 1 / (alpha - beta),
    //      w_c = tau (y_c(0) + rd d_c), y_c(0) -= w_c, y_c(r) -= (w_c rd) x_r.
    // Columns are spread over warps 0..PNW-2 with g threads per column (g a
    // power of two, a group never crosses a warp), so the FP64 work of a step
    // is spread over the SM's four sub-partitions however few columns remain.
    const int first = max(0, s + 1 - lo);
    const int ncol = cnt - first;
    int g = 1;
    while (g < 32 && ncol * (2 * g) <= (PNW - 1) * 32) g *= 2;
    const int lg = __ffs(g) - 1;
    const int span = ((PNW - 1) * 32) >> lg;  // columns per pass
    const int kk = tid & (g - 1);             // this thread's place in its column's group
    if (warp == PNW - 1) {
      T ss = T(0);
      for (int r = lane; r < L; r += 32) ss += v[r] * v[r];
      ss = warp_sum(ss);
      if (lane == 0) {
        const T alpha = v[0];
        T tau = T(0), rd = T(1);
        if (L >= 2 && ss > T(0)) {
          const T beta = -sgn0(alpha) * sqrt(ss);
          pnl::tau_and_rd(alpha, beta, alpha - beta, tau, rd);
        }
        s_tau = tau;
        s_rd = rd;
      }
    } else {
      for (int base = first; base < cnt; base += span) {
        const int pl = base + (tid >> lg);
        T d0 = T(0), d1 = T(0);
        if (pl < cnt) {
          const T* y = tile + (size_t)pl * LS + s;
          int r = 1 + kk;
          for (; r + g < L; r += 2 * g) {
            d0 += v[r] * y[r];
            d1 += v[r + g] * y[r + g];
          }
          if (r < L) d0 += v[r] * y[r];
        }
        T d = d0 + d1;
        for (int o = g >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (pl < cnt && kk == 0) dsh[pl] = d;
      }
    }
    __syncthreads();
    // ---- phase B: row s of every column, and the norms of rows s+1..
    // (downdated: the reflector keeps the norm of rows s.., so
    // |y(s+1:)|^2 = |y(s:)|^2 - y_s^2 with y_s updated). Rows s+1.. follow at
    // the next step's publication (w_c rd kept in wsh), except for a column
    // whose norm is recomputed exactly: the whole warp updates it first.
    const T tau = s_tau, rd = s_rd;
    wn = -1;
    wp = 0x7fffffff;
    if (warp < PNW - 1) {
      for (int base = first; base < cnt; base += span) {
        const int pl = base + (tid >> lg);
        const bool act = pl < cnt && kk == 0;
        T nn = T(-1);
        bool redo = false;
        if (act) {
          T* y = tile + (size_t)pl * LS + s;
          T y0 = y[0];
          const T wc = tau * (y0 + rd * dsh[pl]);
          y0 -= wc;
          y[0] = y0;
          wsh[pl] = wc * rd;
          nn = nrm[pl] - y0 * y0;
          redo = !(nn > kRecompute * ref[pl]);
        }
        unsigned m = __ballot_sync(0xffffffffu, redo);
        while (m) {
          // rows s+1.. of a leader's column, then their exact squared norm, by the whole warp
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int pc = base + (((tid & ~31) + src) >> lg);
          T* yc = tile + (size_t)pc * LS + s;
          __syncwarp();
          const T wr = wsh[pc];
          for (int r = 1 + lane; r < L; r += 32) yc[r] -= wr * v[r];
          __syncwarp();
          if (lane == 0) wsh[pc] = T(0);
          T ss = T(0);
          for (int r = 1 + lane; r < L; r += 32) ss += yc[r] * yc[r];
          ss = warp_sum(ss);
          if (lane == src) {
            nn = ss;
            ref[pc] = ss;
          }
        }
        if (act) {
          nrm[pl] = nn;
          const long long key = norm_key(nn);
          if (better(key, lo + pl, wn, wp)) {
            wn = key;
            wp = lo + pl;
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------ panel
// Arguments of the persistent panel QR below: the panel, its tau, and the
// exchange words (flagged like the pivot kernel's; per step parity: every
// CTA's partial sums, the totals, the published row).
template <typename T>
struct QArgs {
  int mp, nc, R;
  T* P;
  int ldp;
  T* tau;
  llw* pw;  // [2][C][nc + 1] values: CTA partials (entry 0: squared norm below the diagonal, 1 + c: dot with column c)
  llw* tw;  // [2][nc + 1] values: totals, entry e added up by CTA e mod C
  llw* rw;  // [2][nc] values: the row of the next reflector's diagonal, from the CTA that holds it
  int* status;
  unsigned long long wait_ns;  // limit of each wait for another CTA's words
};

// Householder QR of an mp x nc panel (Sec. 3.2) as one cooperative launch:
// each CTA keeps its rows of all nc columns in shared memory for the whole
// panel. Per column j: the CTAs update column j+1 and the columns after it and
// publish partial sums (squared norm of column j+1 below the diagonal, its
// dot products with the later columns) as flagged words; CTA e mod C waits
// for entry e of every CTA, adds them in CTA order and publishes the total;
// every CTA waits for the totals and the published row it needs and computes
// the next reflector's coefficients itself. No grid barrier and no fence: each
// word is waited for where it is used, and the totals of a step are complete
// only after every CTA has published that step's partials, so no CTA can
// overwrite a word of one parity while another still waits for it.
template <typename T>
__global__ void __launch_bounds__(pnl::PT) k_panel_persist(QArgs<T> a) {
  using namespace pnl;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int WV = sizeof(T) / 4;  // flagged words per value
  const int nc = a.nc, R = a.R, C = gridDim.x;
  T* w = reinterpret_cast<T*>(smem_raw);  // [nc]
  T* tile = w + nc;                       // [nc][RS]: tile[c * RS + rr] = P(r0 + rr, c)
  __shared__ T wsum[PT / 32];
  __shared__ T s_coef[NCOEF];
  __shared__ T s_rd;  // 1 / d of the current reflector: one division per column, not one per row
  __shared__ volatile int s_fail;  // a wait of this CTA gave up: the others stop waiting too
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // an earlier step failed: leave the panel as it is (no CTA of this launch
  // can set the word before every CTA has passed this point: the first
  // exchange waits for the partials of all of them)
  if (*(volatile int*)a.status != 0) return;
  if (tid == 0) s_fail = 0;
  const int RS = R | 1;  // odd column stride: a thread per column reads without bank conflicts
  const int r0 = q * R, r1 = min(a.mp, r0 + R), nr = max(0, r1 - r0);
  for (int e = tid; e < nr * nc; e += PT) {
    const int rr = e % nr, cc = e / nr;
    tile[(size_t)cc * RS + rr] = a.P[r0 + rr + (size_t)cc * a.ldp];
  }
  __syncthreads();
  auto pword = [&](int par, int cta, int e) { return a.pw + ((size_t)(par * C + cta) * (nc + 1) + e) * WV; };
  auto tword = [&](int par, int e) { return a.tw + ((size_t)par * (nc + 1) + e) * WV; };
  auto rword = [&](int par, int c) { return a.rw + ((size_t)par * nc + c) * WV; };
  auto fail = [&]() {
    if (tid == 0) atomicCAS(a.status, 0, RQR_ERR_TIMEOUT);
    return false;
  };
  // Exchange after the partials of column jn are published (tag jn + 1):
  // totals, then the coefficients of jn's reflector and
  // w[c] = tau (x_jn,c + dot_c / d), c > jn.
  auto exchange = [&](int jn) -> bool {
    const uint32_t tag = (uint32_t)jn + 1u;
    const int par = jn & 1;
    bool bad = false;
    for (int e = q; e <= nc; e += C) {
      if (!(e == 0 || e >= jn + 2)) continue;
      T x = T(0);
      for (int t = tid; t < C && !bad; t += PT) {
        T v;
        if (!ll_get<T>(pword(par, t, e), tag, v, a.wait_ns, &s_fail)) bad = true;
        else x += v;
      }
      x = warp_sum(x);
      if (lane == 0) wsum[warp] = x;
      __syncthreads();
      if (tid == 0 && !bad) {
        T t = T(0);
        for (int k = 0; k < PT / 32; ++k) t += wsum[k];
        ll_put<T>(tword(par, e), t, tag);
      }
      __syncthreads();
    }
    if (__syncthreads_or(bad)) return fail();
    // this thread's first column's row entry and total, in the same round
    // trip as thread 0's coefficient inputs
    // (a panel with more columns than rows has no row jn >= mp: nobody
    // publishes it, and its reflector is the identity, tau = 0)
    const bool rowx = jn < a.mp;
    T rbc = T(0), totc = T(0), alpha = T(0), below = T(0);
    if (tid < nc && tid > jn)
      bad = (rowx && !ll_get<T>(rword(par, tid), tag, rbc, a.wait_ns, &s_fail)) ||
            !ll_get<T>(tword(par, 1 + tid), tag, totc, a.wait_ns, &s_fail);
    if (tid == 0)
      bad = (rowx && !ll_get<T>(rword(par, jn), tag, alpha, a.wait_ns, &s_fail)) ||
            !ll_get<T>(tword(par, 0), tag, below, a.wait_ns, &s_fail);
    if (__syncthreads_or(bad)) return fail();
    if (tid == 0) {
      T rd1;
      reflector_coef<T>(jn, a.mp, alpha, below, s_coef, q == 0 ? a.tau : nullptr, a.status, &rd1);
      s_rd = rd1;
    }
    __syncthreads();
    const T tau = s_coef[0], rd = s_rd;
    if (tid < nc) w[tid] = (tid > jn && tau != T(0)) ? tau * (rbc + totc * rd) : T(0);
    for (int c = tid + PT; c < nc && !bad; c += PT) {
      T rv = T(0), tv = T(0);
      if (c > jn && ((rowx && !ll_get<T>(rword(par, c), tag, rv, a.wait_ns, &s_fail)) ||
                     !ll_get<T>(tword(par, 1 + c), tag, tv, a.wait_ns, &s_fail)))
        bad = true;
      w[c] = (c > jn && tau != T(0)) ? tau * (rv + tv * rd) : T(0);
    }
    if (__syncthreads_or(bad)) return fail();
    return true;
  };
  // partials of column 0 (below the diagonal) and row 0
  {
    T ssum = T(0);
    for (int rr = tid; rr < nr; rr += PT)
      if (r0 + rr > 0) ssum += tile[rr] * tile[rr];
    ssum = block_sum(ssum, wsum);
    if (tid == 0) ll_put<T>(pword(0, q, 0), ssum, 1u);
    for (int c = 1 + warp; c < nc; c += PT / 32) {
      T acc = T(0);
      for (int rr = lane; rr < nr; rr += 32)
        if (r0 + rr > 0) acc += tile[rr] * tile[(size_t)c * RS + rr];
      acc = warp_sum(acc);
      if (lane == 0) ll_put<T>(pword(0, q, 1 + c), acc, 1u);
    }
    if (r0 == 0 && nr > 0)
      for (int c = tid; c < nc; c += PT) ll_put<T>(rword(0, c), tile[(size_t)c * RS], 1u);
    if (!exchange(0)) return;
  }
  for (int j = 0; j < nc; ++j) {
    const T tauj = s_coef[0], beta = s_coef[1], rd = s_rd;
    const bool has = s_coef[3] != T(0);
    const int lo = min(nr, max(0, j - r0));
    T* tj = tile + (size_t)j * RS;
    for (int rr = lo + tid; rr < nr; rr += PT) {
      const int i = r0 + rr;
      if (i > j) {
        if (has) tj[rr] = tauj == T(0) ? T(0) : tj[rr] * rd;
      } else if (has) {
        tj[rr] = beta;
      }
    }
    __syncthreads();
    if (j + 1 >= nc) break;
    T* t1 = tile + (size_t)(j + 1) * RS;
    const T w1 = w[j + 1];
    for (int rr = lo + tid; rr < nr; rr += PT) {
      const int i = r0 + rr;
      t1[rr] -= w1 * (i == j ? T(1) : tj[rr]);
    }
    __syncthreads();
    // Partials of column j+1: its squared norm below the diagonal and, while
    // reflector j is applied to columns j+2.., its dot products with them.
    // Items c = j+1 .. nc-1 (c = j+1: the norm) are spread over the block with
    // g threads per item (g a power of two, a group inside one warp, rows
    // interleaved), so the FP64 work of a column step keeps all four SM
    // sub-partitions busy however few columns remain.
    const uint32_t ntag = (uint32_t)j + 2u;  // the tag of exchange j + 1
    const int npar = (j + 1) & 1;
    const int nitem = nc - (j + 1);
    int g = 1;
    while (g < 32 && nitem * (2 * g) <= PT) g *= 2;
    const int lg = __ffs(g) - 1;
    const int span = PT >> lg, kk = tid & (g - 1);
    const int rs = min(nr, max(lo, j + 2 - r0));  // first local row below column j+1's diagonal
    for (int base = j + 1; base < nc; base += span) {
      const int c = base + (tid >> lg);
      T acc0 = T(0), acc1 = T(0);
      if (c == j + 1) {
        int rr = rs + kk;
        for (; rr + g < nr; rr += 2 * g) {
          acc0 += t1[rr] * t1[rr];
          acc1 += t1[rr + g] * t1[rr + g];
        }
        if (rr < nr) acc0 += t1[rr] * t1[rr];
      } else if (c < nc) {
        T* x = tile + (size_t)c * RS;
        const T wc = w[c];
        if (kk == 0)
          for (int rr = lo; rr < rs; ++rr)  // rows j (the reflector's unit entry) and j+1 (not in the dot product)
            x[rr] -= r0 + rr == j ? wc : wc * tj[rr];
        int rr = rs + kk;
        for (; rr + g < nr; rr += 2 * g) {
          const T x0 = x[rr] - wc * tj[rr], x1 = x[rr + g] - wc * tj[rr + g];
          x[rr] = x0;
          x[rr + g] = x1;
          acc0 += t1[rr] * x0;
          acc1 += t1[rr + g] * x1;
        }
        if (rr < nr) {
          const T x0 = x[rr] - wc * tj[rr];
          x[rr] = x0;
          acc0 += t1[rr] * x0;
        }
      }
      T acc = acc0 + acc1;
      for (int o = g >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (c < nc && kk == 0) ll_put<T>(pword(npar, q, c == j + 1 ? 0 : 1 + c), acc, ntag);
    }
    __syncthreads();  // row j+1 of every column is final before it is published
    if (j + 1 >= r0 && j + 1 < r1)
      for (int c = j + 1 + tid; c < nc; c += PT) ll_put<T>(rword(npar, c), tile[(size_t)c * RS + (j + 1 - r0)], ntag);
    if (!exchange(j + 1)) return;
  }
  __syncthreads();
  for (int e = tid; e < nr * nc; e += PT) {
    const int rr = e % nr, cc = e / nr;
    a.P[r0 + rr + (size_t)cc * a.ldp] = tile[(size_t)cc * RS + rr];
  }
}

}  // namespace

// Flagged words of the panel exchange: partials [2][C][nc + 1], totals
// [2][nc + 1], row [2][nc], each value in sizeof(T) / 4 words.
size_t panel_exchange_words(int nc, int C, size_t elem) {
  return (2 * (size_t)C * (nc + 1) + 2 * (size_t)(nc + 1) + 2 * (size_t)nc) * (elem / 4);
}

// Householder QR of the mp x nc panel as one cooperative launch; false (and
// nothing queued) when the rows of one CTA do not fit in shared memory or the
// grid cannot be co-scheduled. scratch: the panel scratch of panel.cu (at
// least panel_exchange_words(nc, C, sizeof(T)) words after 16-byte alignment).
template <typename T>
bool panel_qr_persist(const Ctx& c, int mp, int nc, T* P, int ldp, T* tau, T* scratch, int C, int R) {
  if (mp <= 0 || nc <= 0) return true;
  const size_t smem = sizeof(T) * ((size_t)nc + (size_t)nc * (R | 1));
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
  // flagged exchange words, zeroed before every launch: no word carries a tag
  // of this launch until written by it
  llw* words = reinterpret_cast<llw*>((reinterpret_cast<uintptr_t>(scratch) + 15) & ~uintptr_t(15));
  const size_t wv = sizeof(T) / 4;
  llw* pw = words;
  llw* tw = pw + 2 * (size_t)C * (nc + 1) * wv;
  llw* rw = tw + 2 * (size_t)(nc + 1) * wv;
  cudaMemsetAsync(words, 0, sizeof(llw) * panel_exchange_words(nc, C, sizeof(T)), c.stream);
  QArgs<T> a{mp, nc, R, P, ldp, tau, pw, tw, rw, c.status, c.wait_ns};
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
  return sizeof(double) * ((size_t)per * (l | 1) + l + 4 * (size_t)per);
}

// Flagged words of the pivot exchange: slots [2][C][4], candidate columns
// [2][C][2 l], the column leaving the pivot position [2][2 (l + 2)].
static size_t ypick_exchange_words(int l, int C) {
  return 2 * (size_t)C * 4 + 2 * (size_t)C * 2 * l + 2 * 2 * ((size_t)l + 2);
}

size_t ypick_persist_scratch_bytes(int l, int np, int sms) {
  int C, per;
  persist_smem(l, np, sms, C, per);
  return sizeof(unsigned long long) * ypick_exchange_words(l, C) + 256;
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
  // zeroed before every launch: no word carries a tag of this launch until written by it
  llw* w = static_cast<llw*>(scratch);
  cudaMemsetAsync(w, 0, sizeof(llw) * ypick_exchange_words(l, C), c.stream);
  llw* slots = w;
  llw* col = slots + 2 * (size_t)C * 4;
  llw* colbuf = col + 2 * (size_t)C * 2 * l;
  PArgs<T> a{l, np, per, bsteps, Y, ldy, picks, slots, col, colbuf, c.status, c.wait_ns};
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
