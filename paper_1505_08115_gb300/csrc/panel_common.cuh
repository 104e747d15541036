// panel_common.cuh -- reflector coefficients and the last-CTA reduction shared
// by the multi-launch panel (panel.cu) and the persistent panel (persist.cu).
#pragma once
#include "common.cuh"

namespace rqr {
namespace pnl {

constexpr int PT = 256;        // threads per panel CTA
constexpr int NCOEF = 4;       // tau, beta, d, has-reflector

struct PanelArgs {
  int mp, nc, R, ldp;
};

// tau = (beta - alpha) / beta and rd = 1 / d of a reflector, d = alpha - beta
// (nonzero: beta has the opposite sign of alpha), with one division:
// r = 1 / (d beta), rd = beta r, tau = -d / beta = -d^2 r (FP64 division is a
// long dependent chain on GB300's FP64 pipe); two divisions when d beta
// leaves the normal range.
template <typename T>
__device__ __forceinline__ void tau_and_rd(T alpha, T beta, T d, T& tau, T& rd) {
  const T db = d * beta;
  const T tiny = sizeof(T) == 8 ? T(2.2250738585072014e-308) : T(1.1754943508222875e-38);
  if (fabs(db) >= tiny && isfinite(db)) {
    const T r = T(1) / db;
    rd = beta * r;
    tau = -(d * d) * r;
  } else {
    rd = T(1) / d;
    tau = (beta - alpha) / beta;
  }
}

// Coefficients of the reflector of column j from its squared norm below the
// diagonal (s_below) and its diagonal entry alpha (Sec. 3.1 with sign(0)=+1);
// rd_out (if given) receives 1 / d.
template <typename T>
__device__ __forceinline__ void reflector_coef(int j, int mp, T alpha, T s_below, T* coef, T* tau_out, int* status,
                                               T* rd_out = nullptr) {
  T tau = T(0), beta = alpha, d = T(1), has = T(0), rd = T(1);
  if (mp - j >= 2) {
    has = T(1);
    const T s = alpha * alpha + s_below;
    if (!isfinite(s)) atomicCAS(status, 0, RQR_ERR_NONFINITE);
    if (s == T(0)) {
      beta = T(0);
    } else {
      const T nrm = sqrt(s);
      beta = -sgn0(alpha) * nrm;
      d = alpha - beta;
      tau_and_rd(alpha, beta, d, tau, rd);
    }
  }
  coef[0] = tau;
  coef[1] = beta;
  coef[2] = d;
  coef[3] = has;
  if (tau_out) tau_out[j] = tau;
  if (rd_out) *rd_out = rd;
}

// Last-CTA step: totals of the partials for column jn (entry 0 = squared norm
// below the diagonal, entry 1 + c = dot with column c) and its coefficients.
// Lane l of every warp owns columns jn + l + 32k; warp w adds the partials of
// CTAs w, w + 8, ... (independent loads, no long serial chain); the eight warp
// sums are then added in warp order, so the result does not depend on timing.
template <typename T>
__device__ __forceinline__ void finish_coef(int jn, const PanelArgs& a, const T* part, const T* rowbuf, T* coef, T* tau_out,
                            int* status, T* red) {
  constexpr int NW = PT / 32;
  __shared__ T wred[NW][32 * 4];
  const int C = gridDim.x, tid = threadIdx.x, nc = a.nc, lane = tid & 31, warp = tid >> 5;
  for (int c0 = jn; c0 < nc; c0 += 32 * 4) {
    T acc[4] = {T(0), T(0), T(0), T(0)};
    for (int q = warp; q < C; q += NW) {
      const T* pq = part + (size_t)q * (nc + 1);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int c = c0 + lane + 32 * k;
        if (c < nc) acc[k] += __ldcg(pq + (c == jn ? 0 : 1 + c));
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) wred[warp][lane + 32 * k] = acc[k];
    __syncthreads();
    for (int t = tid; t < 32 * 4; t += PT) {
      const int c = c0 + t;
      if (c < nc) {
        T s = T(0);
        for (int w = 0; w < NW; ++w) s += wred[w][t];
        red[c] = s;
      }
    }
    __syncthreads();
  }
  if (tid == 0) reflector_coef<T>(jn, a.mp, __ldcg(rowbuf + jn), red[jn], coef, tau_out, status);
  __syncthreads();
  const T tau = coef[0], d = coef[2];
  for (int c = jn + 1 + tid; c < nc; c += PT)
    coef[NCOEF + c] = tau == T(0) ? T(0) : tau * (__ldcg(rowbuf + c) + red[c] / d);
}

// Ticket: returns true in exactly one CTA, the last one to get here, after all
// other CTAs' global writes are visible to it.
__device__ __forceinline__ bool last_cta(int* counter) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int t = atomicAdd(counter, 1);
    last = (t == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0)
    for (int i = 0; i < PT / 32; ++i) s += sh[i];
  __syncthreads();
  return s;  // valid in thread 0
}


}  // namespace pnl
}  // namespace rqr
