// batched.cu -- thousands of small FP32 factorizations in one persistent
// launch: randomized QRCP (Method 1 with over-sampling, a fresh Gaussian
// sketch per block as in Fig. blockQR, Sec. 4.1, 4.3, 5.1) or the truncated
// orthonormal-pivot factorization (Method 2 with the power scheme, Sec. 4.2,
// 6.3, 6.4, stopped once k columns are done), each matrix with its own shape
// and block size b.
//
// One CTA factors one matrix at a time: it takes the next entry of a work
// queue (the caller's order, normally longest first) with one atomic, runs
// every step of the method for that matrix with CTA barriers between the
// steps, and takes the next. The matrix stays in global memory (at most
// 1024 x 512, L1/L2-resident while the CTA works on it); the sketch, the panel
// and the block products go through a per-CTA scratch area and shared memory.
//
// Arithmetic follows the oracle's step order: Householder reflectors with
// beta = -sign(a1)||a|| (sign(0) = +1), tau = (beta - a1)/beta, no reflector for a
// column of length 1; T by the forward column recursion; pivot steps take the
// largest exactly recomputed squared norm, lowest position on ties, with
// sequential swaps mirrored on all m rows and on perm.
#include <algorithm>

#include "common.cuh"
#include "philox.cuh"

namespace rqr {

namespace {

constexpr int BT = 256, BW = BT / 32;
constexpr int kCtasPerSm = 2;  // resident CTAs per SM at 256 threads (register-bound)
constexpr int kMaxB = 32, kMaxL = 64;  // b and l = b + p; m <= 1024, n <= 512 are checked on the host

// Per-matrix descriptor: BD_LEN int64 per matrix (see include/rqr.h).
enum { BD_M, BD_N, BD_B, BD_K, BD_A, BD_T, BD_P, BD_W, BD_TV, BD_G, BD_LEN };

struct BArgs {
  int method, count, p, q;
  const long long* desc;
  const int* order;
  float* A;
  float* T;
  int32_t* perm;
  float* WV;
  float* TV;
  const float* G;  // explicit Gaussians or null (drawn from seed)
  uint64_t seed;
  float* scratch;
  size_t per_cta;  // scratch floats per CTA
  int* queue;
  int* status;
};

// ------------------------------------------------------------------ reductions
__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// CTA-wide sum (every thread gets the total); sh: BW floats of shared memory.
__device__ float cta_sum(float v, float* sh) {
  v = wsum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < BW; ++i) s += sh[i];
  return s;
}

// ------------------------------------------------------------------ Gaussian
// The first `count` values of stream (seed, s) into out (FP32): the same
// values as rqr_gauss_fill, rounded to FP32.
__device__ void cta_gauss(uint64_t seed, uint64_t s, int count, float* out) {
  for (int q = threadIdx.x; 4 * q < count; q += BT) {
    double z[4];
    gauss4((uint64_t)q, seed, s, z);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (4 * q + t < count) out[4 * q + t] = (float)z[t];
  }
}

// ------------------------------------------------------------------ Householder
// Reflector of x = P(j:r, j) (column j of an r x nc panel, ld ldp) per
// Sec. 3.1: writes v below the diagonal, beta on it, returns tau (0 when the
// column has length 1 or is zero). sh: BW floats.
__device__ float cta_reflector(int r, int j, float* P, int ldp, float* sh) {
  float* x = P + (size_t)j * ldp;
  if (r - j < 2) return 0.f;
  float ss = 0.f;
  for (int i = j + 1 + threadIdx.x; i < r; i += BT) ss += x[i] * x[i];
  ss = cta_sum(ss, sh);
  const float alpha = x[j];
  const float s = alpha * alpha + ss;
  if (s == 0.f) {
    __syncthreads();
    return 0.f;
  }
  const float beta = (alpha < 0.f ? 1.f : -1.f) * sqrtf(s);
  const float d = alpha - beta, tau = (beta - alpha) / beta;
  for (int i = j + 1 + threadIdx.x; i < r; i += BT) x[i] = x[i] / d;
  __syncthreads();
  if (threadIdx.x == 0) x[j] = beta;
  __syncthreads();
  return tau;
}

// Applies H_j = I - tau v v^T (v = [1; P(j+1:r, j)]) from the left to columns
// c0..c1-1 of P (rows j..r-1): warp per column.
__device__ void cta_apply_reflector(int r, int j, float tau, float* P, int ldp, int c0, int c1) {
  if (tau == 0.f) return;
  const float* v = P + (size_t)j * ldp;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int c = c0 + w; c < c1; c += BW) {
    float* x = P + (size_t)c * ldp;
    float s = lane == 0 ? x[j] : 0.f;
    for (int i = j + 1 + lane; i < r; i += 32) s += v[i] * x[i];
    s = wsum(s) * tau;
    if (lane == 0) x[j] -= s;
    for (int i = j + 1 + lane; i < r; i += 32) x[i] -= s * v[i];
  }
  __syncthreads();
}

// Unpivoted Householder QR of the r x nc panel P (Sec. 3.2); tau in shared
// memory (nc entries).
__device__ void cta_geqr2(int r, int nc, float* P, int ldp, float* tau, float* sh) {
  for (int j = 0; j < nc; ++j) {
    const float t = cta_reflector(r, j, P, ldp, sh);
    if (threadIdx.x == 0) tau[j] = t;
    cta_apply_reflector(r, j, t, P, ldp, j + 1, nc);
  }
  __syncthreads();
}

// T (nc x nc, ld ldt) of the reflectors below the diagonal of P (r x nc) by
// the forward recursion of the compact WY form (Sec. 5.1 remark):
// T(0:j, j) = -tau_j T(0:j, 0:j) (V^T v_j)(0:j), T(j, j) = tau_j.
// g: nc shared floats of scratch.
__device__ void cta_larft(int r, int nc, const float* P, int ldp, const float* tau, float* T, int ldt, float* g) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = 0; j < nc; ++j) {
    // g(i) = v_i^T v_j for i < j (v_i has its unit entry at row i)
    const float* vj = P + (size_t)j * ldp;
    for (int i = w; i < j; i += BW) {
      const float* vi = P + (size_t)i * ldp;
      float s = lane == 0 ? vi[j] : 0.f;  // row j: v_i(j) times v_j's unit entry
      for (int t = j + 1 + lane; t < r; t += 32) s += vi[t] * vj[t];
      s = wsum(s);
      if (lane == 0) g[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < j; i += BT) {
      float s = 0.f;
      for (int t = i; t < j; ++t) s += T[i + (size_t)t * ldt] * g[t];
      T[i + (size_t)j * ldt] = -tau[j] * s;
    }
    if (threadIdx.x == 0) T[j + (size_t)j * ldt] = tau[j];
    __syncthreads();
  }
}

// ------------------------------------------------------------------ block products
// W (nb x nc, ld ldw) = V^T X for the unit-lower V stored below the diagonal
// of P (r x nb, ld ldp; unit entry implicit) and X (r x nc, ld ldx): one warp
// per output, lanes along the rows.
__device__ void cta_vtx(int r, int nb, const float* P, int ldp, int nc, const float* X, int ldx, float* W, int ldw) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int e = w; e < nb * nc; e += BW) {
    const int a = e % nb, c = e / nb;
    const float* v = P + (size_t)a * ldp;
    const float* x = X + (size_t)c * ldx;
    float s = lane == 0 && a < r ? x[a] : 0.f;
    for (int i = a + 1 + lane; i < r; i += 32) s += v[i] * x[i];
    s = wsum(s);
    if (lane == 0) W[a + (size_t)c * ldw] = s;
  }
  __syncthreads();
}

// W2 (nb x nc) = op(T) W for the upper-triangular T (nb x nb, ld ldt):
// op = T^T (trans) or T.
__device__ void cta_tw(int nb, const float* T, int ldt, bool trans, int nc, const float* W, int ldw, float* W2,
                       int ldw2) {
  for (int e = threadIdx.x; e < nb * nc; e += BT) {
    const int a = e % nb, c = e / nb;
    float s = 0.f;
    if (trans)
      for (int t = 0; t <= a; ++t) s += T[t + (size_t)a * ldt] * W[t + (size_t)c * ldw];
    else
      for (int t = a; t < nb; ++t) s += T[a + (size_t)t * ldt] * W[t + (size_t)c * ldw];
    W2[a + (size_t)c * ldw2] = s;
  }
  __syncthreads();
}

// X (r x nc) -= V W2 with V as in cta_vtx: thread per element, rows fastest.
__device__ void cta_xmvw(int r, int nb, const float* P, int ldp, int nc, float* X, int ldx, const float* W2, int ldw2) {
  for (int e = threadIdx.x; e < r * nc; e += BT) {
    const int i = e % r, c = e / r;
    float s = 0.f;
    const int amax = min(i, nb - 1);
    for (int a = 0; a <= amax; ++a) s += (a == i ? 1.f : P[i + (size_t)a * ldp]) * W2[a + (size_t)c * ldw2];
    X[i + (size_t)c * ldx] -= s;
  }
  __syncthreads();
}

// Trailing update X <- (I - V T V^T)^T X (Fig. blockQR), scratch W, W2 (nb x nc).
__device__ void cta_block_update(int r, int nb, const float* P, int ldp, const float* T, int ldt, int nc, float* X,
                                 int ldx, float* W, float* W2) {
  if (nc <= 0 || nb <= 0) return;
  cta_vtx(r, nb, P, ldp, nc, X, ldx, W, nb);
  cta_tw(nb, T, ldt, true, nc, W, nb, W2, nb);
  cta_xmvw(r, nb, P, ldp, nc, X, ldx, W2, nb);
}

// ------------------------------------------------------------------ pivot steps
// Swaps columns c1 and c2 of P over rows -above..r-1 (rows above the block
// included) and the two perm entries (perm may be null).
__device__ void cta_swap(float* P, int ldp, int above, int r, int c1, int c2, int32_t* perm) {
  if (c1 == c2) return;
  float* x = P + (size_t)c1 * ldp;
  float* y = P + (size_t)c2 * ldp;
  for (int i = -above + (int)threadIdx.x; i < r; i += BT) {
    const float t = x[i];
    x[i] = y[i];
    y[i] = t;
  }
  if (perm && threadIdx.x == 0) {
    const int32_t t = perm[c1];
    perm[c1] = perm[c2];
    perm[c2] = t;
  }
  __syncthreads();
}

// nsteps steps of Fig. QR on the r x nc matrix P: at step j the column of
// largest squared norm over rows j.. (exactly recomputed, lowest position on
// ties) is swapped into position j (rows -above.. of both columns and perm
// entries), then its reflector is stored in place and applied to the later
// columns. tau receives the nsteps scalings (shared memory); nrm: nc floats
// of scratch; picks (optional, shared) the position swapped in at each step.
__device__ void cta_qrcp(int r, int nc, int nsteps, float* P, int ldp, int above, int32_t* perm, float* tau,
                         float* nrm, float* sh, int* shi, int* picks = nullptr) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = 0; j < nsteps; ++j) {
    for (int c = j + w; c < nc; c += BW) {
      const float* x = P + (size_t)c * ldp;
      float s = 0.f;
      for (int i = j + lane; i < r; i += 32) s += x[i] * x[i];
      s = wsum(s);
      if (lane == 0) nrm[c] = s;
    }
    __syncthreads();
    // argmax over c >= j: largest norm, lowest position on ties
    float bn = -1.f;
    int bp = nc;
    for (int c = j + (int)threadIdx.x; c < nc; c += BT)
      if (nrm[c] > bn) {
        bn = nrm[c];
        bp = c;
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float n2 = __shfl_xor_sync(0xffffffffu, bn, o);
      const int p2 = __shfl_xor_sync(0xffffffffu, bp, o);
      if (n2 > bn || (n2 == bn && p2 < bp)) {
        bn = n2;
        bp = p2;
      }
    }
    if (lane == 0) {
      sh[w] = bn;
      shi[w] = bp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = 1; i < BW; ++i)
        if (sh[i] > sh[0] || (sh[i] == sh[0] && shi[i] < shi[0])) {
          sh[0] = sh[i];
          shi[0] = shi[i];
        }
      // an all-NaN remainder leaves position j in place
      if (shi[0] >= nc) shi[0] = j;
    }
    __syncthreads();
    const int best = shi[0];
    __syncthreads();
    if (picks && threadIdx.x == 0) picks[j] = best;
    cta_swap(P, ldp, above, r, j, best, perm);
    const float t = cta_reflector(r, j, P, ldp, sh);
    if (threadIdx.x == 0) tau[j] = t;
    cta_apply_reflector(r, j, t, P, ldp, j + 1, nc);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ thin Q
// Q (r x nc, ld ldq) = H_0 ... H_{nc-1} [I; 0] from the reflectors below the
// diagonal of P (r x nc), tau (shared): the identity's columns, reflectors
// applied last to first.
__device__ void cta_form_q(int r, int nc, const float* P, int ldp, const float* tau, float* Q, int ldq) {
  for (int e = threadIdx.x; e < r * nc; e += BT) {
    const int i = e % r, c = e / r;
    Q[i + (size_t)c * ldq] = i == c ? 1.f : 0.f;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = nc - 1; j >= 0; --j) {
    const float t = tau[j];
    if (t == 0.f) continue;
    const float* v = P + (size_t)j * ldp;
    for (int c = j + w; c < nc; c += BW) {
      float* x = Q + (size_t)c * ldq;
      float s = lane == 0 ? x[j] : 0.f;
      for (int i = j + 1 + lane; i < r; i += 32) s += v[i] * x[i];
      s = wsum(s) * t;
      if (lane == 0) x[j] -= s;
      for (int i = j + 1 + lane; i < r; i += 32) x[i] -= s * v[i];
    }
    __syncthreads();
  }
}

// C (r x nc, ld ldc) = op(X) B with X (rows x cols, ld ldx), op = X^T (tx:
// C(c, a) = sum_i X(i, c) B(i, a)) or X (C(i, a) = sum_c X(i, c) B(c, a));
// B (kk x nc, ld ldb) with kk = rows (tx) or cols. Warp per output (tx, lanes
// along X's column) or thread per output (rows fastest).
__device__ void cta_xb(bool tx, int rows, int cols, const float* X, int ldx, int nc, const float* B, int ldb, float* C,
                       int ldc) {
  if (tx) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int e = w; e < cols * nc; e += BW) {
      const int c = e % cols, a = e / cols;
      const float* x = X + (size_t)c * ldx;
      const float* bcol = B + (size_t)a * ldb;
      float s = 0.f;
      for (int i = lane; i < rows; i += 32) s += x[i] * bcol[i];
      s = wsum(s);
      if (lane == 0) C[c + (size_t)a * ldc] = s;
    }
  } else {
    for (int e = threadIdx.x; e < rows * nc; e += BT) {
      const int i = e % rows, a = e / rows;
      float s = 0.f;
      for (int c = 0; c < cols; ++c) s += X[i + (size_t)c * ldx] * B[c + (size_t)a * ldb];
      C[i + (size_t)a * ldc] = s;
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------------ one matrix
struct Shared {
  float tau[kMaxL];
  float g[kMaxL];
  float sh[BW];
  int shi[BW];
  int picks[kMaxB];
};

// Scratch floats of one CTA for the largest matrix of a batch.
__host__ __device__ inline size_t batch_scratch_floats(int method, int m, int n, int b, int p) {
  const size_t l = (size_t)b + p;
  const size_t qr = l * m + l * n + n + 2 * (size_t)b * n;
  const size_t urv = (size_t)b * m + 2 * (size_t)n * b + 4 * (size_t)m * b + 2 * (size_t)b * n + n;
  return (method == RQR_BATCH_URV ? urv : qr) + 64;
}

// Method 1 with over-sampling p, a fresh sketch per block (Fig. blockQR,
// Sec. 4.1, 4.3, 5.1): Y = G_i A(k0:m, k0:n); the first b pivot steps of
// Fig. QR on Y, mirrored on all m rows of A and on perm; Householder QR of
// the panel, T, trailing update; the last block by Fig. QR.
__device__ void batch_rqrcp(const BArgs& a, int mi, const long long* d, float* scr, Shared& S) {
  const int m = (int)d[BD_M], n = (int)d[BD_N], b = (int)d[BD_B], l = b + a.p;
  float* A = a.A + d[BD_A];
  float* Tm = a.T + d[BD_T];
  int32_t* perm = a.perm + d[BD_P];
  const float* Gx = a.G ? a.G + d[BD_G] : nullptr;
  float* Gs = scr;
  float* Y = Gs + (size_t)l * m;
  float* nrm = Y + (size_t)l * n;
  float* W = nrm + n;
  float* W2 = W + (size_t)b * n;
  for (int j = threadIdx.x; j < n; j += BT) perm[j] = j;
  for (int e = threadIdx.x; e < b * n; e += BT) Tm[e] = 0.f;
  __syncthreads();
  size_t goff = 0;
  int k0 = 0, blk = 0;
  while (k0 < n) {
    const int np = n - k0, mp = m - k0;
    float* X = A + k0 + (size_t)k0 * m;
    if (np <= b) {
      const int steps = max(0, min(np, mp - 1));
      cta_qrcp(mp, np, steps, X, m, k0, perm + k0, S.tau, nrm, S.sh, S.shi);
      for (int j = steps + (int)threadIdx.x; j < np; j += BT) S.tau[j] = 0.f;
      __syncthreads();
      cta_larft(mp, np, X, m, S.tau, Tm + (size_t)k0 * b, b, S.g);
      break;
    }
    const float* Gi;
    if (Gx) {
      Gi = Gx + goff;
    } else {
      cta_gauss(a.seed, ((uint64_t)mi << 16) | (uint64_t)blk, l * mp, Gs);
      __syncthreads();
      Gi = Gs;
    }
    goff += (size_t)l * mp;
    // Y (l x np) = G_i (l x mp) X: warp per entry, lanes along the rows of X
    {
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      for (int e = w; e < l * np; e += BW) {
        const int r = e % l, c = e / l;
        const float* x = X + (size_t)c * m;
        float acc = 0.f;
        for (int i = lane; i < mp; i += 32) acc += Gi[r + (size_t)i * l] * x[i];
        acc = wsum(acc);
        if (lane == 0) Y[r + (size_t)c * l] = acc;
      }
      __syncthreads();
    }
    cta_qrcp(l, np, b, Y, l, 0, nullptr, S.tau, nrm, S.sh, S.shi, S.picks);
    for (int j = 0; j < b; ++j) cta_swap(X, m, k0, mp, j, S.picks[j], perm + k0);
    cta_geqr2(mp, b, X, m, S.tau, S.sh);
    cta_larft(mp, b, X, m, S.tau, Tm + (size_t)k0 * b, b, S.g);
    cta_block_update(mp, b, X, m, Tm + (size_t)k0 * b, b, np - b, X + (size_t)b * m, m, W, W2);
    k0 += b;
    ++blk;
  }
  __syncthreads();
}

// Method 2 with the power scheme, truncated at k (Sec. 4.2, 6.3, 6.4), no
// over-sampling: per block Z = (G_i X)^T, q times {Z <- orth(Z); W <- orth(X Z);
// Z <- X^T W}; Householder QR of Z's first b_i columns gives S_i = I - W TS W^T;
// A(0:m, k0:n) <- A(0:m, k0:n) S_i; panel QR, T, trailing update.
__device__ void batch_rurv(const BArgs& a, int mi, const long long* d, float* scr, Shared& S) {
  const int m = (int)d[BD_M], n = (int)d[BD_N], b = (int)d[BD_B];
  const int kr = d[BD_K] > 0 ? (int)min((long long)n, d[BD_K]) : n;
  float* A = a.A + d[BD_A];
  float* TU = a.T + d[BD_T];
  float* WV = a.WV + d[BD_W];
  float* TV = a.TV + d[BD_TV];
  const float* Gx = a.G ? a.G + d[BD_G] : nullptr;
  float* Gs = scr;                      // b x m
  float* Z = Gs + (size_t)b * m;        // n x b
  float* Zq = Z + (size_t)n * b;        // n x b
  float* Wm = Zq + (size_t)n * b;       // m x b
  float* Wq = Wm + (size_t)m * b;       // m x b
  float* P1 = Wq + (size_t)m * b;       // m x b
  float* P2 = P1 + (size_t)m * b;       // m x b
  float* W = P2 + (size_t)m * b;        // b x n
  float* W2 = W + (size_t)b * n;        // b x n
  for (int e = threadIdx.x; e < b * n; e += BT) {
    TU[e] = 0.f;
    TV[e] = 0.f;
  }
  for (int e = threadIdx.x; e < n * n; e += BT) WV[e] = 0.f;
  __syncthreads();
  size_t goff = 0;
  int k0 = 0, blk = 0;
  while (k0 < n) {
    const int np = n - k0, mp = m - k0, bi = min(b, np);
    float* X = A + k0 + (size_t)k0 * m;
    const float* Gi;
    if (Gx) {
      Gi = Gx + goff;
    } else {
      cta_gauss(a.seed, ((uint64_t)mi << 16) | (uint64_t)blk, b * mp, Gs);
      __syncthreads();
      Gi = Gs;
    }
    goff += (size_t)b * mp;
    // Z (np x b): Z(c, r) = sum_i X(i, c) G_i(r, i)
    {
      const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
      for (int e = w; e < np * b; e += BW) {
        const int c = e % np, r = e / np;
        const float* x = X + (size_t)c * m;
        float acc = 0.f;
        for (int i = lane; i < mp; i += 32) acc += x[i] * Gi[r + (size_t)i * b];
        acc = wsum(acc);
        if (lane == 0) Z[c + (size_t)r * np] = acc;
      }
      __syncthreads();
    }
    int zc = b;
    for (int t = 0; t < a.q; ++t) {
      const int kz = min(np, zc);
      cta_geqr2(np, zc, Z, np, S.tau, S.sh);
      cta_form_q(np, kz, Z, np, S.tau, Zq, np);
      cta_xb(false, mp, np, X, m, kz, Zq, np, Wm, mp);         // W = X Zq
      const int kw = min(mp, kz);
      cta_geqr2(mp, kz, Wm, mp, S.tau, S.sh);
      cta_form_q(mp, kw, Wm, mp, S.tau, Wq, mp);
      cta_xb(true, mp, np, X, m, kw, Wq, mp, Z, np);           // Z = X^T Wq
      zc = kw;
    }
    // orthonormal pivot: Householder QR of Z(:, 0:bi) (a full basis for the
    // last block, whatever columns span it)
    cta_geqr2(np, bi, Z, np, S.tau, S.sh);
    float* TS = TV + (size_t)k0 * b;
    cta_larft(np, bi, Z, np, S.tau, TS, b, S.g);
    for (int e = threadIdx.x; e < np * bi; e += BT) {
      const int i = e % np, c = e / np;
      if (i > c) WV[k0 + i + (size_t)(k0 + c) * n] = Z[i + (size_t)c * np];
    }
    // A(0:m, k0:n) <- A(0:m, k0:n) (I - W TS W^T), all m rows
    float* Ak = A + (size_t)k0 * m;
    for (int e = threadIdx.x; e < m * bi; e += BT) {
      const int i = e % m, t = e / m;
      float acc = Ak[i + (size_t)t * m];  // unit entry of column t of W
      for (int c = t + 1; c < np; ++c) acc += Ak[i + (size_t)c * m] * Z[c + (size_t)t * np];
      P1[i + (size_t)t * m] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * bi; e += BT) {
      const int i = e % m, t = e / m;
      float acc = 0.f;
      for (int u = 0; u <= t; ++u) acc += P1[i + (size_t)u * m] * TS[u + (size_t)t * b];
      P2[i + (size_t)t * m] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < m * np; e += BT) {
      const int i = e % m, c = e / m;
      float acc = 0.f;
      const int tmax = min(c, bi - 1);
      for (int t = 0; t <= tmax; ++t) acc += P2[i + (size_t)t * m] * (t == c ? 1.f : Z[c + (size_t)t * np]);
      Ak[i + (size_t)c * m] -= acc;
    }
    __syncthreads();
    // panel QR, T, trailing update (Fig. blockRRQR / blockQR)
    cta_geqr2(mp, bi, X, m, S.tau, S.sh);
    cta_larft(mp, bi, X, m, S.tau, TU + (size_t)k0 * b, b, S.g);
    cta_block_update(mp, bi, X, m, TU + (size_t)k0 * b, b, np - bi, X + (size_t)bi * m, m, W, W2);
    k0 += bi;
    ++blk;
    if (k0 >= kr) break;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(BT, 2) k_batched(BArgs a, int max_m, int max_n, int max_b) {
  __shared__ Shared S;
  __shared__ int s_next;
  float* scr = a.scratch + (size_t)blockIdx.x * a.per_cta;
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
    __syncthreads();
    const int slot = s_next;
    __syncthreads();
    if (slot >= a.count) break;
    const int mi = a.order ? a.order[slot] : slot;
    if (mi < 0 || mi >= a.count) {
      if (threadIdx.x == 0) atomicCAS(a.status, 0, RQR_ERR_SIZE);
      continue;
    }
    const long long* d = a.desc + (size_t)mi * BD_LEN;
    const long long m = d[BD_M], n = d[BD_N], b = d[BD_B];
    // shapes outside the launch's limits (the scratch is sized by them) are skipped
    if (m < 1 || n < 1 || n > m || m > max_m || n > max_n || b < 1 || b > max_b) {
      if (threadIdx.x == 0) atomicCAS(a.status, 0, RQR_ERR_SIZE);
      continue;
    }
    if (a.method == RQR_BATCH_URV) batch_rurv(a, mi, d, scr, S);
    else batch_rqrcp(a, mi, d, scr, S);
  }
}

}  // namespace

size_t batched_workspace_bytes(int method, int count, int max_m, int max_n, int max_b, int p, int sms) {
  const int grid = std::max(1, std::min(count, kCtasPerSm * sms));
  return 256 + sizeof(float) * batch_scratch_floats(method, max_m, max_n, max_b, p) * (size_t)grid;
}

int batched_factor(const Ctx& c, int method, int count, const long long* desc, const int* order, float* A, float* T,
                   int32_t* perm, float* WV, float* TV, const float* G, int p, int q, uint64_t seed, int max_m,
                   int max_n, int max_b, void* work, size_t lwork) {
  if (count <= 0) return RQR_OK;
  if (lwork < batched_workspace_bytes(method, count, max_m, max_n, max_b, p, c.sms)) return RQR_ERR_WORKSPACE;
  const int grid = std::max(1, std::min(count, kCtasPerSm * c.sms));
  char* w = static_cast<char*>(work);
  int* queue = reinterpret_cast<int*>(w);
  BArgs a{};
  a.method = method;
  a.count = count;
  a.p = p;
  a.q = q;
  a.desc = desc;
  a.order = order;
  a.A = A;
  a.T = T;
  a.perm = perm;
  a.WV = WV;
  a.TV = TV;
  a.G = G;
  a.seed = seed;
  a.scratch = reinterpret_cast<float*>(w + 256);
  a.per_cta = batch_scratch_floats(method, max_m, max_n, max_b, p);
  a.queue = queue;
  a.status = c.status;
  cudaMemsetAsync(queue, 0, sizeof(int), c.stream);
  k_batched<<<grid, BT, 0, c.stream>>>(a, max_m, max_n, max_b);
  note_launch(c);
  return RQR_OK;
}

}  // namespace rqr
