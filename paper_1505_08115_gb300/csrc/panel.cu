// panel.cu -- Householder QR of a tall panel (Sec. 3.2), classical pivoted QR
// of the last block (Fig. QR, Sec. 3.3), and the compact-WY T factor
// (Sec. 5.1, WY remark).
//
// A panel of mp x nc (mp up to ~16k, nc = b <= 512) is spread over C CTAs,
// each owning a contiguous slice of rows. One launch handles one column j:
//   * every CTA reads the reflector coefficients of column j (tau, beta,
//     d = alpha - beta and w_c = tau * v^T x_c for c > j) prepared by the
//     previous launch, writes v = x_j/d over its rows, applies
//     x_c <- x_c - w_c v to its rows, and in the same pass accumulates its
//     partial sums for column j+1 (||x_{j+1}||^2 below the diagonal and
//     x_{j+1}^T x_c), which need only the freshly updated values;
//   * the owner of row j+1 publishes that row;
//   * the last CTA to finish (atomic ticket after a fence, no waiting) adds
//     the partials in CTA order and prepares the coefficients of column j+1.
// The identity v^T x_c = x_c(j) + (sum_{i>j} x_j(i) x_c(i)) / d lets one
// reduction per column serve both the norm and every dot product.
#include <algorithm>

#include "common.cuh"
#include "panel_common.cuh"

namespace rqr {

namespace {

using namespace pnl;

// ------------------------------------------------------------ unpivoted panel
template <typename T>
__global__ void __launch_bounds__(PT) k_panel_init(PanelArgs a, const T* __restrict__ P, T* part, T* rowbuf,
                                                   T* coef, T* tau, int* counter, int* status) {
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);
  __shared__ T wsum[PT / 32];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = q * a.R, r1 = min(a.mp, r0 + a.R), nr = max(0, r1 - r0);
  T* myp = part + (size_t)q * (a.nc + 1);
  // norm of column 0 below the diagonal
  T s = T(0);
  for (int rr = tid; rr < nr; rr += PT) {
    const int i = r0 + rr;
    if (i > 0) {
      const T x = P[i];
      s += x * x;
    }
  }
  s = block_sum(s, wsum);
  if (tid == 0) myp[0] = s;
  for (int c = 1 + warp; c < a.nc; c += PT / 32) {
    T acc = T(0);
    for (int rr = lane; rr < nr; rr += 32) {
      const int i = r0 + rr;
      if (i > 0) acc += P[i] * P[i + (size_t)c * a.ldp];
    }
    acc = warp_sum(acc);
    if (lane == 0) myp[1 + c] = acc;
  }
  if (r0 == 0 && nr > 0)
    for (int c = tid; c < a.nc; c += PT) rowbuf[c] = P[(size_t)c * a.ldp];
  if (last_cta(counter)) {
    finish_coef<T>(0, a, part, rowbuf, coef, tau, status, red);
    if (tid == 0) *counter = 0;
  }
}

// One column step. The CTA's rows >= j of the active columns j..nc-1 are
// staged in shared memory with one parallel load (tile[cc*R + rr] holds
// P(r0 + rr, j + cc)), updated there, and written back once.
template <typename T>
__global__ void __launch_bounds__(PT) k_panel_step(int j, PanelArgs a, T* __restrict__ P, const T* coef_in,
                                                   T* coef_out, T* part, T* rowbuf_out, T* tau, int* counter,
                                                   int* status) {
  extern __shared__ unsigned char smem_raw[];
  const int nc = a.nc, ldp = a.ldp, R = a.R, wj = nc - j;
  T* w = reinterpret_cast<T*>(smem_raw);  // [nc]
  T* tile = w + nc;                       // [wj][R]
  __shared__ T wsum[PT / 32];
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = q * R, r1 = min(a.mp, r0 + R), nr = max(0, r1 - r0);
  const int lo = min(nr, max(0, j - r0));  // first local row with global index >= j
  const int h = nr - lo;
  for (int c = tid; c < nc; c += PT) w[c] = c > j ? coef_in[NCOEF + c] : T(0);
  const T tauj = coef_in[0], beta = coef_in[1], d = coef_in[2];
  const bool has = coef_in[3] != T(0);
  for (int e = tid; e < h * wj; e += PT) {
    const int rr = lo + e % h, cc = e / h;
    tile[cc * R + rr] = P[r0 + rr + (size_t)(j + cc) * ldp];
  }
  __syncthreads();
  // column j becomes v below the diagonal and beta on it
  for (int rr = lo + tid; rr < nr; rr += PT) {
    const int i = r0 + rr;
    if (i > j) {
      if (has) tile[rr] = tauj == T(0) ? T(0) : tile[rr] / d;
    } else if (has) {
      tile[rr] = beta;
    }
  }
  __syncthreads();
  const bool next = j + 1 < nc;
  if (next) {
    // column j+1 first: its updated values feed the dot products below
    const T w1 = w[j + 1];
    for (int rr = lo + tid; rr < nr; rr += PT) {
      const int i = r0 + rr;
      const T vi = i == j ? T(1) : tile[rr];
      tile[R + rr] -= w1 * vi;
    }
    __syncthreads();
    T* myp = part + (size_t)q * (nc + 1);
    T s = T(0);
    for (int rr = lo + tid; rr < nr; rr += PT)
      if (r0 + rr > j + 1) s += tile[R + rr] * tile[R + rr];
    s = block_sum(s, wsum);
    if (tid == 0) myp[0] = s;
    for (int c = j + 2 + warp; c < nc; c += PT / 32) {
      T* x = tile + (size_t)(c - j) * R;
      const T wc = w[c];
      T acc = T(0);
      for (int rr = lo + lane; rr < nr; rr += 32) {
        const int i = r0 + rr;
        const T vi = i == j ? T(1) : tile[rr];
        const T xv = x[rr] - wc * vi;
        x[rr] = xv;
        if (i > j + 1) acc += tile[R + rr] * xv;
      }
      acc = warp_sum(acc);
      if (lane == 0) myp[1 + c] = acc;
    }
    __syncthreads();
    if (j + 1 >= r0 && j + 1 < r1)
      for (int c = j + 1 + tid; c < nc; c += PT) rowbuf_out[c] = tile[(size_t)(c - j) * R + (j + 1 - r0)];
  }
  for (int e = tid; e < h * wj; e += PT) {
    const int rr = lo + e % h, cc = e / h;
    P[r0 + rr + (size_t)(j + cc) * ldp] = tile[cc * R + rr];
  }
  if (next && last_cta(counter)) {
    finish_coef<T>(j + 1, a, part, rowbuf_out, coef_out, tau, status, w);
    if (tid == 0) *counter = 0;
  }
}

// ------------------------------------------------------------ pivoted block
// Norms of all columns c >= jn over rows >= jn (partials), then the last CTA
// picks the largest (lowest position on ties) into piv[jn].
template <typename T>
__device__ void norms_and_pick(int jn, int nsteps, const PanelArgs& a, const T* P, T* part, int* piv, int* counter,
                               T* red) {
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = q * a.R, r1 = min(a.mp, r0 + a.R), nr = max(0, r1 - r0);
  T* myp = part + (size_t)q * (a.nc + 1);
  for (int c = jn + warp; c < a.nc; c += PT / 32) {
    const T* Pc = P + (size_t)c * a.ldp;
    T acc = T(0);
    for (int rr = lane; rr < nr; rr += 32) {
      const int i = r0 + rr;
      if (i >= jn) acc += Pc[i] * Pc[i];
    }
    acc = warp_sum(acc);
    if (lane == 0) myp[1 + c] = acc;
  }
  if (last_cta(counter)) {
    for (int c = jn + tid; c < a.nc; c += PT) {
      T s = T(0);
      for (int qq = 0; qq < (int)gridDim.x; ++qq) s += __ldcg(part + (size_t)qq * (a.nc + 1) + 1 + c);
      red[c] = s;
    }
    __syncthreads();
    if (tid == 0) {
      int best = jn;
      T bn = T(-1);
      for (int c = jn; c < a.nc; ++c)
        if (red[c] > bn) { bn = red[c]; best = c; }
      piv[jn] = best;
      *counter = 0;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(PT) k_qrcp_init(PanelArgs a, const T* P, T* part, int* piv, int* counter) {
  extern __shared__ unsigned char smem_raw[];
  norms_and_pick<T>(0, 0, a, P, part, piv, counter, reinterpret_cast<T*>(smem_raw));
}

// Swap column j with piv[j] over all m rows of A (the block starts at row and
// column k0 of A), swap perm, then partials of column j and coefficients.
template <typename T>
__global__ void __launch_bounds__(PT) k_qrcp_pick(int j, PanelArgs a, int k0, int m, T* A, int lda, int32_t* perm,
                                                  const int* piv, T* part, T* rowbuf, T* coef, T* tau, int* counter,
                                                  int* status) {
  extern __shared__ unsigned char smem_raw[];
  T* red = reinterpret_cast<T*>(smem_raw);
  __shared__ T wsum[PT / 32];
  const int q = blockIdx.x, C = gridDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nc = a.nc;
  const int cs = piv[j];
  T* P = A + k0 + (size_t)k0 * lda;  // block origin; ldp == lda
  const int r0 = q * a.R, r1 = min(a.mp, r0 + a.R), nr = max(0, r1 - r0);
  if (cs != j) {
    T* x = A + (size_t)(k0 + j) * lda;
    T* y = A + (size_t)(k0 + cs) * lda;
    for (int rr = tid; rr < nr; rr += PT) {
      const int i = k0 + r0 + rr;
      const T t = x[i];
      x[i] = y[i];
      y[i] = t;
    }
    const int Rt = (k0 + C - 1) / C;  // rows above the block
    const int t0 = q * Rt, t1 = min(k0, t0 + Rt);
    for (int i = t0 + tid; i < t1; i += PT) {
      const T t = x[i];
      x[i] = y[i];
      y[i] = t;
    }
    if (q == 0 && tid == 0) {
      const int32_t t = perm[k0 + j];
      perm[k0 + j] = perm[k0 + cs];
      perm[k0 + cs] = t;
    }
  }
  __syncthreads();
  const T* Pj = P + (size_t)j * lda;
  T* myp = part + (size_t)q * (nc + 1);
  T s = T(0);
  for (int rr = tid; rr < nr; rr += PT) {
    const int i = r0 + rr;
    if (i > j) s += Pj[i] * Pj[i];
  }
  s = block_sum(s, wsum);
  if (tid == 0) myp[0] = s;
  for (int c = j + 1 + warp; c < nc; c += PT / 32) {
    const T* Pc = P + (size_t)c * lda;
    T acc = T(0);
    for (int rr = lane; rr < nr; rr += 32) {
      const int i = r0 + rr;
      if (i > j) acc += Pj[i] * Pc[i];
    }
    acc = warp_sum(acc);
    if (lane == 0) myp[1 + c] = acc;
  }
  if (j >= r0 && j < r1)
    for (int c = j + tid; c < nc; c += PT) rowbuf[c] = P[j + (size_t)c * lda];
  if (last_cta(counter)) {
    finish_coef<T>(j, a, part, rowbuf, coef, tau, status, red);
    if (tid == 0) *counter = 0;
  }
}

// Apply the coefficients of column j to every later column; then partial norms
// for the next pick.
template <typename T>
__global__ void __launch_bounds__(PT) k_qrcp_apply(int j, int nsteps, PanelArgs a, T* P, const T* coef, T* part,
                                                   int* piv, int* counter) {
  extern __shared__ unsigned char smem_raw[];
  T* w = reinterpret_cast<T*>(smem_raw);  // [nc]
  T* vs = w + a.nc;                       // [R]
  const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nc = a.nc, ldp = a.ldp;
  const int r0 = q * a.R, r1 = min(a.mp, r0 + a.R), nr = max(0, r1 - r0);
  for (int c = tid; c < nc; c += PT) w[c] = c > j ? coef[NCOEF + c] : T(0);
  const T tauj = coef[0], beta = coef[1], d = coef[2];
  const bool has = coef[3] != T(0);
  __syncthreads();
  T* Pj = P + (size_t)j * ldp;
  for (int rr = tid; rr < nr; rr += PT) {
    const int i = r0 + rr;
    if (i > j) {
      T v = Pj[i];
      if (has) v = tauj == T(0) ? T(0) : v / d;
      Pj[i] = v;
      vs[rr] = v;
    } else if (i == j) {
      if (has) Pj[j] = beta;
      for (int c = j + 1; c < nc; ++c) P[j + (size_t)c * ldp] -= w[c];
    }
  }
  __syncthreads();
  for (int c = j + 1 + warp; c < nc; c += PT / 32) {
    T* Pc = P + (size_t)c * ldp;
    const T wc = w[c];
    for (int rr = lane; rr < nr; rr += 32) {
      const int i = r0 + rr;
      if (i > j) Pc[i] -= wc * vs[rr];
    }
  }
  if (j + 1 < nsteps) {
    __syncthreads();
    norms_and_pick<T>(j + 1, nsteps, a, P, part, piv, counter, w);
  }
}

// ------------------------------------------------------------ T factor
// T(0:j, j) = -tau_j T(0:j, 0:j) (V^T V)(0:j, j), T(j, j) = tau_j (Sec. 5.1),
// column by column in one CTA, T built in global memory. Used only when the
// Gram triangle of k_larft_inv below does not fit in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_larft_tri(int kb, const T* __restrict__ gram, int ldg, const T* tau, T* Tm,
                                                   int ldt) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kb * kb; e += blockDim.x) {
    const int i = e % kb, c = e / kb;
    Tm[i + (size_t)c * ldt] = T(0);
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const T tj = tau[j];
    for (int i = tid; i < j; i += blockDim.x) {
      T s = T(0);
      for (int l = i; l < j; ++l) s += Tm[i + (size_t)l * ldt] * gram[l + (size_t)j * ldg];
      Tm[i + (size_t)j * ldt] = -tj * s;
    }
    if (tid == 0) Tm[j + (size_t)j * ldt] = tj;
    __syncthreads();
  }
}

// T as the inverse of S = diag(1/tau) + striu(V^T V): S has the same
// column recursion as T (Sec. 5.1), so S T = I. Column j of T is then one
// back substitution, x_j = tau_j and x_i = -tau_i sum_{k=i+1..j} G_ik x_k,
// independent of the other columns: one CTA per column, all columns at once.
// The CTA's threads copy G's strict upper triangle up to column j into
// shared memory, packed (column k at k (k - 1) / 2), eight independent loads
// per thread at a time; one warp then runs the substitution, lane l keeping
// the running sums of rows l, l + 32, .... A zero tau_i (no reflector) gives
// a zero row and column, as in the recursion.
constexpr int kLarftRows = 8;  // rows per lane: kb <= 256
constexpr int kLarftT = 256;   // threads per CTA for the copy
constexpr int kLarftU = 8;     // loads in flight per thread

template <typename T>
__global__ void __launch_bounds__(kLarftT) k_larft_inv(int kb, const T* __restrict__ gram, int ldg,
                                                       const T* __restrict__ tau, T* Tm, int ldt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ts = reinterpret_cast<T*>(smem_raw);  // [kb] tau
  T* Gp = ts + kb;                         // packed strict upper triangle, columns 1..j
  const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31;
  for (int i = tid; i < kb; i += kLarftT) ts[i] = tau[i];
  const int tot = j * (j + 1) / 2;  // entries of columns 1..j
  for (int e0 = tid; e0 < tot; e0 += kLarftT * kLarftU) {
    T v[kLarftU];
#pragma unroll
    for (int u = 0; u < kLarftU; ++u) {
      const int e = e0 + u * kLarftT;
      if (e < tot) {
        // column k = the largest k with k (k - 1) / 2 <= e, row i = the rest
        int k = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
        if (k * (k - 1) / 2 > e) --k;
        if ((k + 1) * k / 2 <= e) ++k;
        v[u] = gram[(e - k * (k - 1) / 2) + (size_t)k * ldg];
      }
    }
#pragma unroll
    for (int u = 0; u < kLarftU; ++u) {
      const int e = e0 + u * kLarftT;
      if (e < tot) Gp[e] = v[u];
    }
  }
  __syncthreads();
  if (tid >= 32) return;
  T acc[kLarftRows];
#pragma unroll
  for (int r = 0; r < kLarftRows; ++r) acc[r] = T(0);
  T* tcol = Tm + (size_t)j * ldt;
  T xk = ts[j];  // x_j
  if (lane == 0) tcol[j] = xk;
  for (int i = j + 1 + lane; i < kb; i += 32) tcol[i] = T(0);
  for (int k = j; k >= 1; --k) {
    // add column k of G times x_k to the rows above k, then finish row k - 1
    const T* gk = Gp + (size_t)k * (k - 1) / 2;
#pragma unroll
    for (int r = 0; r < kLarftRows; ++r) {
      const int i = lane + 32 * r;
      if (32 * r < k && i < k) acc[r] += gk[i] * xk;
    }
    const int o = k - 1, orow = o >> 5;
    T a = acc[0];
#pragma unroll
    for (int r = 1; r < kLarftRows; ++r)
      if (r == orow) a = acc[r];
    a = __shfl_sync(0xffffffffu, a, o & 31);
    xk = -ts[o] * a;
    if (lane == (o & 31)) tcol[o] = xk;
  }
}

// Gram matrix of V = E + L from the Gram matrix of its strictly lower part:
// V^T V = L^T L + I + L1 + L1^T, L1 = the top kb x kb block of L.
template <typename T>
__global__ void k_gram_from_lower(int kb, const T* __restrict__ L, int ldl, T* gram, int ldg) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kb * kb; e += gridDim.x * blockDim.x) {
    const int i = e % kb, j = e / kb;
    T add = i == j ? T(1) : (i > j ? L[i + (size_t)j * ldl] : L[j + (size_t)i * ldl]);
    gram[i + (size_t)j * ldg] += add;
  }
}

// ------------------------------------------------------------ helpers
template <typename T>
__global__ void k_copy_mat(int r, int cols, const T* __restrict__ s, int lds, T* __restrict__ d, int ldd) {
  const int64_t n = (int64_t)r * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % r, j = e / r;
    d[i + j * ldd] = s[i + j * lds];
  }
}

// dst (cols x r) = src (r x cols)^T, 32 x 32 tiles through shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_transpose(int r, int cols, const T* __restrict__ s, int lds,
                                                   T* __restrict__ d, int ldd) {
  __shared__ T tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32, tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int y = ty; y < 32; y += 8) {
    const int i = i0 + tx, j = j0 + y;
    if (i < r && j < cols) tile[y][tx] = s[i + (size_t)j * lds];
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {
    const int j = j0 + tx, i = i0 + y;
    if (i < r && j < cols) d[j + (size_t)i * ldd] = tile[tx][y];
  }
}

template <typename T>
__global__ void k_set_mat(int r, int cols, T val, T* d, int ldd) {
  const int64_t n = (int64_t)r * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % r, j = e / r;
    d[i + j * ldd] = val;
  }
}

template <typename T>
__global__ void k_make_vx(int mp, int kb, const T* __restrict__ F, int ldf, T* __restrict__ V, int ldv) {
  const int64_t n = (int64_t)mp * kb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % mp), j = (int)(e / mp);
    V[i + (int64_t)j * ldv] = i > j ? F[i + (int64_t)j * ldf] : (i == j ? T(1) : T(0));
  }
}

template <typename T>
__global__ void k_make_vlow(int mp, int kb, const T* __restrict__ F, int ldf, T* __restrict__ V, int ldv) {
  const int64_t n = (int64_t)mp * kb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % mp), j = (int)(e / mp);
    V[i + (int64_t)j * ldv] = i > j ? F[i + (int64_t)j * ldf] : T(0);
  }
}

template <typename T>
__global__ void k_add_mat(int r, int cols, T alpha, const T* __restrict__ s, int lds, T* d, int ldd) {
  const int64_t n = (int64_t)r * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % r, j = e / r;
    d[i + j * ldd] += alpha * s[i + j * lds];
  }
}

int grid1d(int64_t n, int sms) {
  int64_t g = (n + 255) / 256;
  g = std::min<int64_t>(g, (int64_t)sms * 16);
  return (int)std::max<int64_t>(g, 1);
}

constexpr size_t kPanelSmemBytes = 200 * 1024;

// ~one CTA per SM for tall panels, at least 32 rows per CTA, and few enough
// rows that the step kernel's tile (R x nc values) fits in shared memory.
void panel_geometry(int mp, int nc, size_t elem, int sms, int& C, int& R) {
  const int rmax = std::max(8, (int)std::min<size_t>(2048, (kPanelSmemBytes / elem - nc) / std::max(nc, 1)));
  C = std::max(1, std::min(sms, ceil_div(mp, 32)));
  C = std::max(C, ceil_div(mp, rmax));
  R = ceil_div(std::max(mp, 1), C);
  C = ceil_div(std::max(mp, 1), R);
}

}  // namespace

template <typename T>
size_t panel_scratch_elems(int mp, int nc, int sms) {
  int C, R;
  panel_geometry(mp, nc, sizeof(T), sms, C, R);
  // multi-launch path: part [C][nc+1] + rowbuf[2][nc] + coef[2][NCOEF+nc] + counter/piv (as T) + slack;
  // persistent path: its flagged exchange words after 16-byte alignment
  const size_t steps = (size_t)C * (nc + 1) + 2 * (size_t)nc + 2 * (size_t)(NCOEF + nc) + 2 * (size_t)nc + 64;
  const size_t words = (8 * panel_exchange_words(nc, C, sizeof(T)) + 16) / sizeof(T) + 1;
  return std::max(steps, words);
}

struct PanelScratch {};

template <typename T>
static void carve_panel(T* scratch, int C, int nc, T*& part, T*& rowbuf, T*& coef, int*& counter, int*& piv) {
  part = scratch;
  rowbuf = part + (size_t)C * (nc + 1);
  coef = rowbuf + 2 * (size_t)nc;
  T* tail = coef + 2 * (size_t)(NCOEF + nc);
  // align tail to 16 bytes for the int area
  uintptr_t p = reinterpret_cast<uintptr_t>(tail);
  p = (p + 15) & ~uintptr_t(15);
  counter = reinterpret_cast<int*>(p);
  piv = counter + 4;
}

template <typename T>
void panel_qr(const Ctx& c, int mp, int nc, T* P, int ldp, T* tau, T* scratch) {
  if (mp <= 0 || nc <= 0) return;
  int C, R;
  panel_geometry(mp, nc, sizeof(T), c.sms, C, R);
  // one cooperative launch with the panel resident in shared memory when it fits
  if (panel_qr_persist<T>(c, mp, nc, P, ldp, tau, scratch, C, R)) return;
  T *part, *rowbuf, *coef;
  int *counter, *piv;
  carve_panel(scratch, C, nc, part, rowbuf, coef, counter, piv);
  cudaMemsetAsync(counter, 0, sizeof(int), c.stream);
  PanelArgs a{mp, nc, R, ldp};
  const size_t sm_init = sizeof(T) * (size_t)nc;
  const size_t sm_step = sizeof(T) * ((size_t)nc + (size_t)nc * R);
  if (sm_step > 48 * 1024)
    cudaFuncSetAttribute(k_panel_step<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_step);
  k_panel_init<T><<<C, PT, sm_init, c.stream>>>(a, P, part, rowbuf, coef, tau, counter, c.status);
  note_launch(c, 1 + nc);
  for (int j = 0; j < nc; ++j) {
    const T* cin = coef + (size_t)(j & 1) * (NCOEF + nc);
    T* cout = coef + (size_t)((j + 1) & 1) * (NCOEF + nc);
    T* rb = rowbuf + (size_t)((j + 1) & 1) * nc;
    k_panel_step<T><<<C, PT, sm_step, c.stream>>>(j, a, P, cin, cout, part, rb, tau, counter, c.status);
  }
}

template <typename T>
void qrcp_block(const Ctx& c, int m, int r0, int c0, int nc, T* A, int lda, int32_t* perm, T* tau, T* scratch) {
  const int mp = m - r0;
  if (mp <= 0 || nc <= 0) return;
  const int nsteps = std::min(nc, mp - 1);
  int C, R;
  panel_geometry(mp, nc, sizeof(T), c.sms, C, R);
  T *part, *rowbuf, *coef;
  int *counter, *piv;
  carve_panel(scratch, C, nc, part, rowbuf, coef, counter, piv);
  cudaMemsetAsync(counter, 0, sizeof(int), c.stream);
  set_mat<T>(c, nc, 1, T(0), tau, nc);
  PanelArgs a{mp, nc, R, lda};
  T* P = A + r0 + (size_t)c0 * lda;
  const size_t sm_small = sizeof(T) * (size_t)nc;
  const size_t sm_apply = sizeof(T) * ((size_t)nc + (size_t)R);
  if (nsteps <= 0) return;
  // r0 == c0 for every caller (the block sits on the diagonal)
  k_qrcp_init<T><<<C, PT, sm_small, c.stream>>>(a, P, part, piv, counter);
  note_launch(c, 1 + 2 * (int64_t)nsteps);
  for (int j = 0; j < nsteps; ++j) {
    k_qrcp_pick<T><<<C, PT, sm_small, c.stream>>>(j, a, c0, m, A, lda, perm, piv, part, rowbuf, coef, tau, counter,
                                                 c.status);
    k_qrcp_apply<T><<<C, PT, sm_apply, c.stream>>>(j, nsteps, a, P, coef, part, piv, counter);
  }
}

template <typename T>
void larft_tri(const Ctx& c, int kb, const T* gram, int ldg, const T* tau, T* Tm, int ldt) {
  if (kb <= 0) return;
  // column-parallel back substitution while G's triangle fits in shared memory
  const size_t inv_sm = sizeof(T) * ((size_t)kb + (size_t)kb * (kb - 1) / 2);
  if (kb <= 32 * kLarftRows && inv_sm <= 200 * 1024) {
    if (inv_sm > 48 * 1024) cudaFuncSetAttribute(k_larft_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)inv_sm);
    k_larft_inv<T><<<kb, kLarftT, inv_sm, c.stream>>>(kb, gram, ldg, tau, Tm, ldt);
    note_launch(c);
    return;
  }
  k_larft_tri<T><<<1, 256, 0, c.stream>>>(kb, gram, ldg, tau, Tm, ldt);
  note_launch(c);
}

template <typename T>
void gram_from_lower(const Ctx& c, int kb, const T* L, int ldl, T* gram, int ldg) {
  if (kb <= 0) return;
  k_gram_from_lower<T><<<ceil_div(kb * kb, 256), 256, 0, c.stream>>>(kb, L, ldl, gram, ldg);
  note_launch(c);
}
template void gram_from_lower<double>(const Ctx&, int, const double*, int, double*, int);
template void gram_from_lower<float>(const Ctx&, int, const float*, int, float*, int);

template <typename T>
void transpose_mat(const Ctx& c, int r, int cols, const T* src, int lds, T* dst, int ldd) {
  if (r <= 0 || cols <= 0) return;
  dim3 g(ceil_div(r, 32), ceil_div(cols, 32));
  k_transpose<T><<<g, 256, 0, c.stream>>>(r, cols, src, lds, dst, ldd);
  note_launch(c);
}

template <typename T>
void copy_mat(const Ctx& c, int r, int cols, const T* src, int lds, T* dst, int ldd) {
  if (r <= 0 || cols <= 0) return;
  k_copy_mat<T><<<grid1d((int64_t)r * cols, c.sms), 256, 0, c.stream>>>(r, cols, src, lds, dst, ldd);
  note_launch(c);
}

template <typename T>
void set_mat(const Ctx& c, int r, int cols, T val, T* dst, int ldd) {
  if (r <= 0 || cols <= 0) return;
  k_set_mat<T><<<grid1d((int64_t)r * cols, c.sms), 256, 0, c.stream>>>(r, cols, val, dst, ldd);
  note_launch(c);
}

template <typename T>
void make_vx(const Ctx& c, int mp, int kb, const T* F, int ldf, T* V, int ldv) {
  if (mp <= 0 || kb <= 0) return;
  k_make_vx<T><<<grid1d((int64_t)mp * kb, c.sms), 256, 0, c.stream>>>(mp, kb, F, ldf, V, ldv);
  note_launch(c);
}

template <typename T>
void make_vlow(const Ctx& c, int mp, int kb, const T* F, int ldf, T* V, int ldv) {
  if (mp <= 0 || kb <= 0) return;
  k_make_vlow<T><<<grid1d((int64_t)mp * kb, c.sms), 256, 0, c.stream>>>(mp, kb, F, ldf, V, ldv);
  note_launch(c);
}

template <typename T>
void add_mat(const Ctx& c, int r, int cols, T alpha, const T* src, int lds, T* dst, int ldd) {
  if (r <= 0 || cols <= 0) return;
  k_add_mat<T><<<grid1d((int64_t)r * cols, c.sms), 256, 0, c.stream>>>(r, cols, alpha, src, lds, dst, ldd);
  note_launch(c);
}

#define RQR_INST(T)                                                                                      \
  template void make_vlow<T>(const Ctx&, int, int, const T*, int, T*, int);                               \
  template void add_mat<T>(const Ctx&, int, int, T, const T*, int, T*, int);                              \
  template size_t panel_scratch_elems<T>(int, int, int);                                                \
  template void panel_qr<T>(const Ctx&, int, int, T*, int, T*, T*);                                       \
  template void qrcp_block<T>(const Ctx&, int, int, int, int, T*, int, int32_t*, T*, T*);                 \
  template void larft_tri<T>(const Ctx&, int, const T*, int, const T*, T*, int);                          \
  template void copy_mat<T>(const Ctx&, int, int, const T*, int, T*, int);                                \
  template void transpose_mat<T>(const Ctx&, int, int, const T*, int, T*, int);                           \
  template void set_mat<T>(const Ctx&, int, int, T, T*, int);                                             \
  template void make_vx<T>(const Ctx&, int, int, const T*, int, T*, int);
RQR_INST(double)
RQR_INST(float)
#undef RQR_INST

}  // namespace rqr
