// svd.cu -- small FP64 singular value decomposition for the l -> b reduction
// of the orthonormal-pivot sketch (Sec. 4.2 with the over-sampling of
// Sec. 4.3): one-sided Jacobi (Hestenes 1958) on the r x c matrix M,
// accumulating the c x c rotation J so that M J has orthogonal columns; the
// columns of J sorted by the norms of M J are the right singular vectors of M.
//
// Parallel ordering: the round-robin (circle) tournament pairs the c columns
// into c/2 disjoint pairs per round, so all rotations of a round touch
// different columns and run at once, one warp per pair. The rounds of a sweep
// are separated by the hardware cluster barrier of an 8-CTA thread-block
// cluster (no software spin). Sweeps stop when no pair rotated, at most
// kMaxSweeps times.
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rqr {

namespace {

constexpr int kClusterCtas = 8;
constexpr int kThreads = 512;
constexpr int kMaxSweeps = 60;

__device__ __forceinline__ void pair_of_round(int k, int r, int cp, int& a, int& b) {
  // circle method: player 0 fixed, players 1..cp-1 rotate by r
  a = (k == 0) ? 0 : 1 + ((k - 1 + r) % (cp - 1));
  b = 1 + ((cp - 2 - k + r) % (cp - 1));
}

__global__ void __cluster_dims__(kClusterCtas, 1, 1) __launch_bounds__(kThreads)
    k_jacobi(int r, int c, double* M, int ldm, double* J, int ldj, int* flags, double tol) {
  cg::cluster_group cluster = cg::this_cluster();
  const int cta = (int)cluster.block_rank();
  const int lane = threadIdx.x & 31;
  const int gw = cta * (kThreads / 32) + (threadIdx.x >> 5);
  const int nw = kClusterCtas * (kThreads / 32);
  const int cp = c + (c & 1);  // even number of players (c itself, or c + one dummy)
  // J = I
  for (int e = cta * kThreads + threadIdx.x; e < c * c; e += kClusterCtas * kThreads) {
    const int i = e % c, j = e / c;
    J[i + (size_t)j * ldj] = i == j ? 1.0 : 0.0;
  }
  volatile int* vflags = flags;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    if (cta == 0 && threadIdx.x == 0) vflags[sweep & 1] = 0;
    cluster.sync();
    for (int rd = 0; rd < cp - 1; ++rd) {
      for (int k = gw; k < cp / 2; k += nw) {
        int a, b;
        pair_of_round(k, rd, cp, a, b);
        if (a >= c || b >= c) continue;  // dummy player
        const int i = min(a, b), j = max(a, b);
        double* x = M + (size_t)i * ldm;
        double* y = M + (size_t)j * ldm;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int t = lane; t < r; t += 32) {
          const double xi = x[t], yi = y[t];
          al += xi * xi;
          be += yi * yi;
          ga += xi * yi;
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (ga == 0.0 || fabs(ga) <= tol * sqrt(al * be)) continue;
        const double zeta = (be - al) / (2.0 * ga);
        const double t = (zeta < 0.0 ? -1.0 : 1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int q = lane; q < r; q += 32) {
          const double xi = x[q], yi = y[q];
          x[q] = cs * xi - sn * yi;
          y[q] = sn * xi + cs * yi;
        }
        double* u = J + (size_t)i * ldj;
        double* w = J + (size_t)j * ldj;
        for (int q = lane; q < c; q += 32) {
          const double ui = u[q], wi = w[q];
          u[q] = cs * ui - sn * wi;
          w[q] = sn * ui + cs * wi;
        }
        if (lane == 0) vflags[sweep & 1] = 1;
      }
      cluster.sync();
    }
    if (vflags[sweep & 1] == 0) break;
  }
}

// Column norms of M J (stored in M), ranks by descending norm (ties: lower
// column first), and the sorted copy Js = J(:, order[0:nkeep]) (c x nkeep).
__global__ void __launch_bounds__(1024) k_jacobi_sort(int r, int c, const double* M, int ldm, const double* J,
                                                      int ldj, int nkeep, double* Js, int ldjs, double* sv,
                                                      int* order) {
  extern __shared__ double nrm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int col = warp; col < c; col += nwarp) {
    const double* x = M + (size_t)col * ldm;
    double s = 0.0;
    for (int t = lane; t < r; t += 32) s += x[t] * x[t];
    s = warp_sum(s);
    if (lane == 0) nrm[col] = sqrt(s);
  }
  __syncthreads();
  for (int col = threadIdx.x; col < c; col += blockDim.x) {
    const double v = nrm[col];
    int rank = 0;
    for (int o = 0; o < c; ++o) rank += (nrm[o] > v) || (nrm[o] == v && o < col);
    order[rank] = col;
    sv[rank] = v;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < c * nkeep; e += blockDim.x) {
    const int i = e % c, k = e / c;
    Js[i + (size_t)k * ldjs] = J[i + (size_t)order[k] * ldj];
  }
}

// M (c x kk, ld ldm) = R^T where R = upper triangle of rows 0..kk-1 of F (kk x c).
template <typename T>
__global__ void k_r_transpose(int kk, int c, const T* __restrict__ F, int ldf, T* __restrict__ M, int ldm) {
  const int64_t n = (int64_t)c * kk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e % c), i = (int)(e / c);
    M[t + (int64_t)i * ldm] = i <= t ? F[i + (int64_t)t * ldf] : T(0);
  }
}

// dst(i, j) = src(i, j) strictly below the diagonal, 0 elsewhere (r x cols).
template <typename T>
__global__ void k_copy_lower(int r, int cols, const T* __restrict__ s, int lds, T* __restrict__ d, int ldd) {
  const int64_t n = (int64_t)r * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e % r), j = (int)(e / r);
    d[i + (int64_t)j * ldd] = i > j ? s[i + (int64_t)j * lds] : T(0);
  }
}

int grid_of(int64_t n, int sms) {
  int64_t g = (n + 255) / 256;
  g = std::min<int64_t>(g, (int64_t)sms * 16);
  return (int)std::max<int64_t>(g, 1);
}

}  // namespace

template <typename T>
void r_transpose(const Ctx& c, int kk, int cols, const T* F, int ldf, T* M, int ldm) {
  if (kk <= 0 || cols <= 0) return;
  k_r_transpose<T><<<grid_of((int64_t)kk * cols, c.sms), 256, 0, c.stream>>>(kk, cols, F, ldf, M, ldm);
  note_launch(c);
}

template <typename T>
void copy_lower(const Ctx& c, int r, int cols, const T* src, int lds, T* dst, int ldd) {
  if (r <= 0 || cols <= 0) return;
  k_copy_lower<T><<<grid_of((int64_t)r * cols, c.sms), 256, 0, c.stream>>>(r, cols, src, lds, dst, ldd);
  note_launch(c);
}

template void r_transpose<double>(const Ctx&, int, int, const double*, int, double*, int);
template void copy_lower<double>(const Ctx&, int, int, const double*, int, double*, int);
template void r_transpose<float>(const Ctx&, int, int, const float*, int, float*, int);
template void copy_lower<float>(const Ctx&, int, int, const float*, int, float*, int);

void jacobi_svd(const Ctx& c, int r, int cols, double* M, int ldm, double* J, int ldj, int nkeep, double* Js,
                int ldjs, double* sv, int* order, int* flags) {
  if (cols <= 0) return;
  k_jacobi<<<kClusterCtas, kThreads, 0, c.stream>>>(r, cols, M, ldm, J, ldj, flags, 1e-15);
  k_jacobi_sort<<<1, 1024, sizeof(double) * cols, c.stream>>>(r, cols, M, ldm, J, ldj, nkeep, Js, ldjs, sv, order);
  note_launch(c, 2);
}

// Finishes the diagonalisation of a b_i x b_i block (Sec. 6.2): with
// M = R11^T J from jacobi_svd (unsorted columns), `order` and the sorted norms
// sv, the right factor Vt(:, c) = M(:, order[c]) / sv[c]; a zero norm gets the
// first unit vector that two Gram-Schmidt passes against the columns already set
// leave with norm above 1/2, or, if none does, the one they leave with the
// largest norm, normalised. U' = Js is copied to DU, Vt to DV, and the upper
// triangle of the block (F, ld ldf) becomes diag(sv). One CTA.
__global__ void __launch_bounds__(256) k_diag_finish(int bi, const double* __restrict__ M, int ldm,
                                                     const int* __restrict__ order, const double* __restrict__ sv,
                                                     const double* __restrict__ Js, int ldjs, double* DU, int lddu,
                                                     double* DV, int lddv, double* F, int ldf) {
  __shared__ double red[8];
  __shared__ double s_norm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < bi * bi; e += blockDim.x) {
    const int i = e % bi, j = e / bi;
    DU[i + (size_t)j * lddu] = Js[i + (size_t)j * ldjs];
  }
  for (int c = 0; c < bi; ++c) {
    double* v = DV + (size_t)c * lddv;
    const double s = sv[c];
    if (s > 0.0) {
      const double* mc = M + (size_t)order[c] * ldm;
      for (int i = tid; i < bi; i += blockDim.x) v[i] = mc[i] / s;
      __syncthreads();
      continue;
    }
    // unit vector e_k, Gram-Schmidt twice against columns 0..c-1; returns the
    // residual norm (the same value in every thread)
    auto project_unit = [&](int e) -> double {
      for (int i = tid; i < bi; i += blockDim.x) v[i] = (i == e) ? 1.0 : 0.0;
      __syncthreads();
      for (int pass = 0; pass < 2; ++pass)
        for (int t = 0; t < c; ++t) {
          const double* u = DV + (size_t)t * lddv;
          double d = 0.0;
          for (int i = tid; i < bi; i += blockDim.x) d += u[i] * v[i];
          d = warp_sum(d);
          if (lane == 0) red[warp] = d;
          __syncthreads();
          if (tid == 0) {
            double sum = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
            s_norm = sum;
          }
          __syncthreads();
          d = s_norm;
          for (int i = tid; i < bi; i += blockDim.x) v[i] -= d * u[i];
          __syncthreads();
        }
      double nv = 0.0;
      for (int i = tid; i < bi; i += blockDim.x) nv += v[i] * v[i];
      nv = warp_sum(nv);
      if (lane == 0) red[warp] = nv;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
        s_norm = sqrt(sum);
      }
      __syncthreads();
      return s_norm;
    };
    // the first e_k left with norm above 1/2, else the one left with the
    // largest norm (their squared norms add up to bi - c >= 1)
    int best = 0;
    double best_nv = -1.0, nv = -1.0;
    bool done = false;
    for (int e = 0; e < bi && !done; ++e) {
      nv = project_unit(e);
      if (nv > 0.5) {
        done = true;
      } else if (nv > best_nv) {
        best_nv = nv;
        best = e;
      }
    }
    if (!done) nv = project_unit(best);
    for (int i = tid; i < bi; i += blockDim.x) v[i] /= nv;
    __syncthreads();
  }
  for (int e = tid; e < bi * bi; e += blockDim.x) {
    const int i = e % bi, j = e / bi;
    if (i <= j) F[i + (size_t)j * ldf] = i == j ? sv[j] : 0.0;
  }
}

void diag_finish(const Ctx& c, int bi, const double* M, int ldm, const int* order, const double* sv, const double* Js,
                 int ldjs, double* DU, int lddu, double* DV, int lddv, double* F, int ldf) {
  if (bi <= 0) return;
  k_diag_finish<<<1, 256, 0, c.stream>>>(bi, M, ldm, order, sv, Js, ldjs, DU, lddu, DV, lddv, F, ldf);
  note_launch(c);
}

}  // namespace rqr
