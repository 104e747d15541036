// rng.cu -- Gaussian sketching matrices (Sec. 4.1: Omega with i.i.d. N(0,1)
// entries) from the counter-based Philox4x32-10 generator (Salmon, Moraes,
// Dror, Shaw, SC'11) and the Box-Muller transform. Stream layout: element e is
// lane e%4 of the block with counter {lo(e/4), hi(e/4), lo(stream),
// hi(stream)} and key {lo(seed), hi(seed)}; lanes (0,1) and (2,3) form the
// Box-Muller pairs with u = (x + 0.5) 2^-32.
#include "common.cuh"
#include "philox.cuh"

namespace rqr {

namespace {

template <typename T>
__global__ void k_gauss_fill(uint64_t seed, uint64_t stream, int64_t count, T* out) {
  const int64_t nblk = (count + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    double z[4];
    gauss4((uint64_t)b, seed, stream, z);
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (4 * b + t < count) out[4 * b + t] = (T)z[t];
  }
}

template <typename T>
__global__ void k_gauss_fill_2d(uint64_t seed, uint64_t stream, int r, int cols, T* out, int ld) {
  const int64_t count = (int64_t)r * cols;
  const int64_t nblk = (count + 3) / 4;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
    double z[4];
    gauss4((uint64_t)b, seed, stream, z);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = 4 * b + t;
      if (e < count) {
        const int64_t i = e % r, j = e / r;
        out[i + j * (int64_t)ld] = (T)z[t];
      }
    }
  }
}

__global__ void k_philox_raw(uint32_t ctr0, uint32_t ctr2, uint32_t ctr3, uint32_t k0, uint32_t k1, int64_t count,
                             uint32_t* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c0 = ctr0 + (uint32_t)i, c1 = 0, c2 = ctr2, c3 = ctr3;
    philox10(c0, c1, c2, c3, k0, k1);
    out[4 * i + 0] = c0;
    out[4 * i + 1] = c1;
    out[4 * i + 2] = c2;
    out[4 * i + 3] = c3;
  }
}

int grid_for(int64_t items, int sms) {
  int64_t g = (items + 255) / 256;
  if (g > (int64_t)sms * 16) g = (int64_t)sms * 16;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

template <typename T>
void gauss_fill(const Ctx& c, uint64_t seed, uint64_t stream, int64_t count, T* out) {
  if (count <= 0) return;
  k_gauss_fill<T><<<grid_for((count + 3) / 4, c.sms), 256, 0, c.stream>>>(seed, stream, count, out);
  note_launch(c);
}

template <typename T>
void gauss_fill_2d(const Ctx& c, uint64_t seed, uint64_t stream, int r, int cols, T* out, int ld) {
  const int64_t count = (int64_t)r * cols;
  if (count <= 0) return;
  k_gauss_fill_2d<T><<<grid_for((count + 3) / 4, c.sms), 256, 0, c.stream>>>(seed, stream, r, cols, out, ld);
  note_launch(c);
}

void philox_raw(const Ctx& c, uint32_t ctr0, uint32_t ctr2, uint32_t ctr3, uint32_t k0, uint32_t k1, int64_t count,
                uint32_t* out) {
  if (count <= 0) return;
  k_philox_raw<<<grid_for(count, c.sms), 256, 0, c.stream>>>(ctr0, ctr2, ctr3, k0, k1, count, out);
  note_launch(c);
}

template void gauss_fill<double>(const Ctx&, uint64_t, uint64_t, int64_t, double*);
template void gauss_fill<float>(const Ctx&, uint64_t, uint64_t, int64_t, float*);
template void gauss_fill_2d<double>(const Ctx&, uint64_t, uint64_t, int, int, double*, int);
template void gauss_fill_2d<float>(const Ctx&, uint64_t, uint64_t, int, int, float*, int);

}  // namespace rqr
