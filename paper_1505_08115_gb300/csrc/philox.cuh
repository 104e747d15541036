// philox.cuh -- the counter-based Philox4x32-10 generator (Salmon, Moraes,
// Dror, Shaw, SC'11) and the Box-Muller transform of the Gaussian sketches:
// block counter {lo(blk), hi(blk), lo(stream), hi(stream)}, key {lo(seed),
// hi(seed)}, lanes (0,1) and (2,3) form the Box-Muller pairs with
// u = (x + 0.5) 2^-32. Shared by rng.cu (rqr_gauss_fill) and batched.cu (the
// per-block sketches of the batched factorizations), so both draw the same
// stream.
#pragma once
#include <stdint.h>

namespace rqr {
namespace {

__device__ __forceinline__ void philox10(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3, uint32_t k0,
                                         uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = M0 * c0, hi0 = __umulhi(M0, c0);
    const uint32_t lo1 = M1 * c2, hi1 = __umulhi(M1, c2);
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += W0;
    k1 += W1;
  }
}

__device__ __forceinline__ void gauss4(uint64_t blk, uint64_t seed, uint64_t stream, double z[4]) {
  uint32_t c0 = (uint32_t)blk, c1 = (uint32_t)(blk >> 32), c2 = (uint32_t)stream, c3 = (uint32_t)(stream >> 32);
  philox10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
  const uint32_t x[4] = {c0, c1, c2, c3};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const double u1 = ((double)x[2 * h] + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)x[2 * h + 1] + 0.5) * 2.3283064365386963e-10;
    const double r = sqrt(-2.0 * log(u1));
    double s, co;
    sincospi(2.0 * u2, &s, &co);
    z[2 * h] = r * co;
    z[2 * h + 1] = r * s;
  }
}

}  // namespace
}  // namespace rqr
