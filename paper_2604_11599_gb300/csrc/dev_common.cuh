// dev_common.cuh -- device helpers shared by the libsv kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sv_plan.h"

namespace svk {

template <typename T> struct CxT;
template <> struct CxT<float> { using V = float2; using V4 = float4; };
template <> struct CxT<double> { using V = double2; using V4 = double2; };

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

// m0*x + m1*y (complex)
template <typename V>
__device__ __forceinline__ V cmac2(V m0, V x, V m1, V y) {
  return mkc(fma(m0.x, x.x, fma(-m0.y, x.y, fma(m1.x, y.x, -m1.y * y.y))),
             fma(m0.x, x.y, fma(m0.y, x.x, fma(m1.x, y.y, m1.y * y.x))));
}
template <typename V>
__device__ __forceinline__ V cmul(V a, V b) {
  return mkc(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename V>
__device__ __forceinline__ V cadd(V a, V b) { return mkc(a.x + b.x, a.y + b.y); }

// ---------------------------------------------------------------------- shared-memory swizzle
// Tile-local amplitude index x is stored at x ^ fold(x >> B), fold = XOR of the
// B-bit groups, so tile-local bit p lands on bank bit (p mod B).  B = 4 for
// 8-byte amplitudes (16 per 128-byte row), 3 for 16-byte amplitudes.  The map
// is linear over GF(2): swz(a ^ b) = swz(a) ^ swz(b).
template <typename T> struct SwzBits;
template <> struct SwzBits<float> { static constexpr int B = 4; };
template <> struct SwzBits<double> { static constexpr int B = 3; };

template <typename T>
__device__ __forceinline__ uint32_t swz(uint32_t x) {
  constexpr int B = SwzBits<T>::B;
  uint32_t y = x >> B, f = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    f ^= y & ((1u << B) - 1);
    y >>= B;
  }
  return x ^ f;
}

// scatter the low bits of v to the positions pos[0..nb-1]
__device__ __forceinline__ uint32_t deposit_bits(uint32_t v, const uint8_t* pos, int nb) {
  uint32_t out = 0;
  for (int k = 0; k < nb; ++k) out |= ((v >> k) & 1u) << pos[k];
  return out;
}

// ---------------------------------------------------------------------- Philox4x64-10
// Counter-based generator of Salmon et al. (SC'11), 4 words of 64 bits, 10
// rounds: each round multiplies counter words 0 and 2 by the Philox
// multipliers (high/low halves), XORs the high halves with words 1, 3 and the
// round key; the key advances by the Weyl increments between rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = M0 * c[0], hi0 = __umul64hi(M0, c[0]);
    const uint64_t lo1 = M1 * c[2], hi1 = __umul64hi(M1, c[2]);
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

// uniform in [0,1) with 53 bits for draw (seed, stream, shot, m)
__device__ __forceinline__ double draw_uniform(uint64_t seed, uint64_t stream, uint64_t shot, uint64_t m) {
  uint64_t c[4] = {shot, m, 0ull, 0ull};
  philox4x64_10(c, seed, stream);
  return (double)(c[0] >> 11) * 0x1.0p-53;
}

}  // namespace svk
