// dev_common.cuh -- device helpers shared by the libsv kernels.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "sv_plan.h"

namespace svk {

template <typename T> struct CxT;
template <> struct CxT<float> { using V = float2; using V4 = float4; };
template <> struct CxT<double> { using V = double2; using V4 = double2; };

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

// two complex64 amplitudes in one 16-byte vector (complex128: one amplitude;
// the pair helpers are used for complex64 only)
__device__ __forceinline__ float2 pair_lo(float4 q) { return make_float2(q.x, q.y); }
__device__ __forceinline__ float2 pair_hi(float4 q) { return make_float2(q.z, q.w); }
__device__ __forceinline__ float4 make_pair4(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ double2 pair_lo(double2 q) { return q; }
__device__ __forceinline__ double2 pair_hi(double2 q) { return q; }
__device__ __forceinline__ double2 make_pair4(double2 a, double2) { return a; }

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
// Tile layout in 16-byte granules: granule g at g ^ fold(g >> 3), fold = XOR
// of 3-bit groups (the same map as tile_swizzle in sv_plan.h).  A = log2
// amplitudes per granule.  Linear over GF(2): swz(a ^ b) = swz(a) ^ swz(b).
template <typename T> struct GranuleBits;
template <> struct GranuleBits<float> { static constexpr int A = 1; };
template <> struct GranuleBits<double> { static constexpr int A = 0; };

template <typename T>
__device__ __forceinline__ uint32_t swz(uint32_t x) {
  constexpr int A = GranuleBits<T>::A;
  uint32_t y = x >> (A + 3), f = 0;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    f ^= y & 7u;
    y >>= 3;
  }
  return x ^ (f << A);
}

// Ampere-style asynchronous 16-byte global -> shared copies (no register staging)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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
