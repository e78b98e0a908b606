// pass_body.cuh -- device code of one state sweep, shared by the grid pass
// kernel (kern_pass.cu) and the persistent batched kernel (kern_batch.cu).
//
// One pass sweeps the state once.  A tile is the 2^M amplitudes that share
// the values of the n-M qubits outside the pass's tile set.  Tiles are read
// with 16-byte coalesced copies (runs of 2^L contiguous amplitudes): with no
// pending projector they stream in by cp.async, the next tile in flight while
// the current one is processed; otherwise they are loaded with the pending
// measurement projector applied on the way in (the collapse and 1/sqrt(p)
// renormalisation of the previous measurement group, fused into this load).
// In swizzled shared memory the tile is processed in stages: each thread
// pulls 16 amplitudes (four register qubits) into registers, applies the
// stage's gates there and writes them back.  If a measurement group follows,
// the |amp|^2 table of its qubits is accumulated (FP32 within a warp for
// complex64, FP64 across warps and CTAs) and one thread draws the outcomes
// (Philox4x64-10 keyed on seed, stream, shot and draw index), updates the
// classical register and evaluates the feed-forward predicates that follow
// (Sec. III-C) -- all on the device.
#pragma once
#include "dev_common.cuh"
#include "dev_tc.cuh"
#include "kernels.h"

namespace svk {
using namespace svp;

// ============================================================ gates on 16 registers
// a[j] holds the amplitude whose register bits are j; template parameters
// are register-bit positions, so every index below is a compile-time constant.

template <int P, typename V>
__device__ __forceinline__ void g_u(V* a, const V* m) {
  const V m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << P)) continue;
    const int k = j | (1 << P);
    const V x = a[j], y = a[k];
    a[j] = cmac2(m0, x, m1, y);
    a[k] = cmac2(m2, x, m3, y);
  }
}

template <int P, typename V>
__device__ __forceinline__ void g_r(V* a, const V* m) {
  const auto r00 = m[0].x, r01 = m[1].x, r10 = m[2].x, r11 = m[3].x;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << P)) continue;
    const int k = j | (1 << P);
    const V x = a[j], y = a[k];
    a[j] = mkc(fma(r00, x.x, r01 * y.x), fma(r00, x.y, r01 * y.y));
    a[k] = mkc(fma(r10, x.x, r11 * y.x), fma(r10, x.y, r11 * y.y));
  }
}

// RX: [c, -i s; -i s, c]
template <int P, typename V>
__device__ __forceinline__ void g_rx(V* a, const V* m) {
  const auto c = m[0].x, s = m[1].x;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << P)) continue;
    const int k = j | (1 << P);
    const V x = a[j], y = a[k];
    a[j] = mkc(fma(c, x.x, s * y.y), fma(c, x.y, -s * y.x));
    a[k] = mkc(fma(s, x.y, c * y.x), fma(-s, x.x, c * y.y));
  }
}

// Factored rotations (forward plans): the scalar factor m[1] is applied by the
// pass, so each output is one fused multiply-add per component.
// RX: form 0 [1 -it; -it 1] (t = m[0].x), form 1 [u -i; -i u] (u = m[0].x).
template <int P, typename V>
__device__ __forceinline__ void g_rxf(V* a, const V* m) {
  const auto k = m[0].x;
  if (m[0].y == 0) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << P)) continue;
      const int h = j | (1 << P);
      const V x = a[j], y = a[h];
      a[j] = mkc(fma(k, y.y, x.x), fma(-k, y.x, x.y));
      a[h] = mkc(fma(k, x.y, y.x), fma(-k, x.x, y.y));
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << P)) continue;
      const int h = j | (1 << P);
      const V x = a[j], y = a[h];
      a[j] = mkc(fma(k, x.x, y.y), fma(k, x.y, -y.x));
      a[h] = mkc(fma(k, y.x, x.y), fma(k, y.y, -x.x));
    }
  }
}

// RY: form 0 [1 -t; t 1], form 1 [u -1; 1 u].
template <int P, typename V>
__device__ __forceinline__ void g_ryf(V* a, const V* m) {
  const auto k = m[0].x;
  if (m[0].y == 0) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << P)) continue;
      const int h = j | (1 << P);
      const V x = a[j], y = a[h];
      a[j] = mkc(fma(-k, y.x, x.x), fma(-k, y.y, x.y));
      a[h] = mkc(fma(k, x.x, y.x), fma(k, x.y, y.y));
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if (j & (1 << P)) continue;
      const int h = j | (1 << P);
      const V x = a[j], y = a[h];
      a[j] = mkc(fma(k, x.x, -y.x), fma(k, x.y, -y.y));
      a[h] = mkc(fma(k, y.x, x.x), fma(k, y.y, x.y));
    }
  }
}

// diag(1, p) on bit P (the factor d0 of diag(d0, d1) is applied by the pass)
template <int P, typename V>
__device__ __forceinline__ void g_dz(V* a, const V* m) {
  const V p = m[0];
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j & (1 << P)) a[j] = cmul(p, a[j]);
}

template <int P, typename V>
__device__ __forceinline__ void g_d(V* a, const V* m) {
  const V d0 = m[0], d1 = m[1];
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = cmul((j & (1 << P)) ? d1 : d0, a[j]);
}

template <int P, typename V>
__device__ __forceinline__ void g_x(V* a, const V*) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << P)) continue;
    const int k = j | (1 << P);
    const V t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

template <int C, int T, typename V>
__device__ __forceinline__ void g_cu(V* a, const V* m) {
  const V m0 = m[0], m1 = m[1], m2 = m[2], m3 = m[3];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!(j & (1 << C)) || (j & (1 << T))) continue;
    const int k = j | (1 << T);
    const V x = a[j], y = a[k];
    a[j] = cmac2(m0, x, m1, y);
    a[k] = cmac2(m2, x, m3, y);
  }
}

template <int C, int T, typename V>
__device__ __forceinline__ void g_cx(V* a, const V*) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!(j & (1 << C)) || (j & (1 << T))) continue;
    const int k = j | (1 << T);
    const V t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

template <int A, int B, typename V>
__device__ __forceinline__ void g_cz(V* a, const V*) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if ((j & (1 << A)) && (j & (1 << B))) a[j] = mkc(-a[j].x, -a[j].y);
}

template <int C, int T, typename V>
__device__ __forceinline__ void g_cd(V* a, const V* m) {
  const V d0 = m[0], d1 = m[1];
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (j & (1 << C)) a[j] = cmul((j & (1 << T)) ? d1 : d0, a[j]);
}

template <int A, int B, typename V>
__device__ __forceinline__ void g_swap(V* a, const V*) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!(j & (1 << A)) || (j & (1 << B))) continue;
    const int k = (j ^ (1 << A)) | (1 << B);
    const V t = a[j];
    a[j] = a[k];
    a[k] = t;
  }
}

// dense 4x4; matrix index bit 0 <-> register bit P0, bit 1 <-> P1
template <int P0, int P1, typename V>
__device__ __forceinline__ void g_u4(V* a, const V* m) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if ((j & (1 << P0)) || (j & (1 << P1))) continue;
    const int i0 = j, i1 = j | (1 << P0), i2 = j | (1 << P1), i3 = j | (1 << P0) | (1 << P1);
    const V v0 = a[i0], v1 = a[i1], v2 = a[i2], v3 = a[i3];
    a[i0] = cadd(cmac2(m[0], v0, m[1], v1), cmac2(m[2], v2, m[3], v3));
    a[i1] = cadd(cmac2(m[4], v0, m[5], v1), cmac2(m[6], v2, m[7], v3));
    a[i2] = cadd(cmac2(m[8], v0, m[9], v1), cmac2(m[10], v2, m[11], v3));
    a[i3] = cadd(cmac2(m[12], v0, m[13], v1), cmac2(m[14], v2, m[15], v3));
  }
}

template <typename V>
__device__ __forceinline__ void g_d16(V* a, const V* m) {
  V w[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    V acc = mkc(decltype(a[0].x)(0), decltype(a[0].x)(0));
#pragma unroll
    for (int c = 0; c < 16; c += 2) acc = cadd(acc, cmac2(m[r * 16 + c], a[c], m[r * 16 + c + 1], a[c + 1]));
    w[r] = acc;
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) a[r] = w[r];
}

// Dense 16 x 16 unitary on the register qubits of every group of a
// 2^12-amplitude complex64 tile, on the tensor cores (dev_tc.cuh).  Collective:
// all 256 threads call it together, each holding its group (= its thread
// index) in a[].  Warp w writes its 32 rows (TF32 high and low parts) into
// tensor-memory lanes 32 (w mod 4) ... + 31, columns 64 (w / 4) ...; one
// thread then issues both 128-row products back to back (rows 0..127 into the
// accumulator at column 128, rows 128..255 into the one at 160) and every
// thread reads its output row from its own lane once they complete.
// B of a dense gate (its 32 x 32 real form, TF32 high and low parts) into a
// slot; once per pass, by all threads.
template <typename V>
__device__ __forceinline__ void d16_build_b(const V* m, TcShared& s, int slot) {
  unsigned char* bt0 = reinterpret_cast<unsigned char*>(s.bt[slot][0]);
  unsigned char* bt1 = reinterpret_cast<unsigned char*>(s.bt[slot][1]);
  for (int e = threadIdx.x; e < 256; e += PASS_THREADS) {  // entries (2r + i, 2c + j) from U[r][c] = m[16 r + c]
    const int r = e >> 4, c = e & 15;
    const V u = m[e];
    const float v[4] = {float(u.x), float(-u.y), float(u.y), float(u.x)};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t off = cm_off(uint32_t(2 * r + (q >> 1)), uint32_t(2 * c + (q & 1)));
      const float hi = tf32_hi(v[q]);
      *reinterpret_cast<float*>(bt0 + off) = hi;
      *reinterpret_cast<float*>(bt1 + off) = v[q] - hi;
    }
  }
}

template <typename V>
__device__ __forceinline__ void d16_tc(V* a, const V* m, TcCtx& tc) {
  const int tid = threadIdx.x, warp = tid >> 5;
  TcShared& s = *tc.s;
  const uint32_t mo = uint32_t(m - static_cast<const V*>(tc.smat));
  int slot = 0;
#pragma unroll
  for (int k = 1; k < TC_SLOTS; ++k)
    if (s.slot_mat[k] == mo) slot = k;
  unsigned char* bt0 = reinterpret_cast<unsigned char*>(s.bt[slot][0]);
  unsigned char* bt1 = reinterpret_cast<unsigned char*>(s.bt[slot][1]);
  const uint32_t lane_base = uint32_t(32 * (warp & 3)) << 16;
  const uint32_t half = uint32_t(warp >> 2);
  {  // this thread's row, 16 columns at a time: high parts (columns 0..31), low parts (32..63)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t w[16];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const V x = a[8 * (q & 1) + j];
        const float h0 = tf32_hi(x.x), h1 = tf32_hi(x.y);
        w[2 * j] = __float_as_uint(q < 2 ? h0 : x.x - h0);
        w[2 * j + 1] = __float_as_uint(q < 2 ? h1 : x.y - h1);
      }
      tmem_st16(tc.tmem + lane_base + 64u * half + 16u * uint32_t(q), w);
    }
  }
  tmem_wait_st();
  tc_fence_before();
  __syncthreads();  // all rows in tensor memory, previous results read
  if (tid == 0 && tc.ok) {
    tc_fence_after();
    constexpr uint32_t IDESC = idesc_tf32(128, 32);
    const uint32_t b0 = smem_u32(bt0), b1 = smem_u32(bt1);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t d = tc.tmem + 128u + 32u * uint32_t(h), ah = tc.tmem + 64u * uint32_t(h);
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // K = 8 per MMA; three products per k-step
        const uint32_t ko = uint32_t(k) * 256u, kc = uint32_t(k) * 8u;
        mma_tf32_ts(d, ah + kc, smem_desc(b0 + ko, 128, 1024), IDESC, k > 0 ? 1u : 0u);
        mma_tf32_ts(d, ah + kc, smem_desc(b1 + ko, 128, 1024), IDESC, 1u);
        mma_tf32_ts(d, ah + 32u + kc, smem_desc(b0 + ko, 128, 1024), IDESC, 1u);
      }
    }
    mma_commit(&s.bar);
  }
  // After a wait ran out the thread issues and waits no more (the barriers
  // stay uniform), so the pass ends within one more wait period and the run
  // reports SV_ERR_TIMEOUT with the state undefined; tensor-memory reads of
  // an unfinished batch only yield garbage.  The issuing thread remembers
  // the batch it gave up on: the CTA drains it (tc_drain) before it frees
  // its tensor memory, so no MMA can write columns it no longer owns.
  if (tc.ok && !mbar_wait(&s.bar, tc.phase & 1u, TC_WAIT_POLLS)) {
    tc.ok = false;
    if (tid == 0) tc.drain = 1u + (tc.phase & 1u);
  }
  ++tc.phase;
  tc_fence_after();
  uint32_t r[32];
  tmem_ld32(tc.tmem + lane_base + 128u + 32u * half, r);
  tmem_wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) a[j] = mkc(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
}

// A dense four-qubit unitary: on the tensor cores where the pass enabled them
// (complex64, 2^12-amplitude tiles), else on the FP32 / FP64 pipes.
// The tensor-core variant of a pass kernel runs only with the tensor-core path
// on (sv_set_dense_tc), so it carries no FP32 fallback (its registers would
// spill); the status records it if that is ever violated.
template <typename T, int M, bool TC, typename V>
__device__ __forceinline__ void d16_apply(V* a, const V* m, V* tb, TcCtx& tc) {
  if constexpr (TC && sizeof(T) == 4 && M == 12) {
    if (tc.on) d16_tc(a, m, tc);
    else if (threadIdx.x == 0) tc.ok = false;
  } else {
    g_d16(a, m);
  }
}

#define SVK_K1(OP, FN)                          \
  case OP * 16 + 0: FN<0>(a, mt); break;        \
  case OP * 16 + 4: FN<1>(a, mt); break;        \
  case OP * 16 + 8: FN<2>(a, mt); break;        \
  case OP * 16 + 12: FN<3>(a, mt); break;

#define SVK_K2(OP, FN)                          \
  case OP * 16 + 1: FN<0, 1>(a, mt); break;     \
  case OP * 16 + 2: FN<0, 2>(a, mt); break;     \
  case OP * 16 + 3: FN<0, 3>(a, mt); break;     \
  case OP * 16 + 4: FN<1, 0>(a, mt); break;     \
  case OP * 16 + 6: FN<1, 2>(a, mt); break;     \
  case OP * 16 + 7: FN<1, 3>(a, mt); break;     \
  case OP * 16 + 8: FN<2, 0>(a, mt); break;     \
  case OP * 16 + 9: FN<2, 1>(a, mt); break;     \
  case OP * 16 + 11: FN<2, 3>(a, mt); break;    \
  case OP * 16 + 12: FN<3, 0>(a, mt); break;    \
  case OP * 16 + 13: FN<3, 1>(a, mt); break;    \
  case OP * 16 + 14: FN<3, 2>(a, mt); break;

// one switch on key = op * 16 + p0 * 4 + p1 selects the gate and its register positions
// ---- backward (adjoint) stages: phi in registers 0..7, lambda in 8..15
// Re <lambda| M |phi> over the register pairs of position P (or of target T
// where control C is 1).
template <int P, typename V>
__device__ __forceinline__ auto g_dot(const V* a, const V* m) -> decltype(a[0].x) {
  decltype(a[0].x) r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j & (1 << P)) continue;
    const int k = j | (1 << P);
    const V w0 = cmac2(m[0], a[j], m[1], a[k]);
    const V w1 = cmac2(m[2], a[j], m[3], a[k]);
    r += a[j + 8].x * w0.x + a[j + 8].y * w0.y + a[k + 8].x * w1.x + a[k + 8].y * w1.y;
  }
  return r;
}

template <int C, int T, typename V>
__device__ __forceinline__ auto g_cdot(const V* a, const V* m) -> decltype(a[0].x) {
  decltype(a[0].x) r = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (!(j & (1 << C)) || (j & (1 << T))) continue;
    const int k = j | (1 << T);
    const V w0 = cmac2(m[0], a[j], m[1], a[k]);
    const V w1 = cmac2(m[2], a[j], m[3], a[k]);
    r += a[j + 8].x * w0.x + a[j + 8].y * w0.y + a[k + 8].x * w1.x + a[k + 8].y * w1.y;
  }
  return r;
}

template <typename V>
__device__ __forceinline__ auto apply_dot(const V* a, uint32_t key, const V* mt) -> decltype(a[0].x) {
  switch (key) {
    case OP_DOT * 16 + 0: return g_dot<0>(a, mt);
    case OP_DOT * 16 + 4: return g_dot<1>(a, mt);
    case OP_DOT * 16 + 8: return g_dot<2>(a, mt);
    case OP_CDOT * 16 + 1: return g_cdot<0, 1>(a, mt);
    case OP_CDOT * 16 + 2: return g_cdot<0, 2>(a, mt);
    case OP_CDOT * 16 + 4: return g_cdot<1, 0>(a, mt);
    case OP_CDOT * 16 + 6: return g_cdot<1, 2>(a, mt);
    case OP_CDOT * 16 + 8: return g_cdot<2, 0>(a, mt);
    case OP_CDOT * 16 + 9: return g_cdot<2, 1>(a, mt);
    default: return 0;
  }
}

template <typename V>
__device__ __forceinline__ void apply_gate(V* a, uint32_t key, const V* mt) {
  switch (key) {
    SVK_K1(OP_U, g_u)
    SVK_K1(OP_R, g_r)
    SVK_K1(OP_RX, g_rx)
    SVK_K1(OP_RXF, g_rxf)
    SVK_K1(OP_RYF, g_ryf)
    SVK_K1(OP_DZ, g_dz)
    SVK_K1(OP_D, g_d)
    SVK_K1(OP_X, g_x)
    SVK_K2(OP_CU, g_cu)
    SVK_K2(OP_CX, g_cx)
    SVK_K2(OP_CZ, g_cz)
    SVK_K2(OP_CD, g_cd)
    SVK_K2(OP_SWAP, g_swap)
    SVK_K2(OP_U4, g_u4)
    case OP_D16 * 16: g_d16(a, mt); break;
    default: break;
  }
}

// ============================================================ gate matrices (FP64)
// OpenQASM 3 standard-gate definitions; m = [m00 m01; m10 m11] of the target.
static __device__ void std_gate_2x2(int gate, const double* t, double2* m) {
  const double h = 0.70710678118654752440;
  double c, s, sp, cp, sl, cl;
  for (int k = 0; k < 4; ++k) m[k] = make_double2(0, 0);
  switch (gate) {
    case SV_H: case SV_CH: m[0] = m[1] = m[2] = make_double2(h, 0); m[3] = make_double2(-h, 0); break;
    case SV_X: case SV_CX: m[1] = m[2] = make_double2(1, 0); break;
    case SV_Y: case SV_CY: m[1] = make_double2(0, -1); m[2] = make_double2(0, 1); break;
    case SV_Z: case SV_CZ: m[0] = make_double2(1, 0); m[3] = make_double2(-1, 0); break;
    case SV_S: m[0] = make_double2(1, 0); m[3] = make_double2(0, 1); break;
    case SV_SDG: m[0] = make_double2(1, 0); m[3] = make_double2(0, -1); break;
    case SV_T: m[0] = make_double2(1, 0); m[3] = make_double2(h, h); break;
    case SV_TDG: m[0] = make_double2(1, 0); m[3] = make_double2(h, -h); break;
    case SV_SX:
      m[0] = m[3] = make_double2(0.5, 0.5);
      m[1] = m[2] = make_double2(0.5, -0.5);
      break;
    case SV_RX: case SV_CRX:
      sincos(0.5 * t[0], &s, &c);
      m[0] = m[3] = make_double2(c, 0);
      m[1] = m[2] = make_double2(0, -s);
      break;
    case SV_RY: case SV_CRY:
      sincos(0.5 * t[0], &s, &c);
      m[0] = m[3] = make_double2(c, 0);
      m[1] = make_double2(-s, 0);
      m[2] = make_double2(s, 0);
      break;
    case SV_RZ: case SV_CRZ:
      sincos(0.5 * t[0], &s, &c);
      m[0] = make_double2(c, -s);
      m[3] = make_double2(c, s);
      break;
    case SV_P: case SV_CP:
      sincos(t[0], &s, &c);
      m[0] = make_double2(1, 0);
      m[3] = make_double2(c, s);
      break;
    case SV_U: case SV_CU:
      sincos(0.5 * t[0], &s, &c);
      sincos(t[1], &sp, &cp);
      sincos(t[2], &sl, &cl);
      m[0] = make_double2(c, 0);
      m[1] = make_double2(-cl * s, -sl * s);
      m[2] = make_double2(cp * s, sp * s);
      m[3] = make_double2((cp * cl - sp * sl) * c, (sp * cl + cp * sl) * c);
      break;
    default: m[0] = m[3] = make_double2(1, 0); break;
  }
}


// d/d(angle[slot]) of the target matrix of a parametrised standard gate
// (same conventions as std_gate_2x2); zero for gates without that angle.
static __device__ void std_gate_deriv(int gate, const double* t, int slot, double2* d) {
  double c, s, sp, cp, sl, cl;
  for (int k = 0; k < 4; ++k) d[k] = make_double2(0, 0);
  switch (gate) {
    case SV_RX: case SV_CRX:
      if (slot) break;
      sincos(0.5 * t[0], &s, &c);
      d[0] = d[3] = make_double2(-0.5 * s, 0);
      d[1] = d[2] = make_double2(0, -0.5 * c);
      break;
    case SV_RY: case SV_CRY:
      if (slot) break;
      sincos(0.5 * t[0], &s, &c);
      d[0] = d[3] = make_double2(-0.5 * s, 0);
      d[1] = make_double2(-0.5 * c, 0);
      d[2] = make_double2(0.5 * c, 0);
      break;
    case SV_RZ: case SV_CRZ:
      if (slot) break;
      sincos(0.5 * t[0], &s, &c);
      d[0] = make_double2(-0.5 * s, -0.5 * c);  // (-i/2) e^{-i a/2}
      d[3] = make_double2(-0.5 * s, 0.5 * c);   // (i/2) e^{i a/2}
      break;
    case SV_P: case SV_CP:
      if (slot) break;
      sincos(t[0], &s, &c);
      d[3] = make_double2(-s, c);  // i e^{i a}
      break;
    case SV_U: case SV_CU:
      sincos(0.5 * t[0], &s, &c);
      sincos(t[1], &sp, &cp);
      sincos(t[2], &sl, &cl);
      if (slot == 0) {
        d[0] = make_double2(-0.5 * s, 0);
        d[1] = make_double2(-0.5 * cl * c, -0.5 * sl * c);
        d[2] = make_double2(0.5 * cp * c, 0.5 * sp * c);
        d[3] = make_double2(-0.5 * (cp * cl - sp * sl) * s, -0.5 * (sp * cl + cp * sl) * s);
      } else if (slot == 1) {
        d[2] = make_double2(-sp * s, cp * s);  // i e^{i phi} s
        d[3] = make_double2(-(sp * cl + cp * sl) * c, (cp * cl - sp * sl) * c);
      } else {
        d[1] = make_double2(sl * s, -cl * s);  // -i e^{i lambda} s
        d[3] = make_double2(-(sp * cl + cp * sl) * c, (cp * cl - sp * sl) * c);
      }
      break;
    default: break;
  }
}

static __device__ __forceinline__ uint64_t pdep64(uint64_t v, uint64_t mask) {
  uint64_t out = 0;
  for (uint64_t bb = 1; mask; bb <<= 1) {
    const uint64_t low = mask & (~mask + 1);
    if (v & bb) out |= low;
    mask &= mask - 1;
  }
  return out;
}

// x + y in the spread domain of mask (x and y hold bits of mask only): the
// gaps are filled with ones so that carries cross them.  For x = pdep(a, mask)
// and y = pdep(b, mask) the result is pdep(a + b, mask), modulo 2^popc(mask).
static __device__ __forceinline__ uint64_t spread_add(uint64_t x, uint64_t y, uint64_t mask) {
  return ((x | ~mask) + y) & mask;
}

static __device__ __forceinline__ uint64_t pext64(uint64_t v, uint64_t mask) {
  uint64_t out = 0, bb = 1;
  for (; mask; bb <<= 1) {
    const uint64_t low = mask & (~mask + 1);
    if (v & low) out |= bb;
    mask &= mask - 1;
  }
  return out;
}

// 16 per-lane values -> lane holds the warp sum of slot(lane); 16 shuffles.
template <typename A>
__device__ __forceinline__ A warp_transpose_reduce16(A (&v)[16], int lane) {
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int o = 16 >> st, h = 8 >> st;
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const A send = up ? v[i] : v[i + h];
      const A keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}
// Double-float values: an unevaluated sum hi + lo of two FP32 numbers (about
// 44 significant bits).  two_sum is Knuth's error-free addition.  The complex64
// measurement table forms each |amp|^2 in FP32 (one FMA after a product:
// relative error <= 2^-23) and sums them in double-float from there on -- the
// warp tree and the run over tiles -- so the sums carry no error of their own
// at FP32 scale, on the FP32 pipes (GB300's FP64 rate is 1/64 of FP32's).
struct DF {
  float hi, lo;
};
static __device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return DF{s, e};
}
static __device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = two_sum(a.hi, b.hi);
  const float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s.hi, lo);  // renormalise (|s.hi| >= |lo|)
  return DF{h, __fsub_rn(lo, __fsub_rn(h, s.hi))};
}
// warp_transpose_reduce16 on double-float values (same lane -> slot map)
__device__ __forceinline__ DF warp_transpose_reduce16_df(DF (&v)[16], int lane) {
#pragma unroll
  for (int st = 0; st < 4; ++st) {
    const int o = 16 >> st, h = 8 >> st;
    const bool up = lane & o;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const DF send = up ? v[i] : v[i + h];
      const DF keep = up ? v[i + h] : v[i];
      const DF got{__shfl_xor_sync(0xffffffffu, send.hi, o), __shfl_xor_sync(0xffffffffu, send.lo, o)};
      v[i] = df_add(keep, got);
    }
  }
  const DF got{__shfl_xor_sync(0xffffffffu, v[0].hi, 1), __shfl_xor_sync(0xffffffffu, v[0].lo, 1)};
  return df_add(v[0], got);
}

static __device__ __forceinline__ int transpose_slot(int lane) {
  return (((lane >> 4) & 1) << 3) | (((lane >> 3) & 1) << 2) | (((lane >> 2) & 1) << 1) | ((lane >> 1) & 1);
}

// ---- scalar phase (one thread of the last CTA): draws, classical register, predicates
static __device__ __noinline__ void scalar_phase(const PassArgs& A, const DPass& sp, const double* ctab, bool do_store,
                                          uint64_t pm, uint64_t pv, uint64_t px, double ps) {
  Ctrl* W = A.ctrl;
  uint64_t creg = W->creg, mc = W->m;
  uint64_t npm = do_store ? 0 : pm, npv = do_store ? 0 : pv, npx = do_store ? 0 : px;
  double nps = do_store ? 1.0 : ps;
  double tab[16];
  for (int e = 0; e < 16; ++e) tab[e] = ctab[e];
  const int tsize = 1 << sp.gk;
  bool drew = false;
  for (uint32_t c = 0; c < sp.nc; ++c) {
    const DScalar s = A.scalars[sp.c0 + c];
    if (s.kind == S_COND) {
      const bool par = s.flag < 0 || A.flags[s.flag];
      const bool pred = (creg & s.mask) == s.value;
      A.flags[s.f_then] = (par && pred) ? 1 : 0;
      if (s.f_else >= 0) A.flags[s.f_else] = (par && !pred) ? 1 : 0;
      continue;
    }
    if (!(s.flag < 0 || A.flags[s.flag])) continue;
    double p0 = 0, p1 = 0;
    for (int e = 0; e < tsize; ++e) {
      if ((e >> s.tbit) & 1) p1 += tab[e];
      else p0 += tab[e];
    }
    const double u = draw_uniform(W->seed, W->stream, W->shot, mc);
    int o = 0;
    if (!(p0 + p1 > 0)) W->status = SV_ERR_NUMERIC;
    else o = (u >= p0 / (p0 + p1)) ? 1 : 0;
    if (W->n_trace < MAX_TRACE) {
      DTrace& tr = A.trace[W->n_trace];
      tr.qubit = int(s.qubit);
      tr.is_reset = s.kind == S_RESET;
      tr.outcome = o;
      tr.pad = 0;
      tr.p0 = p0;
      tr.p1 = p1;
      tr.u = u;
      W->n_trace = W->n_trace + 1;
    }
    ++mc;
    const int bt = 1 << s.tbit;
    for (int e = 0; e < tsize; ++e)
      if (((e >> s.tbit) & 1) != o) tab[e] = 0;
    if (s.kind == S_RESET && o)
      for (int e = 0; e < tsize; ++e)
        if (e & bt) {
          tab[e ^ bt] = tab[e];
          tab[e] = 0;
        }
    if (s.kind == S_MEASURE) creg = (creg & ~(1ull << s.cbit)) | (uint64_t(o) << s.cbit);
    const uint64_t qb = 1ull << s.qubit;
    const uint64_t xq = (npx >> s.qubit) & 1ull;
    npm |= qb;
    npv = (npv & ~qb) | ((uint64_t(o) ^ xq) << s.qubit);
    if (s.kind == S_RESET && o) npx ^= qb;
    drew = true;
  }
  if (drew) {
    double mass = 0;
    for (int e = 0; e < tsize; ++e) mass += tab[e];
    if (mass > 0) nps *= 1.0 / sqrt(mass);
    else W->status = SV_ERR_NUMERIC;
  }
  if (A.work && mc > W->m) {  // draws executed, and their amplitude updates (2^n each)
    atomicAdd(A.work + 3, (unsigned long long)(mc - W->m));
    atomicAdd(A.work + 5, (unsigned long long)(mc - W->m) << A.n);
  }
  W->creg = creg;
  W->m = mc;
  W->pm = npm;
  W->pv = npv;
  W->px = npx;
  W->ps = nps;
  W->ticket = 0;
  __threadfence();
}

// register offsets of a stage: off[j] = XOR of R[r] over the set bits r of j
static __device__ __forceinline__ void reg_offsets(const uint16_t* R, uint32_t (&off)[16]) {
  off[0] = 0;
#pragma unroll
  for (int j = 1; j < 16; ++j) off[j] = off[j & (j - 1)] ^ R[__ffs(j) - 1];
}

template <int GB>
__device__ __forceinline__ uint32_t group_base(const uint16_t* E, uint32_t g) {
  uint32_t b = 0;
#pragma unroll
  for (int k = 0; k < GB; ++k)
    if ((g >> k) & 1u) b ^= E[k];
  return b;
}

// The tiles of one unit of a pipelined sweep with a pending projector (bases
// are spread over the non-tile qubits): dst is swept and stored, reading its
// amplitudes from src; with outer flips xo the partner tile dst ^ xo becomes
// zero.  act = false: the projector zeroes dst as well (nothing is copied or
// swept).
struct Unit {
  uint64_t dst, src;
  bool act;
};
static __device__ __forceinline__ Unit unit_tiles(uint64_t ub, uint64_t xo, uint64_t px, uint64_t pm, uint64_t pv,
                                                  uint64_t omask, bool ident) {
  Unit t;
  const uint64_t pmo = pm & omask, pvo = pv & omask;
  const bool ca = ident || (((ub ^ px) & pmo) == pvo);
  if (!xo) {
    t.dst = t.src = ub;
    t.act = ca;
    return t;
  }
  const uint64_t b = ub ^ xo;
  const bool cb = ((b ^ px) & pmo) == pvo;
  t.act = ca || cb;
  t.dst = ca ? ub : (cb ? b : ub);
  t.src = t.dst ^ xo;
  return t;
}

// The measurement table is accumulated from the tile before the pass's scalar
// factor f is multiplied in: |amp|^2 sums scale by |f|^2.
static __device__ __forceinline__ void scale_table(double* ctab, double2 f) {
  const double m = f.x * f.x + f.y * f.y;
  if (m != 1.0)
    for (int i = 0; i < 16; ++i) ctab[i] *= m;
}

// Shared state of one pass (static shared memory of the kernel that runs it);
// the tensor-core part exists only in the variant that may use it.
template <bool TC> struct TcPart {};
template <> struct TcPart<true> {
  TcShared tc;  // tensor-core path of dense gates
};

template <typename T, bool TC = false>
struct PassShared : TcPart<TC> {
  DPass sp;
  uint32_t sgk[MAX_PASS_GATES];  // key | active << 8 | matrix offset << 16
  __align__(16) typename CxT<T>::V smat[MAX_PASS_MAT];
  uint64_t schunk[512];          // global offset of each gathered chunk of the tile
  double ctab[16];               // measurement-group table of this CTA
  double wsum[PASS_THREADS / 32][16];
  double tile16[16];
  double2 pfac;                  // product of the factors of the pass's active factored gates
  int s_last;
};
template <typename T, bool TC>
__device__ __forceinline__ TcShared* tc_shared(PassShared<T, TC>& sh) {
  if constexpr (TC) return &sh.tc;
  else return nullptr;
}

// The pending projector in tile-local bits, for kernels whose first stage
// applies it to the amplitudes it loads (instead of a separate in-place pass
// over the copied tile).  The copy has already applied the flip's bits other
// than tile bit 0; swap0: the flip includes tile bit 0 (complex64 amplitude
// pairs swap in registers).
struct ProjFold {
  bool on;
  uint32_t pm, pv, px;  // tile-local: bit b <-> qubit tq[b]
  bool swap0;
  double ps;
};

// One pass over the state.  GRID mode (CTA = false): the tiles are shared by
// all CTAs of the launch and the last CTA to finish reduces the group table
// and runs the scalar phase.  CTA mode (CTA = true): the calling CTA owns the
// whole trajectory, walks every tile itself and runs the scalar phase after a
// block barrier; used by the persistent batched kernel.
// Data-driven register stages: every stage reads its register / group bit
// addresses and gate records from the plan at run time.
struct GenericStages {
  static constexpr bool kDirect = false;    // the tile is always stored by the pass's store phase
  static constexpr bool kFoldProj = false;  // a pending projector is applied to the copied tile
  template <typename T, int M, bool TC>
  static __device__ __forceinline__ void run(const PassArgs& A, const DPass& sp, const uint32_t* sgk,
                                             const typename CxT<T>::V* smat, typename CxT<T>::V* tb, TcCtx& tc,
                                             const uint64_t, const typename CxT<T>::V, const bool,
                                             const ProjFold&) {
    using V = typename CxT<T>::V;
    constexpr int GB = M - REG_BITS;
    constexpr int NGRP = 1 << GB;
    const int tid = threadIdx.x;
    for (uint32_t si = 0; si < sp.ns; ++si) {
      const DStage st = A.stages[sp.s0 + si];
      uint32_t off[16];
      reg_offsets(st.R, off);
      // complex64 with register bit 0 on tile bit 0: amplitude pairs share a
      // 16-byte granule (the swizzle never touches bit 0), one access per pair
      const bool pairs = sizeof(T) == 4 && st.R[0] == 1;
      for (int grp = tid; grp < NGRP; grp += PASS_THREADS) {
        const uint32_t b = group_base<GB>(st.E, uint32_t(grp));
        V a[16];
        if (pairs) {
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            const typename CxT<T>::V4 q = *reinterpret_cast<const typename CxT<T>::V4*>(tb + (b ^ off[j]));
            a[j] = pair_lo(q);
            a[j + 1] = pair_hi(q);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) a[j] = tb[b ^ off[j]];
        }
        for (int g = st.g0; g < st.g0 + st.ng; ++g) {
          const uint32_t w = sgk[g];
          if (!(w & SGK_ON)) continue;
          if ((w & SGK_KEY) == OP_D16 * 16u) d16_apply<T, M, TC>(a, smat + (w >> 16), tb, tc);
          else apply_gate(a, w & SGK_KEY, smat + (w >> 16));
        }
        if (pairs) {
#pragma unroll
          for (int j = 0; j < 16; j += 2)
            *reinterpret_cast<typename CxT<T>::V4*>(tb + (b ^ off[j])) = make_pair4(a[j], a[j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) tb[b ^ off[j]] = a[j];
        }
      }
      // a direct pass relaxes the barrier after its last stage for kernels that
      // store from registers; this one stores from shared memory
      if (st.bar || (sp.direct && si + 1 == sp.ns)) __syncthreads();
      else __syncwarp();
    }
  }
};

// TC: the kernel variant that may send dense four-qubit gates to the tensor
// cores (launched only for passes that hold one: the mere presence of tcgen05
// instructions in a kernel measured ~20% slower sweeps on GB300).
// PROJ: the variant for passes that may start with a measurement projector
// pending (it keeps the copy pipeline for them; see the tile loop).
template <typename T, int M, bool CTA, typename Stages = GenericStages, bool TC = false, bool PROJ = false>
__device__ __forceinline__ void pass_body(const PassArgs& A, const int pi, PassShared<T, TC>& sh, void* smem_tiles) {
  using V = typename CxT<T>::V;
  using Acc = T;  // per-thread |amp|^2 accumulation: FP32 for complex64, FP64 for complex128
  constexpr int GB = M - REG_BITS;  // group-index bits of a stage
  constexpr int NGRP = 1 << GB;     // 16-amplitude groups per tile
  // tile buffers of the copy pipeline (NBUF - 1 tiles in flight): two when they
  // fit in 128 KiB, else one.  A third buffer measured no faster.
  constexpr size_t TILE_BYTES = (size_t(1) << M) * sizeof(V);
  constexpr int NBUF = 2 * TILE_BYTES <= size_t(128) * 1024 ? 2 : 1;
  constexpr bool DB = NBUF > 1;
  V* tile = reinterpret_cast<V*>(smem_tiles);
  DPass& sp = sh.sp;
  uint32_t* sgk = sh.sgk;
  V* smat = sh.smat;
  uint64_t* schunk = sh.schunk;
  double* ctab = sh.ctab;
  double* tile16 = sh.tile16;
  const uint64_t ustart = CTA ? 0ull : uint64_t(blockIdx.x);
  const uint64_t ustep = CTA ? 1ull : uint64_t(gridDim.x);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) sp = A.passes[pi];
  if (tid < 16) ctab[tid] = 0.0;
  __syncthreads();
  const int L = sp.L, n = A.n;

  int act_any = 0;
  for (int g = tid; g < int(sp.ng); g += PASS_THREADS) {
    const DGate d = A.gates[sp.g0 + g];
    const uint32_t on = d.flag < 0 ? 1u : (A.flags[d.flag] ? 1u : 0u);
    sgk[g] = uint32_t(d.key) | (on << SGK_ON_BIT) | (d.mat << 16);
    act_any |= int(on);
  }
  const bool any_gate = __syncthreads_or(act_any) != 0;
  if (A.work && (CTA || blockIdx.x == 0) && tid == 0 && any_gate) {  // gate records this run executes
    unsigned long long k = 0;
    for (int g = 0; g < int(sp.ng); ++g) k += (sgk[g] & SGK_ON) ? 1ull : 0ull;
    atomicAdd(A.work + 2, k);
    atomicAdd(A.work + 5, k << A.n);
  }
  int need = 0;
  if (sp.gk) {
    if (sp.group_always) need = 1;
    else
      for (int c = tid; c < int(sp.nc); c += PASS_THREADS) {
        const DScalar sc = A.scalars[sp.c0 + c];
        if (sc.kind != S_COND && (sc.flag < 0 || A.flags[sc.flag])) need = 1;
      }
  }
  const bool needed = __syncthreads_or(need) != 0;

  const Ctrl* C = A.ctrl;
  const uint64_t pm = C->pm, pv = C->pv, px = C->px;
  const double ps = C->ps;
  const bool ident = (pm == 0 && px == 0 && ps == 1.0);
  const bool do_store = any_gate || (sp.flush && !ident);
  const bool do_work = do_store || needed;
  const bool need_ticket = sp.nc > 0 || (do_store && !ident);

  TcCtx tc{tc_shared(sh), nullptr, 0u, 0u, false, true, 0u};
  if (do_work) {
    if (any_gate)
      for (int i = tid; i < int(sp.nmat); i += PASS_THREADS) smat[i] = reinterpret_cast<const V*>(A.mats)[sp.mat0 + i];
    const int hb = M - L;
    for (int c = tid; c < (1 << hb); c += PASS_THREADS) {
      uint64_t o = 0;
      for (int k = 0; k < hb; ++k)
        if ((c >> k) & 1) o |= 1ull << sp.tq[L + k];
      schunk[c] = o;
    }
    // Dense four-qubit gates on the tensor cores: this CTA takes 256 columns of
    // tensor memory (the A rows and two 128 x 32 FP32 accumulators, dev_tc.cuh)
    // and an mbarrier for the MMA completions, and gives both back after the
    // tile loop; the B operand of each dense gate is built once, here.
    if constexpr (TC && sizeof(T) == 4 && M == 12 && !CTA) tc.on = A.dense_tc != 0 && sp.dense != 0 && any_gate;
    if (tc.on) {
      if (warp == 0) {
        tmem_alloc(&tc.s->tmem, TC_TMEM_COLS);
        tmem_relinquish();
      }
      if (tid == 0) {
        mbar_init(&tc.s->bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      }
      tc_fence_before();
    }
    __syncthreads();
    // the scalar factors of the factored rotations (OP_RXF / OP_RYF / OP_DZ) that
    // are active in this pass, multiplied into the tile when it is stored
    if (tid == 0) {
      double fr = 1.0, fi = 0.0;
      if (any_gate)
        for (int g = 0; g < int(sp.ng); ++g) {
          const uint32_t w = sgk[g], op = (w & SGK_KEY) >> 4;
          if (!(w & SGK_ON) || (op != OP_RXF && op != OP_RYF && op != OP_DZ)) continue;
          const V f = smat[(w >> 16) + 1];
          const double r = fr * double(f.x) - fi * double(f.y);
          fi = fr * double(f.y) + fi * double(f.x);
          fr = r;
        }
      sh.pfac = make_double2(fr, fi);
    }
    __syncthreads();
    const double2 pf = sh.pfac;
    const bool fscale = !(pf.x == 1.0 && pf.y == 0.0);
    const V fT = mkc(T(pf.x), T(pf.y));
    if (tc.on) {
      tc_fence_after();
      tc.tmem = tc.s->tmem;
      tc.smat = smat;
      // B of the pass's dense gates, once: slot k <- the k-th dense record
      int k = 0;
      for (int g = 0; g < int(sp.ng) && k < TC_SLOTS; ++g)
        if ((sgk[g] & SGK_KEY) == OP_D16 * 16u) {
          const uint32_t mo = sgk[g] >> 16;
          d16_build_b(smat + mo, *tc.s, k);
          if (tid == 0) tc.s->slot_mat[k] = mo;
          ++k;
        }
      if (tid == 0)
        for (int j = k; j < TC_SLOTS; ++j) tc.s->slot_mat[j] = ~0u;  // unused slots match no gate
      fence_async_smem();
      __syncthreads();
    }

    uint64_t tmask = 0;
    for (int j = 0; j < M; ++j) tmask |= 1ull << sp.tq[j];
    const uint64_t full = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    const uint64_t omask = full & ~tmask;
    const uint64_t ntiles = 1ull << (n - M);
    const uint64_t xo = px & omask;  // part of the pending X that moves whole tiles
    const bool pair = xo != 0;
    const uint64_t xt = pair ? pext64(xo, omask) : 0;
    const int hbit = pair ? __ffsll((long long)xt) - 1 : 0;
    const uint64_t nunits = pair ? (ntiles >> 1) : ntiles;
    const T sc = T(ps);
    const uint32_t kmask = (1u << sp.kin) - 1;

    // tile-independent parts of this thread's load/store addresses
    constexpr int VB = sizeof(T) == 4 ? 9 : 8;   // log2 amplitudes covered by one sweep of 256 threads
    constexpr int NVT = 1 << (M - VB);           // 16-byte vectors per thread per tile
    const int vl = sizeof(T) == 4 ? L - 1 : L;   // log2 vectors per contiguous chunk
    const uint32_t wv = uint32_t(tid) & ((1u << vl) - 1u);
    const uint32_t woff = sizeof(T) == 4 ? (wv << 1) : wv;  // amplitude offset inside the chunk
    const uint32_t c0 = uint32_t(tid) >> vl;
    const uint32_t q0 = swz<T>((c0 << L) | woff);

    // Tiles stream in by 16-byte asynchronous copies, the next tile in flight
    // while the current one is processed (two shared-memory buffers), when no
    // measurement projector is pending.  Otherwise the plain variant loads the
    // tile synchronously with the projector applied on the way in, while the
    // PROJ variant (launched for passes that may follow a measurement) keeps
    // the copy pipeline: the copy reads the source of the projector's flip
    // (a'[i] = ps * a[i ^ px] if ((i ^ px) & pm) == pv), and each thread then
    // zeroes, scales and (complex64, flip of bit 0) swaps the vectors it
    // copied.  Flips of qubits outside the tile (xo) pair tile t with t ^ xo in
    // one unit: the tile that satisfies the projector is copied from its
    // partner, and the partner becomes zero.  Tiles that the projector zeroes
    // are neither copied nor swept.
    const bool gen = PROJ && A.gen_init != 0;  // (no projector is pending at the first pass)
    // specialised kernels fold the projector into the first stage when it runs
    // (gates active, a first stage exists; a flip of tile bit 0 needs pairs in it)
    ProjFold pjf{false, 0u, 0u, 0u, false, ps};
    if constexpr (PROJ && Stages::kFoldProj) {
      if (!ident && !gen && any_gate && sp.ns > 0) {
        for (int b = 0; b < M; ++b) {
          pjf.pm |= uint32_t((pm >> sp.tq[b]) & 1) << b;
          pjf.pv |= uint32_t((pv >> sp.tq[b]) & 1) << b;
          pjf.px |= uint32_t((px >> sp.tq[b]) & 1) << b;
        }
        pjf.swap0 = sizeof(T) == 4 && (pjf.px & 1u);
        pjf.on = !pjf.swap0 || A.stages[sp.s0].R[0] == 1;
      }
    }
    const bool pipe = PROJ ? (DB && ((xo & ~pm) == 0)) : (DB && ident);
    pjf.on = pjf.on && pipe;  // the synchronous load applies the projector itself
    const bool upair = PROJ && pipe && pair;  // units are tile pairs
    const uint64_t umask = upair ? (omask & ~(xo & (~xo + 1))) : omask;  // unit index bits
    const uint64_t pxi = PROJ ? (px & tmask & (sizeof(T) == 4 ? ~1ull : ~0ull)) : 0;  // inner flip, granule-aligned
    int cur = 0;
    unsigned long long n_rd = 0, n_wr = 0;
    // Unit bases advance by masked addition instead of a bit-by-bit deposit per unit.
    const uint64_t sstep = pdep64(ustep, umask);
    const uint64_t sahead = pdep64(uint64_t(NBUF - 1) * ustep, umask);
    uint64_t bcur = pdep64(ustart, umask);
    auto buffer = [&](int k) { return tile + size_t(k) * (size_t(1) << M); };
    if (pipe) {  // prologue: the first NBUF - 1 units of this CTA, one commit group each
      for (int k = 0; k < NBUF - 1; ++k) {
        const uint64_t uk = ustart + uint64_t(k) * ustep;
        if (uk < nunits) {
          uint64_t src = pdep64(uk, umask);
          bool go = true;
          if constexpr (PROJ) {
            const Unit Uk = unit_tiles(src, xo, px, pm, pv, omask, ident);
            src = Uk.src;
            go = Uk.act && !gen;
          }
          n_rd += go ? 1ull : 0ull;
          if (go) {
            V* dst = buffer(k);
#pragma unroll
            for (int v = 0; v < NVT; ++v) {
              const uint32_t ch = c0 + (uint32_t(v) << (VB - L));
              cp_async16(dst + (q0 ^ swz<T>(uint32_t(v) << VB)),
                         reinterpret_cast<const V*>(A.state) + ((src | schunk[ch] | woff) ^ pxi));
            }
          }
        }
        cp_async_commit();
      }
    }

    double tacc = 0.0;  // this lane's measurement-table slot over the tiles (all group qubits in the tile)
    DF tdf{0.f, 0.f};   // the same for complex64, in double-float
    // tiles this CTA read from / wrote to the state (thread 0 counts; grid passes report them)
    for (uint64_t u = ustart; u < nunits; u += ustep) {
      uint64_t tl[2] = {u, 0};
      int cnt = 1;
      if (pair && !upair) {
        const uint64_t lo = u & ((1ull << hbit) - 1);
        const uint64_t t0 = ((u >> hbit) << (hbit + 1)) | lo;
        const uint64_t t1 = t0 ^ xt;
        const uint64_t b0 = pdep64(t0, omask);
        const bool t0_reads = (((b0 ^ px) & pm & omask) == (pv & omask));
        tl[0] = t0_reads ? t0 : t1;  // the tile that reads its partner goes first
        tl[1] = t0_reads ? t1 : t0;
        cnt = 2;
      }
      for (int k2 = 0; k2 < cnt; ++k2) {
        V* tb;
        uint64_t base;
        bool act = true;  // false: the projector zeroes this tile (PROJ variant)
        if (pipe) {
          base = bcur;
          tb = buffer(cur);
          cp_async_wait<NBUF - 2>();  // this unit's group; the NBUF - 2 newer ones may still fly
          if constexpr (PROJ) {
            if (gen) {  // the first pass: |0...0> in the tile holding index 0, zeros elsewhere
              act = base == 0;
#pragma unroll
              for (int k = 0; k < NVT; ++k) {
                const uint32_t p = q0 ^ swz<T>(uint32_t(k) << VB);
                const bool one = act && tid == 0 && k == 0;  // local index 0: thread 0's first vector
                if constexpr (sizeof(T) == 4)
                  *reinterpret_cast<float4*>(tb + p) = make_float4(one ? 1.f : 0.f, 0.f, 0.f, 0.f);
                else
                  tb[p] = make_double2(one ? 1.0 : 0.0, 0.0);
              }
            } else if (!ident) {  // the projector, on the vectors this thread copied
              const Unit U = unit_tiles(bcur, xo, px, pm, pv, omask, false);
              base = U.dst;
              act = U.act;
#pragma unroll
              for (int k = 0; k < NVT && !(pjf.on && act); ++k) {  // (a folding first stage applies it)
                const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
                const uint64_t gi = base | schunk[ch] | woff;
                const uint32_t p = q0 ^ swz<T>(uint32_t(k) << VB);
                const uint64_t s0 = gi ^ px;
                if constexpr (sizeof(T) == 4) {
                  float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                  if (act) {
                    const float4 r = *reinterpret_cast<const float4*>(tb + p);
                    const bool ok0 = (s0 & pm) == pv, ok1 = ((s0 ^ 1ull) & pm) == pv;
                    const float2 e0 = make_float2(r.x, r.y), e1 = make_float2(r.z, r.w);
                    const float2 x0 = (px & 1) ? e1 : e0, x1 = (px & 1) ? e0 : e1;
                    q = make_float4(ok0 ? x0.x * sc : 0.f, ok0 ? x0.y * sc : 0.f, ok1 ? x1.x * sc : 0.f,
                                    ok1 ? x1.y * sc : 0.f);
                  }
                  *reinterpret_cast<float4*>(tb + p) = q;
                } else {
                  V x = make_double2(0, 0);
                  if (act && (s0 & pm) == pv) {
                    x = tb[p];
                    x.x *= sc;
                    x.y *= sc;
                  }
                  tb[p] = x;
                }
              }
            }
          }
        } else {
          tb = tile;
          base = pair ? pdep64(tl[k2], omask) : bcur;
          const bool zero_tile = !ident && (((base ^ px) & pm & omask) != (pv & omask));
          n_rd += (gen || zero_tile) ? 0ull : 1ull;
          // a'[i] = ps * a[i ^ px] if ((i ^ px) & pm) == pv, else 0
#pragma unroll
          for (int k = 0; k < NVT; ++k) {
            const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
            const uint64_t gi = base | schunk[ch] | woff;
            const uint32_t p = q0 ^ swz<T>(uint32_t(k) << VB);
            if constexpr (sizeof(T) == 4) {
              const float4* gs = reinterpret_cast<const float4*>(A.state);
              float2 x0, x1;
              if (gen) {  // the first pass generates |0...0>
                x0 = make_float2(gi == 0 ? 1.f : 0.f, 0.f);
                x1 = make_float2(0.f, 0.f);
              } else if (zero_tile) {
                x0 = x1 = make_float2(0.f, 0.f);
              } else if (ident) {
                const float4 q = __ldcg(gs + (gi >> 1));
                x0 = make_float2(q.x, q.y);
                x1 = make_float2(q.z, q.w);
              } else {
                const uint64_t s0 = gi ^ px;
                const bool ok0 = (s0 & pm) == pv, ok1 = ((s0 ^ 1ull) & pm) == pv;
                float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ok0 || ok1) q = __ldcg(gs + (s0 >> 1));
                const float2 e0 = make_float2(q.x, q.y), e1 = make_float2(q.z, q.w);
                x0 = (s0 & 1) ? e1 : e0;
                x1 = (s0 & 1) ? e0 : e1;
                x0 = ok0 ? make_float2(x0.x * sc, x0.y * sc) : make_float2(0.f, 0.f);
                x1 = ok1 ? make_float2(x1.x * sc, x1.y * sc) : make_float2(0.f, 0.f);
              }
              *reinterpret_cast<float4*>(tile + p) = make_float4(x0.x, x0.y, x1.x, x1.y);
            } else {
              const double2* gs = reinterpret_cast<const double2*>(A.state);
              double2 x;
              if (gen) {
                x = make_double2(gi == 0 ? 1.0 : 0.0, 0.0);
              } else if (zero_tile) {
                x = make_double2(0, 0);
              } else if (ident) {
                x = __ldcg(gs + gi);
              } else {
                const uint64_t s0 = gi ^ px;
                if ((s0 & pm) == pv) {
                  x = __ldcg(gs + s0);
                  x.x *= sc;
                  x.y *= sc;
                } else {
                  x = make_double2(0, 0);
                }
              }
              tile[p] = x;
            }
          }
        }
        // This tile has landed, and every thread is done with the previous
        // tile, so its buffer can be refilled.  When the first stage keeps the
        // copies' warp bits, each warp reads only what its own lanes copied and
        // refills only what its own lanes stored: a warp barrier suffices.
        if (pipe && any_gate && act && !sp.bar_in) __syncwarp();
        else __syncthreads();
        if (pipe) {  // refill the buffer processed one iteration ago with the unit NBUF - 1 ahead
          const uint64_t un = u + uint64_t(NBUF - 1) * ustep;
          if (un < nunits) {
            uint64_t src = spread_add(bcur, sahead, umask);
            bool go = true;
            if constexpr (PROJ) {
              if (gen) {
                go = false;
              } else if (!ident) {
                const Unit Un = unit_tiles(src, xo, px, pm, pv, omask, false);
                src = Un.src;
                go = Un.act;
              }
            }
            n_rd += go ? 1ull : 0ull;
            if (go) {
              V* nb = buffer((cur + NBUF - 1) % NBUF);
#pragma unroll
              for (int k = 0; k < NVT; ++k) {
                const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
                cp_async16(nb + (q0 ^ swz<T>(uint32_t(k) << VB)),
                           reinterpret_cast<const V*>(A.state) + ((src | schunk[ch] | woff) ^ pxi));
              }
            }
          }
          cp_async_commit();
        }

        // ---- gate stages
        if (any_gate && act) Stages::template run<T, M, TC && !CTA>(A, sp, sgk, smat, tb, tc, base, fT, fscale, pjf);
        // the last stage stored the tile itself (specialised kernels, direct passes)
        const bool stored = Stages::kDirect && sp.direct && any_gate && act;

        // ---- measurement-group table (a zeroed tile adds nothing)
        if (needed && act) {
          uint32_t off[16];
          reg_offsets(sp.red_R, off);
          double r;
          if constexpr (sizeof(T) == 4) {  // complex64: FP32 |amp|^2, double-float sums
            DF acc[16];
            if constexpr (NGRP == PASS_THREADS) {  // one group per thread
              const uint32_t b = group_base<GB>(sp.red_E, uint32_t(tid));
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const V x = tb[b ^ off[j]];
                acc[j] = DF{__fmaf_rn(x.x, x.x, __fmul_rn(x.y, x.y)), 0.f};
              }
            } else {
#pragma unroll
              for (int j = 0; j < 16; ++j) acc[j] = DF{0.f, 0.f};
              for (int grp = tid; grp < NGRP; grp += PASS_THREADS) {
                const uint32_t b = group_base<GB>(sp.red_E, uint32_t(grp));
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                  const V x = tb[b ^ off[j]];
                  acc[j] = df_add(acc[j], DF{__fmaf_rn(x.x, x.x, __fmul_rn(x.y, x.y)), 0.f});
                }
              }
            }
            const DF d = warp_transpose_reduce16_df(acc, lane);
            if (sp.kin == sp.gk) {  // summed over the tiles in double-float, converted once per pass
              if ((lane & 1) == 0) tdf = df_add(tdf, d);
              r = 0.0;
            } else {
              r = double(d.hi) + double(d.lo);
            }
          } else {  // complex128: FP64 throughout
            Acc acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = Acc(0);
            for (int grp = tid; grp < NGRP; grp += PASS_THREADS) {
              const uint32_t b = group_base<GB>(sp.red_E, uint32_t(grp));
#pragma unroll
              for (int j = 0; j < 16; ++j) {
                const V x = tb[b ^ off[j]];
                acc[j] = fma(Acc(x.x), Acc(x.x), Acc(x.y) * Acc(x.y)) + acc[j];
              }
            }
            r = double(warp_transpose_reduce16(acc, lane));
          }
          if (sp.kin == sp.gk) {
            // every measured qubit is a tile qubit, so a lane's table slot is the
            // same in every tile: lanes accumulate across tiles in FP64
            // (complex64: double-float), in tile order, and the warps are
            // combined once, after the tile loop
            if constexpr (sizeof(T) != 4)
              if ((lane & 1) == 0) tacc += r;
          } else {
            if ((lane & 1) == 0) sh.wsum[warp][transpose_slot(lane)] = r;
            __syncthreads();
            if (tid < 16) {
              double s2 = 0;
              for (int w = 0; w < PASS_THREADS / 32; ++w) s2 += sh.wsum[w][tid];
              tile16[tid] = s2;
            }
            __syncthreads();
            if (tid < (1 << sp.kin)) {
              uint32_t ob = 0;
              for (int k = 0; k < sp.gk - sp.kin; ++k) ob |= uint32_t((base >> sp.outer_gq[k]) & 1) << k;
              double s2 = 0;
              for (int j = 0; j < 16; ++j)
                if ((uint32_t(j) & kmask) == uint32_t(tid)) s2 += tile16[j];
              ctab[tid | (ob << sp.kin)] += s2;
            }
          }
        }

        // ---- store
        if (do_store) {
          n_wr += upair ? 2ull : 1ull;
#pragma unroll
          for (int k = 0; k < NVT && !stored; ++k) {
            const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
            const uint64_t gi = base | schunk[ch] | woff;
            const uint32_t p = q0 ^ swz<T>(uint32_t(k) << VB);
            if constexpr (sizeof(T) == 4) {
              float4 q = *reinterpret_cast<const float4*>(tb + p);
              if (fscale) {
                const float2 a0 = cmul(fT, make_float2(q.x, q.y)), a1 = cmul(fT, make_float2(q.z, q.w));
                q = make_float4(a0.x, a0.y, a1.x, a1.y);
              }
              __stcg(reinterpret_cast<float4*>(A.state) + (gi >> 1), q);
            } else {
              const V x = tb[p];
              __stcg(reinterpret_cast<double2*>(A.state) + gi, fscale ? cmul(fT, x) : x);
            }
          }
          if (upair) {  // the unit's partner tile becomes zero (its data was read above)
#pragma unroll
            for (int k = 0; k < NVT; ++k) {
              const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
              const uint64_t gi = (base ^ xo) | schunk[ch] | woff;
              if constexpr (sizeof(T) == 4)
                __stcg(reinterpret_cast<float4*>(A.state) + (gi >> 1), make_float4(0.f, 0.f, 0.f, 0.f));
              else
                __stcg(reinterpret_cast<double2*>(A.state) + gi, make_double2(0, 0));
            }
          }
        }
        if (pipe) {
          // no barrier: the next iteration's barrier orders these reads before
          // this buffer is refilled
          cur = (cur + 1) % NBUF;
        } else {
          __syncthreads();
        }
      }
      bcur = spread_add(bcur, sstep, umask);
    }
    if (pipe) cp_async_wait<0>();
    if (A.work && tid == 0) {
      atomicAdd(A.work + 0, n_rd * (unsigned long long)TILE_BYTES);
      atomicAdd(A.work + 1, n_wr * (unsigned long long)TILE_BYTES);
      if (CTA || blockIdx.x == 0) atomicAdd(A.work + 4, 1ull);
    }
    if (needed && sp.kin == sp.gk) {  // the lanes' table slots, combined over warps in a fixed order
      if constexpr (sizeof(T) == 4) tacc = double(tdf.hi) + double(tdf.lo);
      if ((lane & 1) == 0) sh.wsum[warp][transpose_slot(lane)] = tacc;
      __syncthreads();
      if (tid < 16) {
        double s2 = 0;
        for (int w = 0; w < PASS_THREADS / 32; ++w) s2 += sh.wsum[w][tid];
        tile16[tid] = s2;
      }
      __syncthreads();
      if (tid < (1 << sp.kin)) {
        double s2 = 0;
        for (int j = 0; j < 16; ++j)
          if ((uint32_t(j) & kmask) == uint32_t(tid)) s2 += tile16[j];
        ctab[tid] += s2;
      }
    }
    if (!tc.ok)  // a completion wait ran out, or a dense gate reached this variant with the path off
      atomicCAS(&A.ctrl->status, 0, int32_t(tc.on ? SV_ERR_TIMEOUT : SV_ERR_UNSUPPORTED));
    if (tc.on) {
      tc_drain(tc);
      tc_fence_before();
      __syncthreads();  // every tensor-memory read of this CTA is complete
      if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tc.tmem, TC_TMEM_COLS);
      }
    }
  }

  if constexpr (CTA) {
    if (need_ticket) {
      __syncthreads();
      if (tid == 0) {
        scale_table(ctab, sh.pfac);
        scalar_phase(A, sp, ctab, do_store, pm, pv, px, ps);
      }
    }
    __syncthreads();
  } else {
    if (!need_ticket) return;
    if (needed && tid < 16) A.partials[blockIdx.x * 16 + tid] = ctab[tid];
    __threadfence();
    __syncthreads();
    if (tid == 0) {
      const unsigned t = atomicAdd(&A.ctrl->ticket, 1u);
      sh.s_last = (t == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!sh.s_last) return;
    __threadfence();
    if (needed && tid < 16) {
      double s = 0;
      for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(A.partials + b * 16 + tid);
      ctab[tid] = s;
    }
    __syncthreads();
    if (tid != 0) return;
    scale_table(ctab, sh.pfac);
    scalar_phase(A, sp, ctab, do_store, pm, pv, px, ps);
  }
}

}  // namespace svk
