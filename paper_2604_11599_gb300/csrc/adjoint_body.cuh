// adjoint_body.cuh -- the batched adjoint-gradient kernel body.
//
// For a parameter set theta, E(theta) = <psi|H|psi> with psi = U_N ... U_1 |0>.
// With phi_{k+1} = U_k phi_k and lambda_k = U_{k+1}^dagger ... U_N^dagger H psi,
//   dE/d theta_p = sum over gates k using theta_p of 2 Re <lambda_k| dU_k |phi_k>
//                = 2 Re <lambda_k| (dU_k U_k^dagger) |phi_{k+1}>,
// so one backward sweep that starts from phi = psi, lambda = H psi and, gate
// by gate in reverse, first accumulates Re <lambda| M_k |phi> (M_k = 2 * scale
// * dU_k U_k^dagger) and then applies U_k^dagger to both phi and lambda gives
// every entry (the adjoint differentiation method; Sec. II-D and IV-D of the
// paper motivate runtime parameters for VQE loops).
//
// One CTA owns one parameter set at a time (persistent over a work queue):
// forward passes in CTA mode, lambda = H psi by a grouped Pauli gather (also
// giving E), then backward passes whose tiles hold phi and lambda side by side:
// register bit 3 selects phi / lambda, so the gate templates apply U^dagger to
// both at once and the accumulations pair each phi amplitude with its lambda.
//
// The body is a template over the stage programs of the forward and backward
// passes, so that it is compiled both ahead of time with the generic,
// plan-driven stage programs (kern_adjoint.cu) and at run time with stage
// programs specialised to one lowered program (jit.cpp).
#pragma once
#include "pass_body.cuh"

namespace svk {
using namespace svp;

__device__ __forceinline__ int popc_w(uint32_t v) { return __popc(v); }
__device__ __forceinline__ int popc_w(uint64_t v) { return __popcll(v); }

// lambda = H psi over this CTA's slot (one gather of psi per X group; the
// group's coefficient at j from its terms' Z masks, in mask type W), and
// this thread's part of <psi|lambda>.
template <typename W, typename T, typename AV>
__device__ __forceinline__ double lambda_h(const AdjArgs& J, const typename CxT<T>::V* phi,
                                           typename CxT<T>::V* lam, const AV* hc, const uint64_t* hz,
                                           uint64_t N) {
  using V = typename CxT<T>::V;
  double e = 0;
  for (uint64_t i = threadIdx.x; i < N; i += PASS_THREADS) {
    T ar = 0, ai = 0;
    for (uint32_t g = 0; g < J.ngroups; ++g) {
      const uint64_t j = i ^ J.hx[g];
      const V pj = phi[j];
      const W jw = W(j);
      T wr = 0, wi = 0;
      for (uint32_t t = J.hg0[g]; t < J.hg0[g + 1]; ++t) {
        const bool neg = popc_w(jw & W(hz[t])) & 1;
        const AV c = hc[t];
        wr += neg ? -c.x : c.x;
        wi += neg ? -c.y : c.y;
      }
      ar += wr * pj.x - wi * pj.y;
      ai += wr * pj.y + wi * pj.x;
    }
    lam[i] = mkc(ar, ai);
    const V pi_ = phi[i];
    e += double(pi_.x) * double(ar) + double(pi_.y) * double(ai);
  }
  return e;
}

// Per-warp derivative accumulators of a backward pass (one per accumulation
// slot): complex64 in double-float on the FP32 pipes (a conversion and an FP64
// add per warp per group would bind the backward passes to GB300's FP64
// rate), complex128 in FP64.
template <typename T> struct DotAcc;
template <> struct DotAcc<float> {
  using type = DF;
  static __device__ __forceinline__ void add(DF& a, float r) { a = df_add(a, DF{r, 0.f}); }
  static __device__ __forceinline__ double get(const DF& a) { return double(a.hi) + double(a.lo); }
  static __device__ __forceinline__ DF zero() { return DF{0.f, 0.f}; }
};
template <> struct DotAcc<double> {
  using type = double;
  static __device__ __forceinline__ void add(double& a, double r) { a += r; }
  static __device__ __forceinline__ double get(const double& a) { return a; }
  static __device__ __forceinline__ double zero() { return 0.0; }
};
template <typename T>
using DotRows = typename DotAcc<T>::type[PASS_THREADS / 32][MAX_PASS_DOTS];

// Backward stage program of the generic kernel: for each stage of backward
// pass bp, the groups of 8 phi + 8 lambda amplitudes in registers, the gate
// records (U^dagger on both halves at once: register bit 3 selects phi or
// lambda) and the derivative accumulations Re <lambda| M |phi> read from the
// plan at run time.
struct GenericBwd {
  template <typename T, int M>
  static __device__ __forceinline__ void run(const DStage* stages, uint32_t, const DPass& sp, const PassShared<T>& sh,
                                             const uint16_t (&sdslot)[MAX_PASS_GATES], typename CxT<T>::V* tphi,
                                             typename CxT<T>::V* tlam,
                                             DotRows<T>& wdot) {
    using V = typename CxT<T>::V;
    using Acc = T;
    constexpr int GB = M - ADJ_REG_BITS;
    constexpr int NGRP = 1 << GB;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (uint32_t si = 0; si < sp.ns; ++si) {
      const DStage st = stages[sp.s0 + si];
      uint32_t off[8];
      off[0] = 0;
#pragma unroll
      for (int j = 1; j < 8; ++j) off[j] = off[j & (j - 1)] ^ st.R[__ffs(j) - 1];
      for (int grp = tid; grp < NGRP; grp += PASS_THREADS) {
        const uint32_t b = group_base<GB>(st.E, uint32_t(grp));
        V a[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          a[j] = tphi[b ^ off[j]];
          a[j + 8] = tlam[b ^ off[j]];
        }
        for (int g = st.g0; g < st.g0 + st.ng; ++g) {
          const uint32_t w = sh.sgk[g];
          const uint32_t key = w & SGK_KEY;
          const uint32_t op = key >> 4;
          const V* mt = sh.smat + (w >> 16);
          if (op == OP_DOT || op == OP_CDOT) {
            Acc r = apply_dot(a, key, mt);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
            if (lane == 0) DotAcc<T>::add(wdot[warp][sdslot[g]], r);
          } else {
            apply_gate(a, key, mt);
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          tphi[b ^ off[j]] = a[j];
          tlam[b ^ off[j]] = a[j + 8];
        }
      }
      __syncthreads();
    }
  }
};

// The kernel body.  One CTA owns one parameter set at a time (persistent over
// a work queue).  Fwd: stage program of the forward passes (pass_body's
// GenericStages or a specialised one, run in CTA mode); Bwd: that of the
// backward passes (GenericBwd or a specialised one).
template <typename T, int M, typename Fwd, typename Bwd>
__device__ __forceinline__ void adjoint_body(const AdjArgs J) {
  using V = typename CxT<T>::V;
  using Acc = T;
  constexpr int VB = sizeof(T) == 4 ? 9 : 8;
  constexpr int NVT = 1 << (M - VB);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassShared<T> sh;
  __shared__ double gacc[MAX_ADJ_PARAMS];
  __shared__ DotRows<T> wdot;
  __shared__ uint16_t sdslot[MAX_PASS_GATES];
  __shared__ uint32_t sdotg[MAX_PASS_DOTS];
  __shared__ double ered[PASS_THREADS / 32];
  __shared__ unsigned s_item;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t N = 1ull << J.n_int;
  V* phi = reinterpret_cast<V*>(J.slots) + size_t(blockIdx.x) * 2 * J.slot_amps;
  V* lam = phi + J.slot_amps;
  Ctrl* C = J.ctrls + blockIdx.x;
  uint8_t* flags = J.flag_slots + size_t(blockIdx.x) * J.slot_flags;

  for (;;) {
    if (tid == 0) s_item = atomicAdd(J.queue, 1u);
    __syncthreads();
    const unsigned set = s_item;
    __syncthreads();
    if (set >= J.nsets) break;

    // ---- forward: psi = U |0>
    for (uint64_t i = tid; i < N; i += PASS_THREADS) phi[i] = (i == 0) ? mkc(T(1), T(0)) : mkc(T(0), T(0));
    if (tid == 0) {
      C->creg = 0;
      C->m = 0;
      C->pm = C->pv = C->px = 0;
      C->ps = 1.0;
      C->ticket = 0;
      C->status = 0;
      C->n_trace = MAX_TRACE;
    }
    __threadfence_block();
    __syncthreads();
    PassArgs A = J.fwd;
    A.state = phi;
    A.ctrl = C;
    A.flags = flags;
    A.mats = reinterpret_cast<const V*>(J.fwd.mats) + uint64_t(set) * J.f_mat_stride;
    A.n = J.n_int;
    for (uint32_t pi = 0; pi < J.f_npasses; ++pi) {
      A.pass = int(pi);  // specialised stage programs select by it
      pass_body<T, M, true, Fwd>(A, int(pi), sh, smem_raw);
    }

    // ---- lambda = H psi and E = <psi|lambda>
    {
      // Hamiltonian terms staged in the (idle) dynamic shared memory, their
      // coefficients converted once to the state's precision (complex64:
      // FP32, whose error stays far below the state's own; converting per
      // term per amplitude, or summing in FP64, would bound this step at
      // GB300's FP64 rate); the coefficients first, so that they stay aligned
      using AV = typename CxT<Acc>::V;
      AV* hc = reinterpret_cast<AV*>(smem_raw);
      uint64_t* hz = reinterpret_cast<uint64_t*>(hc + J.nterms);
      for (uint32_t t = tid; t < J.nterms; t += PASS_THREADS) {
        hz[t] = J.hz[t];
        hc[t] = mkc(Acc(J.hc[t].x), Acc(J.hc[t].y));
      }
      __syncthreads();
      // the group's coefficient at j, sum_t c_t i^k_t (-1)^{|j & z_t|}; the
      // masks in 32 bits where the state has at most 32 qubits
      double e = (J.n_int <= 32) ? lambda_h<uint32_t, T>(J, phi, lam, hc, hz, N)
                                 : lambda_h<uint64_t, T>(J, phi, lam, hc, hz, N);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
      if (lane == 0) ered[warp] = e;
      for (uint32_t p = tid; p < J.n_params; p += PASS_THREADS) gacc[p] = 0.0;
      __threadfence_block();
      __syncthreads();
      if (tid == 0) {
        double s = 0;
        for (int w = 0; w < PASS_THREADS / 32; ++w) s += ered[w];
        J.val_out[set] = s;
      }
    }

    // ---- backward passes over phi and lambda
    V* tphi = reinterpret_cast<V*>(smem_raw);
    V* tlam = tphi + (1 << M);
    const V* bm = reinterpret_cast<const V*>(J.b_mats) + uint64_t(set) * J.b_mat_stride;
    for (uint32_t bp = 0; bp < J.b_npasses; ++bp) {
      if (tid == 0) sh.sp = J.b_passes[bp];
      __syncthreads();
      const DPass& sp = sh.sp;
      const int L = sp.L;
      uint32_t ndots = 0;
      for (int g = tid; g < int(sp.ng); g += PASS_THREADS) {
        const DGate d = J.b_gates[sp.g0 + g];
        sh.sgk[g] = uint32_t(d.key) | SGK_ON | (d.mat << 16);
        sdslot[g] = d.dslot;
        if (d.op == OP_DOT || d.op == OP_CDOT) sdotg[d.dslot] = d.gidx;
      }
      for (int i = tid; i < int(sp.nmat); i += PASS_THREADS) sh.smat[i] = bm[sp.mat0 + i];
      for (int i = tid; i < (PASS_THREADS / 32) * MAX_PASS_DOTS; i += PASS_THREADS) (&wdot[0][0])[i] = DotAcc<T>::zero();
      const int hb = M - L;
      for (int c = tid; c < (1 << hb); c += PASS_THREADS) {
        uint64_t o = 0;
        for (int k = 0; k < hb; ++k)
          if ((c >> k) & 1) o |= 1ull << sp.tq[L + k];
        sh.schunk[c] = o;
      }
      __syncthreads();
      for (int g = 0; g < int(sp.ng); ++g) {
        const uint32_t op = (sh.sgk[g] & SGK_KEY) >> 4;
        if (op == OP_DOT || op == OP_CDOT) ndots = max(ndots, uint32_t(sdslot[g]) + 1);
      }
      uint64_t tmask = 0;
      for (int j = 0; j < M; ++j) tmask |= 1ull << sp.tq[j];
      const uint64_t omask = (N - 1) & ~tmask;
      const uint64_t ntiles = 1ull << (J.n_int - M);
      const int vl = sizeof(T) == 4 ? L - 1 : L;
      const uint32_t wv = uint32_t(tid) & ((1u << vl) - 1u);
      const uint32_t woff = sizeof(T) == 4 ? (wv << 1) : wv;
      const uint32_t c0 = uint32_t(tid) >> vl;
      const uint32_t q0 = swz<T>((c0 << L) | woff);

      const uint64_t s1 = omask & (~omask + 1);  // deposit of 1: the lowest outer bit
      uint64_t base = 0;
      for (uint64_t u = 0; u < ntiles; ++u, base = spread_add(base, s1, omask)) {
#pragma unroll
        for (int k = 0; k < NVT; ++k) {
          const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
          const uint64_t gi = base | sh.schunk[ch] | woff;
          const uint32_t p = q0 ^ swz<T>(uint32_t(k) << VB);
          cp_async16(tphi + p, phi + gi);
          cp_async16(tlam + p, lam + gi);
        }
        cp_async_commit();
        cp_async_wait<0>();
        __syncthreads();
        Bwd::template run<T, M>(J.b_stages, bp, sp, sh, sdslot, tphi, tlam, wdot);
#pragma unroll
        for (int k = 0; k < NVT; ++k) {
          const uint32_t ch = c0 + (uint32_t(k) << (VB - L));
          const uint64_t gi = base | sh.schunk[ch] | woff;
          const uint32_t p = q0 ^ swz<T>(uint32_t(k) << VB);
          if constexpr (sizeof(T) == 4) {
            __stcg(reinterpret_cast<float4*>(phi) + (gi >> 1), *reinterpret_cast<const float4*>(tphi + p));
            __stcg(reinterpret_cast<float4*>(lam) + (gi >> 1), *reinterpret_cast<const float4*>(tlam + p));
          } else {
            __stcg(phi + gi, tphi[p]);
            __stcg(lam + gi, tlam[p]);
          }
        }
        __syncthreads();
      }
      // per-pass accumulators into the gradient (fixed order: warps, then dots)
      if (tid == 0)
        for (uint32_t d = 0; d < ndots; ++d) {
          double s = 0;
          for (int w = 0; w < PASS_THREADS / 32; ++w) s += DotAcc<T>::get(wdot[w][d]);
          gacc[sdotg[d]] += s;
        }
      __syncthreads();
    }
    for (uint32_t p = tid; p < J.n_params; p += PASS_THREADS)
      J.grad_out[uint64_t(set) * J.n_params + p] = gacc[p];
    __syncthreads();
  }
}

}  // namespace svk
