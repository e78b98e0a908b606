// batch_body.cuh -- persistent batched execution of many trajectories.
//
// One launch runs a whole batch: each CTA repeatedly takes the next
// trajectory from an atomic work queue (the host orders the queue longest
// first), initialises its private state slot to |0...0>, runs every pass of
// the trajectory's program itself (CTA mode of pass_body: the CTA walks all
// tiles, keeps the measurement table in shared memory and runs the draws and
// feed-forward predicates after a block barrier), and writes the classical
// register.  Trajectories of different qubit counts share the launch; the
// work queue is the only inter-CTA communication, so no CTA ever waits on
// another.
//
// The body is a template over the passes' stage program, so that it is
// compiled both ahead of time with the generic, plan-driven one (kern_batch.cu)
// and at run time with stage programs specialised to the batch's programs
// (jit.cpp).
#pragma once
#include "pass_body.cuh"

namespace svk {
using namespace svp;

// The kernel body; Stages: the stage program of the passes (pass_body's
// GenericStages, or one specialised to the batch's programs, which selects a
// program's pass by PassArgs::pass = the program's first global pass + pi).
template <typename T, int M, typename Stages>
__device__ __forceinline__ void batch_body(const BatchArgs B) {
  using V = typename CxT<T>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassShared<T> sh;
  __shared__ unsigned s_item;
  const int tid = threadIdx.x;
  V* slot = reinterpret_cast<V*>(B.state_slots) + size_t(blockIdx.x) * B.slot_amps;
  Ctrl* C = B.ctrls + blockIdx.x;
  uint8_t* flags = B.flag_slots + size_t(blockIdx.x) * B.slot_flags;
  for (;;) {
    if (tid == 0) s_item = atomicAdd(B.queue, 1u);
    __syncthreads();
    const unsigned it = s_item;
    __syncthreads();
    if (it >= B.n_items) break;
    const BatchItem w = B.items[it];
    const BatchProg P = B.progs[w.prog];
    const uint64_t N = 1ull << w.n_int;
    for (uint64_t i = tid; i < N; i += PASS_THREADS) slot[i] = (i == 0) ? mkc(T(1), T(0)) : mkc(T(0), T(0));
    if (tid == 0) {
      C->creg = 0;
      C->seed = B.seed;
      C->stream = w.stream;
      C->shot = w.shot;
      C->m = 0;
      C->pm = C->pv = C->px = 0;
      C->ps = 1.0;
      C->ticket = 0;
      C->status = 0;
      C->n_trace = B.trace_out ? 0 : MAX_TRACE;  // draw records only for shot branching
      for (uint32_t k = 0; k < P.ninit; ++k) {  // COND evaluations before the first measurement
        const DScalar s = P.init[k];
        const bool par = s.flag < 0 || flags[s.flag];
        const bool pred = (0ull & s.mask) == s.value;
        flags[s.f_then] = par && pred;
        if (s.f_else >= 0) flags[s.f_else] = par && !pred;
      }
    }
    __threadfence_block();
    __syncthreads();
    PassArgs A;
    A.state = slot;
    A.passes = P.passes;
    A.gates = P.gates;
    A.stages = P.stages;
    A.scalars = P.scalars;
    A.mats = P.mats;
    A.flags = flags;
    A.ctrl = C;
    A.trace = B.trace_out ? B.trace_slots + size_t(blockIdx.x) * MAX_TRACE : nullptr;
    A.partials = nullptr;
    A.n = int(w.n_int);
    A.dense_tc = 0;  // tensor-core dense gates are a grid-pass feature
    A.gen_init = 0;  // each trajectory's slot is initialised by this kernel
    A.work = B.work;
    for (uint32_t pi = 0; pi < P.npasses; ++pi) {
      A.pass = int(P.jit_base + pi);
      pass_body<T, M, true, Stages>(A, int(pi), sh, smem_raw);
    }
    if (tid == 0) {
      B.creg_out[w.out] = C->creg;
      if (C->status) atomicCAS(B.status_out, 0, C->status);
      if (B.trace_out) B.m_out[w.out] = C->m;
    }
    if (B.trace_out) {  // the trajectory's draws, in the compact form the shot walk reads
      const uint64_t m = C->m, lim = B.trace_cap < uint32_t(MAX_TRACE) ? B.trace_cap : uint32_t(MAX_TRACE);
      const uint32_t k = uint32_t(m < lim ? m : lim);
      for (uint32_t d = tid; d < k; d += PASS_THREADS) {
        const DTrace t = A.trace[d];
        BrDraw o;
        o.p0 = t.p0;
        o.p1 = t.p1;
        o.outcome = t.outcome;
        o.child = -1;
        B.trace_out[size_t(w.out) * B.trace_cap + d] = o;
      }
    }
    __syncthreads();
  }
}

}  // namespace svk
