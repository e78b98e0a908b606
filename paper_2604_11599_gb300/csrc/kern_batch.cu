// kern_batch.cu -- persistent batched execution of many trajectories.
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
#include "pass_body.cuh"

namespace svk {
using namespace svp;

template <typename T, int M>
__global__ void __launch_bounds__(PASS_THREADS, (sizeof(T) == 4 ? 2 : 1)) k_batch(const BatchArgs B) {
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
    A.pass = 0;
    A.dense_tc = 0;  // tensor-core dense gates are a grid-pass feature
    A.gen_init = 0;  // each trajectory's slot is initialised by this kernel
    A.work = B.work;
    for (uint32_t pi = 0; pi < P.npasses; ++pi) pass_body<T, M, true>(A, int(pi), sh, smem_raw);
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

template <typename T>
static size_t batch_smem() {
  using V = typename CxT<T>::V;
  const size_t one = (size_t(1) << BATCH_TILE_BITS) * sizeof(V);
  return 2 * one <= size_t(128) * 1024 ? 2 * one : one;
}

cudaError_t launch_batch(int dtype, const BatchArgs& a, int grid, cudaStream_t s) {
  if (dtype == SV_C64)
    k_batch<float, BATCH_TILE_BITS><<<grid, PASS_THREADS, batch_smem<float>(), s>>>(a);
  else
    k_batch<double, BATCH_TILE_BITS><<<grid, PASS_THREADS, batch_smem<double>(), s>>>(a);
  return cudaGetLastError();
}

cudaError_t batch_occupancy(int dtype, int* blocks_per_sm) {
  static int cache[2] = {0, 0};
  int& c = cache[dtype == SV_C64 ? 0 : 1];
  if (c) {
    *blocks_per_sm = c;
    return cudaSuccess;
  }
  cudaError_t e;
  if (dtype == SV_C64) {
    e = cudaFuncSetAttribute(k_batch<float, BATCH_TILE_BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(batch_smem<float>()));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_batch<float, BATCH_TILE_BITS>, PASS_THREADS,
                                                        batch_smem<float>());
  } else {
    e = cudaFuncSetAttribute(k_batch<double, BATCH_TILE_BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             int(batch_smem<double>()));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_batch<double, BATCH_TILE_BITS>, PASS_THREADS,
                                                        batch_smem<double>());
  }
  if (e != cudaSuccess || c < 1) c = 1;
  *blocks_per_sm = c;
  return e;
}

}  // namespace svk
