// kern_pass.cu -- gate matrices, state init and the grid-wide pass kernel.

#include <cstdio>

#include <algorithm>

#include "pass_body.cuh"

namespace svk {
using namespace svp;

// Matrix jobs of a plan from the run-time parameters (FP64, rounded to the
// state precision).  blockIdx.y indexes parameter sets: set y reads
// params + y * params_stride and writes mats + y * mats_stride.
template <typename T>
__global__ void k_prep(PrepArgs P) {
  using V = typename CxT<T>::V;
  V* mats = reinterpret_cast<V*>(P.mats) + uint64_t(blockIdx.y) * P.mats_stride;
  const double* params = P.params ? P.params + uint64_t(blockIdx.y) * P.params_stride : nullptr;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P.njobs) {
    const DJob j = P.jobs[i];
    if (j.kind == J_CONST) {
      for (uint32_t k = 0; k < j.len; ++k)
        mats[j.out + k] = mkc(T(P.consts[2 * (j.src + k)]), T(P.consts[2 * (j.src + k) + 1]));
    } else {
      double t[3];
      for (int k = 0; k < 3; ++k) {
        if (j.pidx[k] >= 0) {
          if (uint64_t(j.pidx[k]) < P.n_params) t[k] = j.angle[k] * params[j.pidx[k]];
          else {
            t[k] = 0;
            if (P.ctrl) P.ctrl->status = SV_ERR_ARG;
          }
        } else {
          t[k] = j.angle[k];
        }
      }
      double2 m[4];
      std_gate_2x2(j.gate, t, m);
      if (j.kind == J_DERIV) {
        // M = 2 * scale * (dU/da) * U^dagger: the gradient entry is Re <lambda| M |phi>
        double2 d[4];
        const int slot = int(j.len);
        std_gate_deriv(j.gate, t, slot, d);
        const double f = 2.0 * j.angle[slot];
        for (int r = 0; r < 2; ++r)
          for (int c = 0; c < 2; ++c) {
            // (d U^dagger)[r][c] = sum_k d[r][k] conj(U[c][k])
            double re = 0, im = 0;
            for (int k = 0; k < 2; ++k) {
              const double2 a = d[2 * r + k], b = m[2 * c + k];
              re += a.x * b.x + a.y * b.y;
              im += a.y * b.x - a.x * b.y;
            }
            mats[j.out + 2 * r + c] = mkc(T(f * re), T(f * im));
          }
      } else {
        if (j.adj) {  // conjugate transpose
          const double2 m01 = m[1];
          m[1] = make_double2(m[2].x, -m[2].y);
          m[2] = make_double2(m01.x, -m01.y);
          m[0].y = -m[0].y;
          m[3].y = -m[3].y;
        }
        switch (j.op) {
          case OP_U: case OP_CU:
            for (int k = 0; k < 4; ++k) mats[j.out + k] = mkc(T(m[k].x), T(m[k].y));
            break;
          case OP_R:
            for (int k = 0; k < 4; ++k) mats[j.out + k] = mkc(T(m[k].x), T(0));
            break;
          case OP_RX:  // m00 = c, m01 = -i s
            mats[j.out] = mkc(T(m[0].x), T(0));
            mats[j.out + 1] = mkc(T(-m[1].y), T(0));
            break;
          case OP_D: case OP_CD:
            mats[j.out] = mkc(T(m[0].x), T(m[0].y));
            mats[j.out + 1] = mkc(T(m[3].x), T(m[3].y));
            break;
          case OP_RXF: case OP_RYF: {
            // RX: m00 = c, m01 = -i s; RY: m00 = c, m10 = s.  Factor the larger of
            // |c|, |s| out so that the remaining coefficient has magnitude <= 1.
            const double c = m[0].x, sn = j.op == OP_RXF ? -m[1].y : m[2].x;
            const bool form1 = fabs(sn) > fabs(c);
            mats[j.out] = mkc(T(form1 ? c / sn : sn / c), T(form1 ? 1 : 0));
            mats[j.out + 1] = mkc(T(form1 ? sn : c), T(0));
            break;
          }
          case OP_DZ: {  // diag(d0, d1) = d0 diag(1, d1 / d0), |d0| = 1
            const double2 d0 = m[0], d1 = m[3];
            mats[j.out] = mkc(T(d1.x * d0.x + d1.y * d0.y), T(d1.y * d0.x - d1.x * d0.y));
            mats[j.out + 1] = mkc(T(d0.x), T(d0.y));
            break;
          }
          default: break;
        }
      }
    }
  }
  if (i == 0 && blockIdx.y == 0 && P.ctrl) {
    Ctrl* C = P.ctrl;
    C->creg = 0;
    C->seed = P.seed;
    C->stream = P.stream;
    C->shot = P.shot;
    C->m = 0;
    C->pm = C->pv = C->px = 0;
    C->ps = 1.0;
    C->ticket = 0;
    C->n_trace = 0;
    for (int k = 0; k < P.ninit; ++k) {  // COND evaluations before the first measurement
      const DScalar s = P.init[k];
      const bool par = s.flag < 0 || P.flags[s.flag];
      const bool pred = (0ull & s.mask) == s.value;
      P.flags[s.f_then] = par && pred;
      if (s.f_else >= 0) P.flags[s.f_else] = par && !pred;
    }
  }
}

template <typename T>
__global__ void k_init_state(void* state, uint64_t n_amp) {
  using V = typename CxT<T>::V;
  V* s = reinterpret_cast<V*>(state);
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n_amp; i += stride)
    s[i] = (i == 0) ? mkc(T(1), T(0)) : mkc(T(0), T(0));
}

// TC: the variant for passes holding a dense four-qubit gate (tensor cores);
// PROJ: the variant for passes that may start with a measurement projector pending
template <typename T, int M, bool TC, bool PROJ>
__global__ void __launch_bounds__(PASS_THREADS, (sizeof(T) == 4 ? 2 : 1)) k_pass(const PassArgs A, const int pi) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PassShared<T, TC> sh;
  pass_body<T, M, false, GenericStages, TC, PROJ>(A, pi, sh, smem_raw);
}

// ============================================================ host launchers

template <typename T, int M>
static size_t pass_smem() {
  using V = typename CxT<T>::V;
  const size_t one = (size_t(1) << M) * sizeof(V);
  return 2 * one <= size_t(128) * 1024 ? 2 * one : one;
}

template <typename T, int M, bool TC, bool PROJ>
static cudaError_t launch_pass_v(const PassArgs& a, int pi, int grid, cudaStream_t s) {
  const size_t smem = pass_smem<T, M>();
  static bool attr = false;  // dynamic shared memory above 48 KiB, once per variant
  if (!attr) {
    const cudaError_t e =
        cudaFuncSetAttribute(k_pass<T, M, TC, PROJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_pass<T, M, TC, PROJ><<<grid, PASS_THREADS, smem, s>>>(a, pi);
  return cudaGetLastError();
}

template <typename T, int M>
static cudaError_t launch_pass_tm(const PassArgs& a, int pi, int grid, cudaStream_t s, bool dense, bool proj) {
  if constexpr (sizeof(T) == 4 && M == 12)
    if (dense && a.dense_tc)
      return proj ? launch_pass_v<T, M, true, true>(a, pi, grid, s) : launch_pass_v<T, M, true, false>(a, pi, grid, s);
  return proj ? launch_pass_v<T, M, false, true>(a, pi, grid, s) : launch_pass_v<T, M, false, false>(a, pi, grid, s);
}

// Resident CTAs per SM from the kernel's own resource counts.  The runtime's
// occupancy query answers 1 for any kernel that holds tcgen05 instructions
// (measured on GB300), although CTAs that each allocate a slice of tensor
// memory run side by side; the pass kernels take 64 of the 512 columns.
static int blocks_per_sm(const cudaFuncAttributes& fa, size_t dyn_smem, int threads) {
  int dev = 0;
  cudaGetDevice(&dev);
  int regs_sm = 65536, smem_sm = 233472, smem_rsv = 1024, thr_sm = 2048, blk_sm = 32;
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
  int n = blk_sm;
  if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
  n = std::min(n, int(size_t(smem_sm) / (fa.sharedSizeBytes + dyn_smem + size_t(smem_rsv))));
  n = std::min(n, thr_sm / threads);
  n = std::min(n, int(512 / TC_TMEM_COLS));
  return n;
}

template <typename T, int M>
static cudaError_t pass_attr_tm(int* per_sm) {
  const size_t smem = pass_smem<T, M>();
  cudaError_t e = cudaFuncSetAttribute(k_pass<T, M, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_pass<T, M, false, false>);
  if (e == cudaSuccess) *per_sm = blocks_per_sm(fa, smem, PASS_THREADS);
  return e;
}

cudaError_t launch_pass(int dtype, const PassArgs& a, int pi, int grid, int m, cudaStream_t s, bool dense,
                        bool proj) {
  if (dtype == SV_C64) {
    switch (m) {
      case 10: return launch_pass_tm<float, 10>(a, pi, grid, s, dense, proj);
      case 11: return launch_pass_tm<float, 11>(a, pi, grid, s, dense, proj);
      case 12: return launch_pass_tm<float, 12>(a, pi, grid, s, dense, proj);
      case 13: return launch_pass_tm<float, 13>(a, pi, grid, s, dense, proj);
      case 14: return launch_pass_tm<float, 14>(a, pi, grid, s, dense, proj);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (m) {
    case 10: return launch_pass_tm<double, 10>(a, pi, grid, s, dense, proj);
    case 11: return launch_pass_tm<double, 11>(a, pi, grid, s, dense, proj);
    case 12: return launch_pass_tm<double, 12>(a, pi, grid, s, dense, proj);
    case 13: return launch_pass_tm<double, 13>(a, pi, grid, s, dense, proj);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_prep(int dtype, const PrepArgs& p, cudaStream_t s) {
  const dim3 blocks(p.njobs > 0 ? (p.njobs + 255) / 256 : 1, p.nsets > 0 ? p.nsets : 1);
  if (dtype == SV_C64) k_prep<float><<<blocks, 256, 0, s>>>(p);
  else k_prep<double><<<blocks, 256, 0, s>>>(p);
  return cudaGetLastError();
}

// The pass kernels' bounded completion wait (mbar_wait, dev_tc.cuh) on an
// mbarrier that nothing arrives at: phase 0 never completes, so the wait gives
// up after `polls` polls and the kernel reports what a timed-out pass reports.
// One warp, no MMA, no tensor memory.
__global__ void k_wait_probe(uint32_t polls, int32_t* status) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const bool done = mbar_wait(&bar, 0u, polls);
  if (__all_sync(0xffffffffu, !done) && threadIdx.x == 0) atomicCAS(status, 0, int32_t(SV_ERR_TIMEOUT));
}

cudaError_t launch_wait_probe(uint32_t polls, int32_t* status, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(polls, status);
  return cudaGetLastError();
}

cudaError_t launch_init_state(int dtype, void* state, uint64_t n_amp, int sms, cudaStream_t s) {
  const uint64_t want = (n_amp + 255) / 256;
  const int blocks = int(want < uint64_t(sms) * 8 ? want : uint64_t(sms) * 8);
  if (dtype == SV_C64) k_init_state<float><<<blocks, 256, 0, s>>>(state, n_amp);
  else k_init_state<double><<<blocks, 256, 0, s>>>(state, n_amp);
  return cudaGetLastError();
}

cudaError_t pass_occupancy(int dtype, int m, int* blocks_per_sm) {
  static int cache[2][MAX_TILE_BITS + 1] = {};
  const int d = dtype == SV_C64 ? 0 : 1;
  if (m < 10 || m > MAX_TILE_BITS || (d == 1 && m > 13)) return cudaErrorInvalidValue;
  int& c = cache[d][m];
  if (c) {
    *blocks_per_sm = c;
    return cudaSuccess;
  }
  cudaError_t e;
  if (d == 0) {
    switch (m) {
      case 10: e = pass_attr_tm<float, 10>(&c); break;
      case 11: e = pass_attr_tm<float, 11>(&c); break;
      case 12: e = pass_attr_tm<float, 12>(&c); break;
      case 13: e = pass_attr_tm<float, 13>(&c); break;
      default: e = pass_attr_tm<float, 14>(&c); break;
    }
  } else {
    switch (m) {
      case 10: e = pass_attr_tm<double, 10>(&c); break;
      case 11: e = pass_attr_tm<double, 11>(&c); break;
      case 12: e = pass_attr_tm<double, 12>(&c); break;
      default: e = pass_attr_tm<double, 13>(&c); break;
    }
  }
  if (e != cudaSuccess || c < 1) c = 1;
  *blocks_per_sm = c;
  return e;
}

}  // namespace svk
