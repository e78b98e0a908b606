// dev_tc.cuh -- fifth-generation tensor cores (tcgen05) for dense four-qubit
// unitaries on complex64 states.
//
// A dense 16 x 16 complex unitary U on the four register qubits of a stage is,
// over all 2^(n-4) register groups of the state, the real product
//   D[g][n] = sum_k A[g][k] * Bt[n][k]   (k, n over 32 = 16 interleaved re/im)
// with A[g] the group's amplitudes (re0 im0 re1 im1 ...) and Bt the 32 x 32
// real form of U: Bt[2r][2c] = Re U_rc, Bt[2r][2c+1] = -Im U_rc,
// Bt[2r+1][2c] = Im U_rc, Bt[2r+1][2c+1] = Re U_rc.  That is a dense
// contraction of 8 flops per amplitude and row of U (128 flops per complex64
// amplitude), so it goes to the tensor pipe as kind::tf32 MMAs.  TF32 keeps
// 10 mantissa bits; FP32-level accuracy comes from the three-product split
// A*B ~= Ahi*Bhi + Ahi*Blo + Alo*Bhi (Ahi = A truncated to TF32, Alo = A - Ahi
// exactly; the dropped Alo*Blo term and the truncation of the low parts are
// ~2^-20 relative), accumulated in FP32 in tensor memory.
//
// A (the amplitudes) goes to tensor memory: every thread writes its group's
// row into its own lane with tcgen05.st, so no shared-memory staging is needed.
// B (the gate) lives in shared memory in the no-swizzle K-major layout of
// core matrices (8 rows x 16 bytes, 128 contiguous bytes): element (row, k)
// of a 32-column matrix at byte (row / 8) * 1024 + (k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4, i.e. 128 bytes between core matrices along K
// and 1024 bytes between 8-row blocks.  Each MMA takes K = 8 (two core
// matrices along K), so k-step s starts 256 bytes further.
#pragma once
#include "dev_common.cuh"

namespace svk {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---------------------------------------------------------------- tensor memory
// Allocation and release are warp-wide (.sync.aligned): one full warp calls them.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
// order tcgen05 operations around thread barriers
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
// make generic-proxy shared-memory writes visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// 32 lanes x 32 columns of 32-bit words: thread l of the warp receives the
// 32 consecutive columns of lane (taddr lane field) + l.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// thread l writes 16 consecutive columns of lane (taddr lane field) + l
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Waits for the phase of the given parity to complete, at most `limit` polls
// (each poll may suspend the thread for a bounded, hardware-defined time).
// Returns false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---------------------------------------------------------------- MMA
// Shared-memory matrix descriptor: start address, leading (K) and stride
// (M/N) byte offsets between core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return uint64_t((saddr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
         (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (uint64_t(1) << 46);
}
// kind::tf32 instruction descriptor: D in FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}
// D (tensor memory) = A * B^T (+ D when acc != 0), A in tensor memory (row i
// in lane i, element k in column a_tmem + k), B in shared memory; issued by
// one thread.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive once on the mbarrier when every MMA issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// x truncated to TF32 (its top 19 bits: sign, exponent, 10 mantissa bits);
// x - tf32_hi(x) is exact in FP32 and below 2^-10 |x|, so the MMA's own
// truncation of that low part leaves ~2^-20 |x| of error
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// byte offset of element (row, k) in the 32-column core-matrix layout
__host__ __device__ constexpr uint32_t cm_off(uint32_t row, uint32_t k) {
  return (row >> 3) * 1024u + (k >> 2) * 128u + (row & 7u) * 16u + (k & 3u) * 4u;
}

// Tensor memory of one CTA: A of rows 0..127 (warps 0-3) in columns 0..63
// (TF32 high parts 0..31, low parts 32..63), A of rows 128..255 (warps 4-7) in
// 64..127, the two 128 x 32 FP32 accumulators in 128..159 and 160..191.
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr uint32_t TC_WAIT_POLLS = 1u << 20;  // bounded MMA completion wait

// Shared state of the tensor-core path (part of the pass kernel's static shared memory).
constexpr int TC_SLOTS = 4;  // dense gates per pass (MAX_PASS_MAT holds four 16 x 16 matrices)

struct TcShared {
  __align__(128) float bt[TC_SLOTS][2][1024];  // B high / low parts per dense gate, core-matrix layout
  uint64_t bar;                                // MMA completion
  uint32_t tmem;                               // tensor-memory base address
  uint32_t slot_mat[TC_SLOTS];                 // matrix offset (in the pass's matrix block) of each slot
};

// Per-thread view of it, passed to the stages.
struct TcCtx {
  TcShared* s;
  const void* smat;  // the pass's matrix block in shared memory
  uint32_t tmem;   // tensor-memory base address
  uint32_t phase;  // completed MMA batches (parity of the next wait)
  bool on;         // dense gates of this pass go to the tensor cores
  bool ok;         // false after a wait ran out: the thread issues and waits no more
  uint32_t drain;  // thread 0: 1 + parity of the batch whose wait ran out (0: none)
};

// Give-up path of a completion wait that ran out (SV_ERR_TIMEOUT): before the
// CTA frees its tensor memory, the issuing thread waits once more, again
// bounded, for the batch it gave up on (the last one it committed), so that
// no MMA it issued can still write columns the CTA no longer owns if that
// batch finishes within the second wait.  Called by every thread of the CTA.
__device__ __forceinline__ void tc_drain(TcCtx& tc) {
  if (threadIdx.x == 0 && tc.drain) mbar_wait(&tc.s->bar, tc.drain - 1u, TC_WAIT_POLLS);
}

}  // namespace svk
