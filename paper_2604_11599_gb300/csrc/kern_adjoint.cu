// kern_adjoint.cu -- batched adjoint gradients of <H> for parameterised
// circuits: the kernel compiled ahead of time with the generic, plan-driven
// stage programs (the method and the kernel body: adjoint_body.cuh).
#include "adjoint_body.cuh"

namespace svk {

// complex64: two CTAs per SM (128 registers, no spills of note), so that the
// dependent FP32 chains of one CTA's stages overlap the other's; complex128
// keeps one (its registers would spill at 128)
template <typename T, int M>
__global__ void __launch_bounds__(PASS_THREADS, sizeof(T) == 4 ? 2 : 1) k_adjoint(const AdjArgs J) {
  adjoint_body<T, M, GenericStages, GenericBwd>(J);
}

template <typename T>
static size_t adjoint_smem(uint32_t nterms) {  // dynamic: two tiles, or the Hamiltonian terms
  using V = typename CxT<T>::V;
  const size_t tiles = 2 * (size_t(1) << BATCH_TILE_BITS) * sizeof(V);
  const size_t terms = size_t(nterms) * (sizeof(uint64_t) + sizeof(double2));
  return tiles > terms ? tiles : terms;
}

size_t adjoint_smem_bytes(int dtype, uint32_t nterms) {
  return dtype == SV_C64 ? adjoint_smem<float>(nterms) : adjoint_smem<double>(nterms);
}

cudaError_t launch_adjoint(int dtype, const AdjArgs& a, int grid, cudaStream_t s) {
  if (dtype == SV_C64) {
    const size_t sm = adjoint_smem<float>(a.nterms);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint<float, BATCH_TILE_BITS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    k_adjoint<float, BATCH_TILE_BITS><<<grid, PASS_THREADS, sm, s>>>(a);
  } else {
    const size_t sm = adjoint_smem<double>(a.nterms);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint<double, BATCH_TILE_BITS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e != cudaSuccess) return e;
    k_adjoint<double, BATCH_TILE_BITS><<<grid, PASS_THREADS, sm, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t adjoint_occupancy(int dtype, uint32_t nterms, int* blocks_per_sm) {
  cudaError_t e;
  if (dtype == SV_C64) {
    const size_t sm = adjoint_smem<float>(nterms);
    e = cudaFuncSetAttribute(k_adjoint<float, BATCH_TILE_BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_adjoint<float, BATCH_TILE_BITS>,
                                                        PASS_THREADS, sm);
  } else {
    const size_t sm = adjoint_smem<double>(nterms);
    e = cudaFuncSetAttribute(k_adjoint<double, BATCH_TILE_BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_adjoint<double, BATCH_TILE_BITS>,
                                                        PASS_THREADS, sm);
  }
  if (e != cudaSuccess || *blocks_per_sm < 1) *blocks_per_sm = 1;
  return e;
}

}  // namespace svk
