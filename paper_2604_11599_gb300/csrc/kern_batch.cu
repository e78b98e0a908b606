// kern_batch.cu -- persistent batched execution of many trajectories: the
// kernel compiled ahead of time with the generic, plan-driven stage program
// (the method and the kernel body: batch_body.cuh).
#include "batch_body.cuh"

namespace svk {

template <typename T, int M>
__global__ void __launch_bounds__(PASS_THREADS, (sizeof(T) == 4 ? 2 : 1)) k_batch(const BatchArgs B) {
  batch_body<T, M, GenericStages>(B);
}

template <typename T>
static size_t batch_smem() {
  using V = typename CxT<T>::V;
  const size_t one = (size_t(1) << BATCH_TILE_BITS) * sizeof(V);
  return 2 * one <= size_t(128) * 1024 ? 2 * one : one;
}

size_t batch_smem_bytes(int dtype) { return dtype == SV_C64 ? batch_smem<float>() : batch_smem<double>(); }

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
