// kern_measure.cu -- terminal sampling and Pauli-sum expectation values.
//
// Sampling (shots, Sec. IV-C): FP64 block sums of |amp|^2 over fixed
// 4096-amplitude blocks, an exclusive scan of the block sums, then one warp
// per shot: Philox draw u for (seed, stream, shot, 2^32), binary search of the
// block whose running CDF passes u * total, and a warp-scan walk through that
// block for the smallest index with CDF > u * total.
//
// Expectation (the energy <H> of the paper's VQE checks, Sec. IV-A.2 and
// IV-D): terms that share an X mask x are evaluated in one read of the state.
// For P = i^{|x&z|} X^x Z^z (Y where both bits are set),
//   <psi|P|psi> = sum_i conj(psi_i) i^k (-1)^{|(i^x)&z|} psi_{i^x},  k = |x&z| mod 4,
// and each pair (i, i^x) contributes s(i) * {2Re w, 2Im w, -2Re w, -2Im w}[k]
// with w = conj(psi_i) psi_{i^x}, s(i) = (-1)^{|i&z|}.
#include "dev_common.cuh"
#include "kernels.h"

namespace svk {
using namespace svp;

constexpr int SAMPLE_BLOCK_BITS = 12;

uint64_t sample_blocks(int n) { return n > SAMPLE_BLOCK_BITS ? (1ull << (n - SAMPLE_BLOCK_BITS)) : 1ull; }

template <typename T>
__device__ __forceinline__ double abs2d(typename CxT<T>::V v) {
  return fma(double(v.x), double(v.x), double(v.y) * double(v.y));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T>
__global__ void __launch_bounds__(256) k_block_sums(SampleArgs a, int bbits) {
  using V = typename CxT<T>::V;
  const V* s = reinterpret_cast<const V*>(a.state);
  __shared__ double ws[8];
  const uint64_t b = blockIdx.x;
  const int tid = threadIdx.x;
  const uint64_t base = b << bbits;
  const int per = (1 << bbits);
  double acc = 0;
  for (int i = tid; i < per; i += 256) acc += abs2d<T>(s[base + i]);
  acc = warp_sum_d(acc);
  if ((tid & 31) == 0) ws[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double t = 0;
    for (int w = 0; w < 8; ++w) t += ws[w];
    a.block_sums[b] = t;
  }
}

// exclusive scan of nb block sums by one CTA (fixed order)
__global__ void __launch_bounds__(1024) k_scan_blocks(SampleArgs a, uint64_t nb) {
  __shared__ double tsum[1024];
  const int tid = threadIdx.x;
  const uint64_t per = (nb + 1023) / 1024;
  const uint64_t lo = tid * per, hi = lo + per < nb ? lo + per : nb;
  double s = 0;
  for (uint64_t i = lo; i < hi; ++i) s += a.block_sums[i];
  tsum[tid] = s;
  __syncthreads();
  if (tid == 0) {
    double run = 0;
    for (int t = 0; t < 1024; ++t) {
      const double v = tsum[t];
      tsum[t] = run;
      run += v;
    }
    a.block_prefix[nb] = run;
  }
  __syncthreads();
  double run = tsum[tid];
  for (uint64_t i = lo; i < hi; ++i) {
    a.block_prefix[i] = run;
    run += a.block_sums[i];
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_sample_search(SampleArgs a, uint64_t nb, int bbits) {
  using V = typename CxT<T>::V;
  const V* st = reinterpret_cast<const V*>(a.state);
  const int lane = threadIdx.x & 31;
  const uint64_t shot = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (shot >= a.shots) return;
  const double total = a.block_prefix[nb];
  const double u = draw_uniform(a.seed, a.stream, a.shot0 + shot, 1ull << 32);
  const double target = u * total;
  // smallest block b with prefix[b+1] > target
  uint64_t lo = 0, hi = nb - 1;
  while (lo < hi) {
    const uint64_t mid = lo + (hi - lo) / 2;
    if (a.block_prefix[mid + 1] > target) hi = mid;
    else lo = mid + 1;
  }
  const uint64_t per = 1ull << bbits;
  uint64_t found = ~0ull, last_nz = 0;
  for (uint64_t b = lo; b < nb && found == ~0ull; ++b) {
    double run = a.block_prefix[b];
    for (uint64_t c = 0; c < per; c += 32) {
      const uint64_t i = (b << bbits) + c + lane;
      const double p = abs2d<T>(st[i]);
      double inc = p;  // inclusive warp scan
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      const unsigned hit = __ballot_sync(0xffffffffu, run + inc > target && p > 0);
      const unsigned nz = __ballot_sync(0xffffffffu, p > 0);
      if (nz) last_nz = (b << bbits) + c + (31 - __clz(nz));
      if (hit) {
        found = (b << bbits) + c + (__ffs(hit) - 1);
        break;
      }
      run += __shfl_sync(0xffffffffu, inc, 31);
    }
  }
  if (lane == 0) a.out[shot] = found != ~0ull ? found : last_nz;
}

template <typename T>
static cudaError_t launch_sample_t(const SampleArgs& a, int sms, cudaStream_t s) {
  const int bbits = a.n > SAMPLE_BLOCK_BITS ? SAMPLE_BLOCK_BITS : a.n;
  const uint64_t nb = sample_blocks(a.n);
  k_block_sums<T><<<unsigned(nb), 256, 0, s>>>(a, bbits);
  k_scan_blocks<<<1, 1024, 0, s>>>(a, nb);
  if (a.shots) {
    const uint64_t warps = a.shots, blocks = (warps * 32 + 255) / 256;
    k_sample_search<T><<<unsigned(blocks), 256, 0, s>>>(a, nb, bbits);
  }
  (void)sms;
  return cudaGetLastError();
}

cudaError_t launch_sample(int dtype, const SampleArgs& a, int sms, cudaStream_t s) {
  return dtype == SV_C64 ? launch_sample_t<float>(a, sms, s) : launch_sample_t<double>(a, sms, s);
}

// ---------------------------------------------------------------------- expectation values
constexpr int EXP_TERMS = 32;
constexpr int EXP_CHUNK = 16;  // pairs summed in the state precision before an FP64 add

template <typename T>
__global__ void __launch_bounds__(256) k_expval_group(ExpvalArgs a) {
  using V = typename CxT<T>::V;
  const V* st = reinterpret_cast<const V*>(a.state);
  __shared__ uint64_t zs[EXP_TERMS];
  __shared__ int ks[EXP_TERMS];
  __shared__ double red[8][EXP_TERMS];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  if (tid < a.nterms) {
    zs[tid] = a.z_masks[tid];
    ks[tid] = a.phase[tid];
  }
  __syncthreads();
  const int nt = a.nterms;
  double acc[EXP_TERMS];
  T part[EXP_TERMS];
#pragma unroll
  for (int t = 0; t < EXP_TERMS; ++t) {
    acc[t] = 0;
    part[t] = 0;
  }
  const uint64_t N = 1ull << a.n;
  const uint64_t x = a.x_mask;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  int cnt = 0;
  if (x == 0) {
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + tid; i < N; i += stride) {
      const V v = st[i];
      const T p = fma(v.x, v.x, v.y * v.y);
#pragma unroll
      for (int t = 0; t < EXP_TERMS; ++t)
        if (t < nt) part[t] += (__popcll(i & zs[t]) & 1) ? -p : p;
      if (++cnt == EXP_CHUNK) {
#pragma unroll
        for (int t = 0; t < EXP_TERMS; ++t) {
          acc[t] += double(part[t]);
          part[t] = 0;
        }
        cnt = 0;
      }
    }
  } else {
    const int h = 63 - __clzll((long long)x);
    const uint64_t half = N >> 1;
    const uint64_t lowm = (1ull << h) - 1;
    for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + tid; r < half; r += stride) {
      const uint64_t i = ((r >> h) << (h + 1)) | (r & lowm);  // bit h of i is 0
      const V pi_ = st[i], pj = st[i ^ x];
      // w = conj(psi_i) psi_j
      const T wr = fma(pi_.x, pj.x, pi_.y * pj.y), wi = fma(pi_.x, pj.y, -pi_.y * pj.x);
#pragma unroll
      for (int t = 0; t < EXP_TERMS; ++t) {
        if (t < nt) {
          const int k = ks[t];
          T c = (k & 1) ? wi : wr;
          if (k >= 2) c = -c;
          c = c + c;
          part[t] += (__popcll(i & zs[t]) & 1) ? -c : c;
        }
      }
      if (++cnt == EXP_CHUNK) {
#pragma unroll
        for (int t = 0; t < EXP_TERMS; ++t) {
          acc[t] += double(part[t]);
          part[t] = 0;
        }
        cnt = 0;
      }
    }
  }
#pragma unroll
  for (int t = 0; t < EXP_TERMS; ++t) acc[t] += double(part[t]);
  // block reduction (fixed order)
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int t = 0; t < EXP_TERMS; ++t) {
    const double v = warp_sum_d(acc[t]);
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (tid < EXP_TERMS) {
    double s = 0;
    for (int w = 0; w < 8; ++w) s += red[w][tid];
    a.partials[blockIdx.x * EXP_TERMS + tid] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < nt) {
    double s = 0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(a.partials + b * EXP_TERMS + tid);
    a.out[tid] = s;
  }
  if (tid == 0) *a.ticket = 0;
}

cudaError_t launch_expval_group(int dtype, const ExpvalArgs& a, int grid, cudaStream_t s) {
  if (dtype == SV_C64) k_expval_group<float><<<grid, 256, 0, s>>>(a);
  else k_expval_group<double><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace svk
