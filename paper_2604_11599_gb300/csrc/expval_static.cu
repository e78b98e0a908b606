// expval_static.cu -- Pauli expectation values without any device allocation.
//
// sv_expval allocates its scratch (per-CTA partial sums, a completion
// counter) with cudaMalloc the first time it runs.  Some callers cannot let a
// library allocate device memory at all: applications whose whole device
// memory is handed out by their own allocator or fixed pool and that forbid
// side allocations, and latency-critical loops where cudaMalloc's implicit
// synchronisation with the device is not acceptable.  For them,
// sv_expval_static evaluates the same quantity with its scratch in the
// file-scope array below, which is part of the library's device image: every
// GPU that loads libsv holds it (kScratchBytes) until the process exits.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it.  Calls are therefore serialised by stream order; two
// calls that overlap on the GPU (different streams, or threads racing on
// one stream) race on the scratch and give wrong results.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/sv.h"
#include "dev_common.cuh"

namespace {

constexpr int kTermsPerLaunch = 32;
constexpr int kMaxCtas = 1024;
constexpr int kMaxTerms = 64;     // terms accepted per call
constexpr int kMaxDevices = 64;
constexpr size_t kCounterBytes = 256;  // completion counter, padded to the array's alignment
constexpr size_t kScratchBytes = kCounterBytes + size_t(kMaxCtas) * kTermsPerLaunch * sizeof(double);

// counter (offset 0) + per-CTA partial sums (offset 256)
static __device__ __align__(256) unsigned char g_expval_scratch[kScratchBytes];

struct StaticTerms {
  const void* state;
  double* out;
  uint64_t x_mask;
  int n;
  int nterms;
  uint64_t z[kTermsPerLaunch];
  int k[kTermsPerLaunch];     // |x & z| mod 4
  int slot[kTermsPerLaunch];  // index in out
};

template <typename T>
__global__ void __launch_bounds__(256) k_expval_static(const StaticTerms a, unsigned char* scratch) {
  using V = typename svk::CxT<T>::V;
  unsigned* counter = reinterpret_cast<unsigned*>(scratch);
  double* partials = reinterpret_cast<double*>(scratch + kCounterBytes);
  const V* st = reinterpret_cast<const V*>(a.state);
  __shared__ double red[8][kTermsPerLaunch];
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double acc[kTermsPerLaunch];
#pragma unroll
  for (int t = 0; t < kTermsPerLaunch; ++t) acc[t] = 0;
  const uint64_t N = 1ull << a.n;
  const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
  if (a.x_mask == 0) {
    // <Z^z> = sum_i |psi_i|^2 (-1)^{|i & z|}
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + tid; i < N; i += stride) {
      const V v = st[i];
      const double p = double(v.x) * double(v.x) + double(v.y) * double(v.y);
#pragma unroll
      for (int t = 0; t < kTermsPerLaunch; ++t)
        if (t < a.nterms) acc[t] += (__popcll(i & a.z[t]) & 1) ? -p : p;
    }
  } else {
    // pairs (i, i ^ x) with the top bit of x clear in i; w = conj(psi_i) psi_{i^x};
    // the pair adds (-1)^{|i&z|} * {2 Re w, 2 Im w, -2 Re w, -2 Im w}[|x&z| mod 4]
    const int h = 63 - __clzll((long long)a.x_mask);
    const uint64_t lowm = (1ull << h) - 1;
    for (uint64_t r = uint64_t(blockIdx.x) * blockDim.x + tid; r < (N >> 1); r += stride) {
      const uint64_t i = ((r >> h) << (h + 1)) | (r & lowm);
      const V pi = st[i], pj = st[i ^ a.x_mask];
      const double wr = double(pi.x) * double(pj.x) + double(pi.y) * double(pj.y);
      const double wi = double(pi.x) * double(pj.y) - double(pi.y) * double(pj.x);
#pragma unroll
      for (int t = 0; t < kTermsPerLaunch; ++t) {
        if (t < a.nterms) {
          double c = (a.k[t] & 1) ? wi : wr;
          if (a.k[t] >= 2) c = -c;
          c += c;
          acc[t] += (__popcll(i & a.z[t]) & 1) ? -c : c;
        }
      }
    }
  }
#pragma unroll
  for (int t = 0; t < kTermsPerLaunch; ++t) {
    double v = acc[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][t] = v;
  }
  __syncthreads();
  if (tid < kTermsPerLaunch) {
    double s = 0;
    for (int w = 0; w < 8; ++w) s += red[w][tid];
    partials[blockIdx.x * kTermsPerLaunch + tid] = s;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < a.nterms) {
    double s = 0;
    for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(partials + b * kTermsPerLaunch + tid);
    a.out[a.slot[tid]] = s;
  }
}

thread_local std::string t_err;

// Device address of the scratch array, looked up once per device (the first
// call with that device current).  cudaDeviceReset unloads the library's
// device image; a process that resets a device must not call
// sv_expval_static on it again, since the cached address would be stale.
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

sv_status scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    t_err = "sv_expval_static: no usable current device";
    return SV_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_expval_scratch);
    if (e != cudaSuccess || !p) {
      t_err = std::string("sv_expval_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
      return SV_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SV_OK;
}

}  // namespace

namespace svapi {
void set_last_error(const std::string& msg);  // sv_api.cu: message returned by sv_last_error()
}

namespace {
sv_status report(sv_status st) {
  if (st != SV_OK) svapi::set_last_error(t_err);
  return st;
}
}  // namespace

extern "C" {

static sv_status expval_static_impl(const void* dev_state, int n, sv_dtype dtype, const sv_pauli* terms,
                                    size_t n_terms, double* dev_out, void* cuda_stream) {
  t_err.clear();
  if (n < 1 || n > 34) {
    t_err = "sv_expval_static: n must be in 1..34";
    return SV_ERR_ARG;
  }
  if (dtype != SV_C64 && dtype != SV_C128) {
    t_err = "sv_expval_static: unknown dtype";
    return SV_ERR_ARG;
  }
  if (n_terms > size_t(kMaxTerms)) {
    t_err = "sv_expval_static: at most 64 Pauli terms per call (the static scratch is sized for that)";
    return SV_ERR_ARG;
  }
  if (!n_terms) return SV_OK;
  if (!dev_state || !dev_out || !terms) {
    t_err = "sv_expval_static: null state, output or terms";
    return SV_ERR_ARG;
  }
  if (reinterpret_cast<uintptr_t>(dev_state) % 16) {
    t_err = "sv_expval_static: state must be 16-byte aligned";
    return SV_ERR_ARG;
  }
  const uint64_t lim = (1ull << n) - 1;
  for (size_t t = 0; t < n_terms; ++t)
    if ((terms[t].x_mask | terms[t].z_mask) & ~lim) {
      t_err = "sv_expval_static: a Pauli term acts on a qubit >= n";
      return SV_ERR_ARG;
    }
  void* scratch = nullptr;
  sv_status st = scratch_address(&scratch);
  if (st != SV_OK) return st;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  // the state and the output must live on the current device, whose copy of
  // the scratch array the kernel uses
  for (const void* p : {dev_state, static_cast<const void*>(dev_out)}) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      cudaGetLastError();
      t_err = "sv_expval_static: state or output is not a CUDA pointer";
      return SV_ERR_ARG;
    }
    const bool dev_mem = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    if (!dev_mem || (pa.type == cudaMemoryTypeDevice && pa.device != dev)) {
      t_err = "sv_expval_static: state and output must be device memory of the current device";
      return SV_ERR_ARG;
    }
  }
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const uint64_t work = (1ull << n) / 256;
  const int grid = int(std::max<uint64_t>(1, std::min<uint64_t>(std::min<uint64_t>(uint64_t(sms) * 4, kMaxCtas), work)));

  // one launch per (X mask, up to 32 terms); launches run in stream order and
  // reuse the scratch one after another
  bool done[kMaxTerms] = {};
  for (size_t first = 0; first < n_terms; ++first) {
    if (done[first]) continue;
    StaticTerms a{};
    a.state = dev_state;
    a.out = dev_out;
    a.x_mask = terms[first].x_mask;
    a.n = n;
    for (size_t t = first; t < n_terms && a.nterms < kTermsPerLaunch; ++t) {
      if (done[t] || terms[t].x_mask != a.x_mask) continue;
      a.z[a.nterms] = terms[t].z_mask;
      a.k[a.nterms] = __builtin_popcountll(terms[t].x_mask & terms[t].z_mask) & 3;
      a.slot[a.nterms] = int(t);
      ++a.nterms;
      done[t] = true;
    }
    // the counter must start at zero whatever an earlier call left behind
    cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
      if (dtype == SV_C64) k_expval_static<float><<<grid, 256, 0, s>>>(a, static_cast<unsigned char*>(scratch));
      else k_expval_static<double><<<grid, 256, 0, s>>>(a, static_cast<unsigned char*>(scratch));
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
      t_err = std::string("sv_expval_static: ") + cudaGetErrorString(e);
      return SV_ERR_CUDA;
    }
  }
  return SV_OK;
}

sv_status sv_expval_static(const void* dev_state, int n, sv_dtype dtype, const sv_pauli* terms, size_t n_terms,
                           double* dev_out, void* cuda_stream) {
  return report(expval_static_impl(dev_state, n, dtype, terms, n_terms, dev_out, cuda_stream));
}

}  // extern "C"
