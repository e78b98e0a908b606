// kern_measure.cu -- terminal sampling and Pauli-sum expectation values.
//
// Sampling (shots, Sec. IV-C): shot s draws u for (seed, stream, s, 2^32)
// and takes the smallest index i whose FP64 CDF exceeds u * total.  The CDF
// is held at two levels, built in one read of the state: the state is cut
// into runs of 32 amplitudes and blocks of 256 runs; k_cdf_runs sums each
// run's |amp|^2 in index order (FP64) and stores, per run, the inclusive
// prefix of run sums within its block; k_scan_blocks scans the block totals.
// A shot then binary-searches the block prefixes, binary-searches the run
// prefixes of its block, and walks the 32 amplitudes of one run.
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

constexpr int RUN_BITS = 5;                 // 32 amplitudes per run
constexpr int RUNS_PER_BLOCK_BITS = 8;      // 256 runs per block (one CTA of 256 threads)
constexpr int SAMPLE_BLOCK_BITS = RUN_BITS + RUNS_PER_BLOCK_BITS;

// blocks of the two-level CDF (states of fewer than 2^13 amplitudes: one block
// of 2^(n - 5) runs)
uint64_t sample_blocks(int n) { return n > SAMPLE_BLOCK_BITS ? (1ull << (n - SAMPLE_BLOCK_BITS)) : 1ull; }
uint64_t sample_runs(int n) { return n > RUN_BITS ? (1ull << (n - RUN_BITS)) : 1ull; }

template <typename T>
__device__ __forceinline__ double abs2d(typename CxT<T>::V v) {
  return fma(double(v.x), double(v.x), double(v.y) * double(v.y));
}

// double-float helpers (an unevaluated sum hi + lo of FP32 values; Knuth's
// error-free sum, the FMA error-free product)
struct DFv {
  float hi, lo;
};
__device__ __forceinline__ DFv dfv_add(DFv a, DFv b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  const float lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, lo);
  return DFv{h, __fsub_rn(lo, __fsub_rn(h, s))};
}
__device__ __forceinline__ DFv dfv_abs2(float x, float y) {
  const float p = __fmul_rn(x, x), q = __fmul_rn(y, y);
  return dfv_add(DFv{p, __fmaf_rn(x, x, -p)}, DFv{q, __fmaf_rn(y, y, -q)});
}

// One CTA per block, one warp per 32 runs (1,024 amplitudes), loaded
// coalesced: at step k, complex64 lane l holds amplitudes 64k + 2l, +1 (run
// 2k + l/16), complex128 lane l holds amplitude 32k + l (run k).  A run's sum
// is a reduction over its lanes (|amp|^2 in FP64, each lane's own pair in
// index order, then a fixed butterfly), handed to lane (run mod 32); then the
// inclusive prefix of the block's run sums (warp scans, warp totals in a
// fixed order) and the block total.  runs_in_block: 2^(block bits) / 32.
template <typename T>
__global__ void __launch_bounds__(256) k_cdf_runs(SampleArgs a, int runs_in_block) {
  __shared__ double wsum[8];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t b = blockIdx.x;
  const int r_local = warp * 32 + lane;  // the run this lane ends up holding
  const bool live = r_local < runs_in_block;
  const uint64_t a0 = (b * uint64_t(runs_in_block) + uint64_t(warp) * 32u) << RUN_BITS;  // warp's first amplitude
  const int wruns = runs_in_block - warp * 32 < 32 ? runs_in_block - warp * 32 : 32;  // runs of this warp
  double mine = 0.0;
  if constexpr (sizeof(T) == 4) {
    // complex64: each warp stages 512 amplitudes (16 runs) at a time in
    // shared memory (coalesced 16-byte loads; one pad granule per 8 keeps the
    // writes and the per-run reads free of bank conflicts), each lane sums
    // half a run in index order as a double-float value (error-free FP32
    // products and sums, ~44 bits; FP64 arithmetic per amplitude would bound
    // this read at GB300's FP64 rate), one shuffle joins the halves
    __shared__ float4 stage[8][288];
    float4* sw = stage[warp];
    const float4* s = reinterpret_cast<const float4*>(a.state) + (a0 >> 1);
    double got[2] = {0.0, 0.0};
    for (int it = 0; it < 2 && it * 16 < wruns; ++it) {
      float4 q[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) q[k] = __ldcs(s + it * 256 + k * 32 + lane);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int f = k * 32 + lane;
        sw[f + (f >> 3)] = q[k];
      }
      __syncwarp();
      const int f0 = 8 * lane;  // run lane/2, half lane&1: granules 16 run + 8 half + j
      DFv v{0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int f = f0 + j;
        const float4 w = sw[f + (f >> 3)];
        v = dfv_add(v, dfv_abs2(w.x, w.y));
        v = dfv_add(v, dfv_abs2(w.z, w.w));
      }
      __syncwarp();
      const DFv o{__shfl_xor_sync(0xffffffffu, v.hi, 1), __shfl_xor_sync(0xffffffffu, v.lo, 1)};
      v = (lane & 1) ? dfv_add(o, v) : dfv_add(v, o);  // first half first, in both lanes
      got[it] = double(v.hi) + double(v.lo);
    }
    // lane j takes run j of the warp: runs 0..15 from iteration 0 (lane 2j), 16..31 from iteration 1
    const double r0 = __shfl_sync(0xffffffffu, got[0], (2 * lane) & 31);
    const double r1 = __shfl_sync(0xffffffffu, got[1], (2 * lane) & 31);
    mine = lane < 16 ? r0 : r1;
  } else {
    const double2* s = reinterpret_cast<const double2*>(a.state) + a0;
    for (int k = 0; k < wruns; ++k) {
      double v = abs2d<T>(__ldcs(s + 32 * k + lane));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == k) mine = v;
    }
  }
  double v = live ? mine : 0.0;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {  // inclusive warp scan
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  double off = 0;
  for (int w = 0; w < warp; ++w) off += wsum[w];
  v += off;
  const uint64_t r = b * uint64_t(runs_in_block) + uint64_t(r_local);
  if (live) a.run_cum[r] = v;
  if (r_local == runs_in_block - 1) a.block_sums[b] = v;
}

// exclusive scan of nb block sums by one CTA (chunk sums per thread, chunk
// bases by a block-wide scan in a fixed order).  At chunk boundaries block_prefix[i + 1] may differ
// from block_prefix[i] + block_sums[i] by rounding; the shot walk then falls
// back to the last nonzero amplitude of the block (a draw within an ulp of a
// boundary).
__global__ void __launch_bounds__(1024) k_scan_blocks(SampleArgs a, uint64_t nb) {
  __shared__ double wtot[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t per = (nb + 1023) / 1024;
  const uint64_t lo = tid * per, hi = lo + per < nb ? lo + per : nb;
  double s = 0;
#pragma unroll 8
  for (uint64_t i = lo; i < hi; ++i) s += a.block_sums[i];
  // exclusive scan of the 1,024 chunk sums: warp scans, then the warp totals
  double v = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) wtot[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = wtot[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    wtot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  double run = (warp > 0 ? wtot[warp - 1] : 0.0) + (v - s);
  if (tid == 1023) a.block_prefix[nb] = wtot[31];
  for (uint64_t i = lo; i < hi; ++i) {
    a.block_prefix[i] = run;
    run += a.block_sums[i];
  }
}

// One thread per shot.
template <typename T>
__global__ void __launch_bounds__(256) k_sample_search(SampleArgs a, uint64_t nb, int runs_in_block) {
  using V = typename CxT<T>::V;
  const V* st = reinterpret_cast<const V*>(a.state);
  const uint64_t shot = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
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
  const uint64_t b = lo;
  const double base = a.block_prefix[b];
  const double* rc = a.run_cum + b * uint64_t(runs_in_block);
  // smallest run r with base + rc[r] > target (non-decreasing in r)
  int rl = 0, rh = runs_in_block - 1;
  while (rl < rh) {
    const int mid = (rl + rh) >> 1;
    if (base + rc[mid] > target) rh = mid;
    else rl = mid + 1;
  }
  // walk the run; its amplitudes were summed in another order for the run
  // sums, so a target within rounding of the run's end may find no crossing
  // here (handled below)
  uint64_t found = ~0ull;
  for (int r = rl; r >= 0 && found == ~0ull; --r) {
    const uint64_t i0 = (b * uint64_t(runs_in_block) + uint64_t(r)) << RUN_BITS;
    // the target relative to the run's start; complex64 accumulates the run in
    // FP32 from there (its relative error, ~1e-7 of one run's mass, only moves
    // draws that fall within it of an amplitude boundary)
    const double rel = target - (base + (r > 0 ? rc[r - 1] : 0.0));
    using Acc = T;
    const Acc trel = Acc(rel);
    Acc c = Acc(0);
    uint64_t last_nz = ~0ull;
    for (int j = 0; j < 32; ++j) {
      const typename CxT<T>::V v = st[i0 + j];
      const Acc p = fma(v.x, v.x, v.y * v.y);
      c += p;
      if (p > 0) last_nz = i0 + j;
      if (p > 0 && c > trel && r == rl) {
        found = i0 + j;
        break;
      }
    }
    // rounding at a run boundary (the target within an ulp of it), or a run
    // of zeros: the last amplitude with nonzero probability at or before it
    if (found == ~0ull && last_nz != ~0ull) found = last_nz;
  }
  a.out[shot] = found != ~0ull ? found : (b << (RUN_BITS + RUNS_PER_BLOCK_BITS));
}

template <typename T>
static cudaError_t launch_sample_t(const SampleArgs& a, int sms, cudaStream_t s) {
  const uint64_t nb = sample_blocks(a.n);
  const int runs_in_block = int((a.n > SAMPLE_BLOCK_BITS ? (1ull << SAMPLE_BLOCK_BITS) : (1ull << a.n)) >> RUN_BITS);
  k_cdf_runs<T><<<unsigned(nb), 256, 0, s>>>(a, runs_in_block);
  k_scan_blocks<<<1, 1024, 0, s>>>(a, nb);
  if (a.shots) {
    const uint64_t blocks = (a.shots + 255) / 256;
    k_sample_search<T><<<unsigned(blocks), 256, 0, s>>>(a, nb, runs_in_block);
  }
  (void)sms;
  return cudaGetLastError();
}

cudaError_t launch_sample(int dtype, const SampleArgs& a, int sms, cudaStream_t s) {
  return dtype == SV_C64 ? launch_sample_t<float>(a, sms, s) : launch_sample_t<double>(a, sms, s);
}

// ---------------------------------------------------------------------- expectation values
constexpr int EXP_TERMS = EXPVAL_TERMS;  // terms per launch (a larger X group takes several launches)
constexpr int EXP_CHUNK = 8;   // warp blocks (128 pairs each) summed in the state precision before the accumulator

// Per-term accumulators of the expectation kernel: complex64 chunk sums go
// into a double-float (on the FP32 pipes; a conversion and an FP64 add per
// term per chunk would bind the kernel to GB300's FP64 rate), complex128 into
// FP64.
template <typename T> struct ExpAcc;
template <> struct ExpAcc<float> {
  DFv v{0.f, 0.f};
  __device__ __forceinline__ void add(float x) { v = dfv_add(v, DFv{x, 0.f}); }
  __device__ __forceinline__ double get() const { return double(v.hi) + double(v.lo); }
};
template <> struct ExpAcc<double> {
  double v = 0.0;
  __device__ __forceinline__ void add(double x) { v += x; }
  __device__ __forceinline__ double get() const { return v; }
};

// One X group (x) per launch, up to 16 of its terms.  The pair index r runs
// over the 2^n / 2 pairs (i, i ^ x) with bit h = top bit of x clear in i (for
// x = 0 over the 2^n amplitudes, f = |psi_i|^2); f(r) = conj(psi_i) psi_{i^x}.
// A warp block is 128 consecutive r: lane l holds r = 128 w + 32 u + l for
// u = 0..3 (each of the four loads coalesced).  A 128-point Walsh-Hadamard
// transform (two butterfly stages over u in registers, five over the lanes by
// shuffles) gives F(p) = sum_r' (-1)^{|p & r'|} f(r') at p = l + 32 u, which
// the warp writes to its slice of shared memory (Re F at p, Im F at 128 + p);
// a term whose Z mask restricted to the block's index bits is zl then reads
// F(zl) (its real or imaginary part, by the phase i^k of the term) with one
// warp-uniform (broadcast) load and adds it with the sign (-1)^{|i0 & zh|} of
// the rest (i0: the block's first index; zh has no bits below 7, so the sign
// is taken on i0 >> 7 and zh >> 7 in 32 bits).  Every lane does the same
// per-term work, so lane 0's sums are the warp's.  NT: the smallest power of
// two >= the term count (chunk sums in the state precision, ExpAcc beyond).
template <typename T, int NT>
__global__ void __launch_bounds__(256, 2) k_expval_group(const ExpvalArgs a) {
  using V = typename CxT<T>::V;
  const V* st = reinterpret_cast<const V*>(a.state);
  __shared__ double red[8][NT];
  __shared__ T wf[8][2][128];  // per warp: Re F, Im F of the current block
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nt = a.nterms;
  const uint64_t x = a.x_mask;
  const int h = x ? 63 - __clzll((long long)x) : 64;
  ExpAcc<T> acc[NT];
  T part[NT];
#pragma unroll
  for (int t = 0; t < NT; ++t) part[t] = 0;
  const uint64_t N = 1ull << a.n;
  const uint64_t npairs = x ? (N >> 1) : N;  // a multiple of 128: states have >= 2^10 amplitudes
  const uint64_t lowm = h < 64 ? ((1ull << h) - 1) : ~0ull;
  auto ins = [&](uint64_t r) -> uint64_t { return x ? (((r >> h) << (h + 1)) | (r & lowm)) : r; };
  // offsets of lane l, register u from the block's first index (the insertion of a zero at bit h
  // is linear on disjoint bits, so i(r0 + d) = i(r0) + i(d) for d < 128 and r0 a multiple of 128)
  uint64_t off[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) off[u] = ins(uint64_t(32 * u + lane));
  T* const fre = wf[warp][0];
  T* const fim = wf[warp][1];  // = fre + 128
  const uint64_t warps = uint64_t(gridDim.x) * (blockDim.x >> 5);
  int cnt = 0;
  for (uint64_t wb = uint64_t(blockIdx.x) * (blockDim.x >> 5) + uint64_t(warp); (wb << 7) < npairs; wb += warps) {
    const uint64_t i0 = ins(wb << 7);
    T fr[4], fi[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint64_t i = i0 + off[u];
      const V p = st[i];
      if (x) {
        const V q = st[i ^ x];
        fr[u] = fma(p.x, q.x, p.y * q.y);   // Re conj(psi_i) psi_j
        fi[u] = fma(p.x, q.y, -p.y * q.x);  // Im
      } else {
        fr[u] = fma(p.x, p.x, p.y * p.y);
        fi[u] = T(0);
      }
    }
    // Walsh-Hadamard over u (registers), then over the lanes
#pragma unroll
    for (int o = 1; o < 4; o <<= 1)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (!(u & o)) {
          const T ar = fr[u], br = fr[u | o], ai = fi[u], bi = fi[u | o];
          fr[u] = ar + br;
          fr[u | o] = ar - br;
          fi[u] = ai + bi;
          fi[u | o] = ai - bi;
        }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const bool up = lane & o;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T qr = __shfl_xor_sync(0xffffffffu, fr[u], o);
        fr[u] = up ? qr - fr[u] : fr[u] + qr;
        if (x) {
          const T qi = __shfl_xor_sync(0xffffffffu, fi[u], o);
          fi[u] = up ? qi - fi[u] : fi[u] + qi;
        }
      }
    }
    __syncwarp();  // the previous block's reads are done
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      fre[32 * u + lane] = fr[u];
      if (x) fim[32 * u + lane] = fi[u];
    }
    __syncwarp();
    const uint32_t i7 = uint32_t(i0 >> 7);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const uint32_t w = a.zw[t];  // parameter block: warp-uniform operands
      const T c = fre[w & 0xFFu];
      const uint32_t sg = (uint32_t(__popc(i7 & a.zh7[t])) ^ (w >> 8)) & 1u;
      part[t] += sg ? -c : c;
    }
    if (++cnt == EXP_CHUNK) {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        acc[t].add(part[t]);
        part[t] = 0;
      }
      cnt = 0;
    }
  }
  // a pair contributes twice its value (the pair (i^x, i) is not visited)
  const double pw = x == 0 ? 1.0 : 2.0;
  if (lane == 0)
#pragma unroll
    for (int t = 0; t < NT; ++t) red[warp][t] = pw * (acc[t].get() + double(part[t]));
  __syncthreads();
  if (tid < NT) {  // block reduction (fixed order)
    double sum = 0;
    for (int w = 0; w < 8; ++w) sum += red[w][tid];
    a.partials[blockIdx.x * EXP_TERMS + tid] = sum;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (tid < nt) {
    double sum = 0;
    for (unsigned b2 = 0; b2 < gridDim.x; ++b2) sum += __ldcg(a.partials + b2 * EXP_TERMS + tid);
    a.out[tid] = sum;
  }
  if (tid == 0) *a.ticket = 0;
}

template <typename T>
static cudaError_t launch_expval_t(const ExpvalArgs& a, int grid, cudaStream_t s) {
  const int nt = a.nterms;
  if (nt <= 1) k_expval_group<T, 1><<<grid, 256, 0, s>>>(a);
  else if (nt <= 2) k_expval_group<T, 2><<<grid, 256, 0, s>>>(a);
  else if (nt <= 4) k_expval_group<T, 4><<<grid, 256, 0, s>>>(a);
  else if (nt <= 8) k_expval_group<T, 8><<<grid, 256, 0, s>>>(a);
  else k_expval_group<T, 16><<<grid, 256, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_expval_group(int dtype, const ExpvalArgs& a, int grid, cudaStream_t s) {
  if (a.nterms > EXP_TERMS) return cudaErrorInvalidValue;
  return dtype == SV_C64 ? launch_expval_t<float>(a, grid, s) : launch_expval_t<double>(a, grid, s);
}

}  // namespace svk
