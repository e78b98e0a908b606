// kern_branch.cu -- shot branching: the walk that routes every shot down the
// tree of outcome paths, and the host loop that grows the tree.
//
// A path is one representative trajectory's draw record: per draw the
// unnormalised masses (p0, p1) it compared against and its outcome.  A shot
// follows a path while its own draws agree with the recorded outcomes: draw m
// of shot s takes outcome 1 iff u(seed, stream, s, m) >= p0 / (p0 + p1), the
// same expression on the same doubles as the measurement's scalar phase, so
// the decision is the one the shot's own trajectory would take.  Where it
// disagrees the shot moves to the path whose representative took the other
// outcome at that draw (a child); if that path does not exist yet the shot
// claims the draw and waits for the next round.
#include <algorithm>
#include <cstring>

#include "branch.h"
#include "dev_common.cuh"

namespace svk {

static __device__ __forceinline__ uint32_t request_of(const BranchArgs& a, uint64_t g) {
  uint32_t lo = 0, hi = a.nreq;  // req_begin[lo] <= g < req_begin[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (a.req_begin[mid] <= g) lo = mid;
    else hi = mid;
  }
  return lo;
}

__global__ void k_branch_init(const BranchArgs a) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < a.nshots;
       g += uint64_t(gridDim.x) * blockDim.x)
    a.walk[g] = uint64_t(a.req_root[request_of(a, g)]) << 32;
}

__global__ void k_branch_walk(const BranchArgs a) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < a.nshots;
       g += uint64_t(gridDim.x) * blockDim.x) {
    const uint64_t w = a.walk[g];
    if (uint32_t(w) >> 31) continue;  // reached the end of its path in an earlier round
    uint32_t j = uint32_t(w >> 32), i = uint32_t(w);
    const uint32_t r = request_of(a, g);
    const uint64_t shot = g - a.req_begin[r], stream = a.req_stream[r];
    BrPath P = a.paths[j];
    for (;;) {
      if (i >= P.len) {
        a.walk[g] = (uint64_t(j) << 32) | i | 0x80000000u;
        break;
      }
      const BrDraw d = a.draws[P.off + i];
      const double u = draw_uniform(a.seed, stream, shot, i);
      const int o = (d.p0 + d.p1 > 0) ? ((u >= d.p0 / (d.p0 + d.p1)) ? 1 : 0) : 0;
      if (o == d.outcome) {
        ++i;
        continue;
      }
      if (d.child >= 0) {  // the other outcome's path shares draws 0 .. i-1 and takes o at i
        j = uint32_t(d.child);
        P = a.paths[j];
        ++i;
        continue;
      }
      const uint32_t key = P.off + i;
      const uint32_t old = atomicCAS(a.claim + key, 0xFFFFFFFFu, uint32_t(g));
      if (old == 0xFFFFFFFFu) a.fresh[atomicAdd(a.nfresh, 1u)] = key;
      else atomicMin(a.claim + key, uint32_t(g));
      a.walk[g] = (uint64_t(j) << 32) | i;
      break;
    }
  }
}

__global__ void k_branch_gather(const BranchArgs a) {
  for (uint64_t g = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; g < a.nshots;
       g += uint64_t(gridDim.x) * blockDim.x)
    a.creg_out[g] = a.paths[uint32_t(a.walk[g] >> 32)].creg;
}

static int walk_grid(uint64_t nshots, int sms) {
  const uint64_t want = (nshots + 255) / 256;
  return int(std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(sms) * 8)));
}

cudaError_t launch_branch_init(const BranchArgs& a, int sms, cudaStream_t s) {
  k_branch_init<<<walk_grid(a.nshots, sms), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_branch_walk(const BranchArgs& a, int sms, cudaStream_t s) {
  k_branch_walk<<<walk_grid(a.nshots, sms), 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_branch_gather(const BranchArgs& a, int sms, cudaStream_t s) {
  k_branch_gather<<<walk_grid(a.nshots, sms), 256, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace svk

namespace svb {

namespace {

template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  ~DBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t reserve(size_t count) {
    count = std::max<size_t>(count, 1);
    if (count <= n) return cudaSuccess;
    const size_t want = std::max(count, 2 * n);  // grows geometrically across rounds
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, want * sizeof(T));
    if (e == cudaSuccess) n = want;
    return e;
  }
  cudaError_t upload(const std::vector<T>& v, cudaStream_t s) {
    cudaError_t e = reserve(v.size());
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  }
};

}  // namespace

struct Work {
  DBuf<svk::BrDraw> draws;
  DBuf<svk::BrPath> paths;
  DBuf<uint64_t> req_begin, req_stream, walk, creg;
  DBuf<uint32_t> req_root, claim, fresh, nfresh;
};

Work* work_new() { return new Work(); }
void work_free(Work* w) { delete w; }

#define SVB_CUDA(call)                                                  \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);         \
      return SV_ERR_CUDA;                                               \
    }                                                                   \
  } while (0)

sv_status sample(Work* w, cudaStream_t s, int sms, const std::vector<uint64_t>& req_stream,
                 const std::vector<uint64_t>& req_shots, uint64_t seed, uint64_t seed_reps, const Runner& run,
                 uint64_t* creg_out, sv_branch_stats* stats, std::string& err) {
  const uint32_t nreq = uint32_t(req_stream.size());
  std::vector<uint64_t> begin(nreq + 1, 0);
  for (uint32_t r = 0; r < nreq; ++r) begin[r + 1] = begin[r] + req_shots[r];
  const uint64_t total = begin[nreq];
  sv_branch_stats st{};
  st.shots = total;
  if (stats) *stats = st;
  if (total == 0) return SV_OK;
  if (total >= 0xFFFFFFFFull) {
    err = "shot branching takes fewer than 2^32 - 1 shots per call";
    return SV_ERR_UNSUPPORTED;
  }

  std::vector<svk::BrPath> paths;
  std::vector<svk::BrDraw> draws;
  std::vector<int64_t> root(nreq, -1);
  // Inserts a representative's record into its request's tree: it follows the
  // paths its outcomes agree with and becomes a new path where it first takes
  // an outcome no path has taken there yet (a duplicate of an existing path
  // adds nothing).  Along the shared prefix its masses must equal the tree's
  // bit for bit: equal outcomes mean equal states.
  auto insert = [&](uint32_t r, const RepOut& o) -> sv_status {
    if (o.status) {
      err = o.status == SV_ERR_NUMERIC ? "a measurement saw a zero-norm state" : "device reported an error";
      return sv_status(o.status);
    }
    if (o.m > o.draws.size() || o.m > uint64_t(svp::MAX_TRACE)) {
      err = "a trajectory executed more draws than shot branching records (" + std::to_string(svp::MAX_TRACE) + ")";
      return SV_ERR_UNSUPPORTED;
    }
    if (draws.size() + o.m >= 0xFFFFFFFFull) {
      err = "shot branching tree too large";
      return SV_ERR_UNSUPPORTED;
    }
    int32_t* link = nullptr;  // where the new path hangs (nullptr: it becomes the root)
    if (root[r] >= 0) {
      uint32_t j = uint32_t(root[r]);
      for (uint64_t i = 0;; ++i) {
        const svk::BrPath& P = paths[j];
        if (i == P.len || i == o.m) {
          if (i == P.len && i == o.m && P.creg == o.creg) return SV_OK;  // a path already in the tree
          err = "a representative trajectory did not replay its path (non-deterministic program)";
          return SV_ERR_UNSUPPORTED;
        }
        svk::BrDraw& d = draws[P.off + i];
        const svk::BrDraw& y = o.draws[i];
        if (std::memcmp(&d.p0, &y.p0, sizeof(double)) != 0 || std::memcmp(&d.p1, &y.p1, sizeof(double)) != 0) {
          err = "a representative trajectory did not replay its path (non-deterministic program)";
          return SV_ERR_UNSUPPORTED;
        }
        if (y.outcome == d.outcome) continue;
        if (d.child < 0) {
          link = &d.child;
          break;
        }
        j = uint32_t(d.child);
      }
    }
    const uint32_t id = uint32_t(paths.size());
    if (link) *link = int32_t(id);
    else root[r] = id;
    svk::BrPath P;
    P.off = uint32_t(draws.size());
    P.len = uint32_t(o.m);
    P.creg = o.creg;
    for (uint64_t k = 0; k < o.m; ++k) {
      svk::BrDraw d = o.draws[k];
      d.child = -1;
      draws.push_back(d);
    }
    paths.push_back(P);
    st.max_draws = std::max<uint64_t>(st.max_draws, o.m);
    return SV_OK;
  };
  auto run_insert = [&](const std::vector<RepReq>& reps) -> sv_status {
    std::vector<RepOut> outs;
    sv_status rs = run(reps, outs, err);
    if (rs != SV_OK) return rs;
    if (outs.size() != reps.size()) {
      err = "runner returned the wrong number of records";
      return SV_ERR_ARG;
    }
    for (size_t k = 0; k < reps.size(); ++k) {
      rs = insert(reps[k].req, outs[k]);
      if (rs != SV_OK) return rs;
    }
    return SV_OK;
  };

  // round 0: the first shots of every request, about seed_reps in all (at
  // least one per request); on an engine that runs them side by side they
  // find most paths at once
  std::vector<RepReq> reps;
  for (uint32_t r = 0; r < nreq; ++r) {
    if (!req_shots[r]) continue;
    const uint64_t k = std::min<uint64_t>(req_shots[r], std::max<uint64_t>(1, seed_reps * req_shots[r] / total));
    for (uint64_t q = 0; q < k; ++q) reps.push_back(RepReq{r, q});
  }
  sv_status rs = run_insert(reps);
  if (rs != SV_OK) return rs;
  std::vector<uint32_t> root32(nreq, 0);
  for (uint32_t r = 0; r < nreq; ++r) root32[r] = root[r] < 0 ? 0u : uint32_t(root[r]);

  SVB_CUDA(w->req_begin.upload(begin, s));
  SVB_CUDA(w->req_stream.upload(req_stream, s));
  SVB_CUDA(w->req_root.upload(root32, s));
  SVB_CUDA(w->walk.reserve(total));
  SVB_CUDA(w->nfresh.reserve(1));
  svk::BranchArgs a{};
  a.req_begin = w->req_begin.p;
  a.req_stream = w->req_stream.p;
  a.req_root = w->req_root.p;
  a.nreq = nreq;
  a.seed = seed;
  a.nshots = total;
  a.walk = w->walk.p;
  a.nfresh = w->nfresh.p;
  SVB_CUDA(svk::launch_branch_init(a, sms, s));

  std::vector<uint32_t> fresh, claim;
  for (;;) {
    SVB_CUDA(w->draws.upload(draws, s));
    SVB_CUDA(w->paths.upload(paths, s));
    SVB_CUDA(w->claim.reserve(draws.size()));
    SVB_CUDA(w->fresh.reserve(draws.size()));
    SVB_CUDA(cudaMemsetAsync(w->claim.p, 0xFF, std::max<size_t>(draws.size(), 1) * sizeof(uint32_t), s));
    SVB_CUDA(cudaMemsetAsync(w->nfresh.p, 0, sizeof(uint32_t), s));
    a.draws = w->draws.p;
    a.paths = w->paths.p;
    a.claim = w->claim.p;
    a.fresh = w->fresh.p;
    SVB_CUDA(svk::launch_branch_walk(a, sms, s));
    ++st.levels;
    // one round trip: the count, and the claim lists at their largest possible size
    uint32_t nf = 0;
    fresh.resize(draws.size());
    claim.resize(draws.size());
    SVB_CUDA(cudaMemcpyAsync(&nf, w->nfresh.p, sizeof(nf), cudaMemcpyDeviceToHost, s));
    if (!draws.empty()) {
      SVB_CUDA(cudaMemcpyAsync(fresh.data(), w->fresh.p, draws.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
      SVB_CUDA(cudaMemcpyAsync(claim.data(), w->claim.p, draws.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    }
    SVB_CUDA(cudaStreamSynchronize(s));
    if (nf == 0) break;
    fresh.resize(nf);
    std::sort(fresh.begin(), fresh.end());
    // one representative per claimed draw: the smallest shot that left the tree there
    reps.clear();
    for (uint32_t key : fresh) {
      const uint64_t g = claim[key];
      const uint32_t r = uint32_t(std::upper_bound(begin.begin(), begin.end(), g) - begin.begin()) - 1;
      reps.push_back(RepReq{r, g - begin[r]});
    }
    const size_t before = paths.size();
    rs = run_insert(reps);
    if (rs != SV_OK) return rs;
    if (paths.size() == before) {  // every claimed draw must gain its path, or the walk would repeat itself
      err = "shot branching made no progress (non-deterministic program)";
      return SV_ERR_UNSUPPORTED;
    }
  }
  SVB_CUDA(w->creg.reserve(total));
  a.creg_out = w->creg.p;
  SVB_CUDA(svk::launch_branch_gather(a, sms, s));
  SVB_CUDA(cudaMemcpyAsync(creg_out, w->creg.p, total * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  SVB_CUDA(cudaStreamSynchronize(s));
  st.paths = paths.size();
  if (stats) *stats = st;
  return SV_OK;
}

}  // namespace svb
