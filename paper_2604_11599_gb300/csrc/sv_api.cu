// sv_api.cu -- the C-ABI of libsv (include/sv.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/sv.h"
#include "jit.h"
#include "branch.h"
#include "kernels.h"
#include "planner.h"

using svp::Ctrl;
using svp::DTrace;

namespace {

thread_local std::string g_err;

sv_status fail(sv_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

sv_status cuda_fail(cudaError_t e, const char* where) {
  return fail(SV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define SV_CUDA(call)                                  \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
  cudaError_t reserve(size_t count) {
    if (count <= n && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T));
    if (e == cudaSuccess) n = std::max<size_t>(count, 1);
    return e;
  }
  template <typename U>
  cudaError_t upload(const std::vector<U>& v, cudaStream_t s) {
    const size_t bytes = v.size() * sizeof(U);
    cudaError_t e = reserve((bytes + sizeof(T) - 1) / sizeof(T));
    if (e != cudaSuccess || bytes == 0) return e;
    return cudaMemcpyAsync(p, v.data(), bytes, cudaMemcpyHostToDevice, s);
  }
};

uint64_t fnv1a(const void* data, size_t len, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < len; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

}  // namespace

namespace svapi {
// lets other translation units report through sv_last_error()
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace svapi

struct sv_program {
  sv_state* owner = nullptr;
  svp::Plan plan;
  DevBuf<svp::DPass> passes;
  DevBuf<svp::DGate> gates;
  DevBuf<svp::DStage> stages;
  DevBuf<svp::DScalar> scalars;
  DevBuf<svp::DScalar> init;
  DevBuf<svp::DJob> jobs;
  DevBuf<double> consts;
  DevBuf<unsigned char> mats;
  DevBuf<uint8_t> flags;
  bool cached = false;  // owned by the state's cache
  std::shared_ptr<svj::JitModule> jit;  // specialised pass kernels (sv_set_jit)
  bool jit_tried = false;
};

struct sv_state {
  int n = 0, n_int = 0;
  sv_dtype dtype = SV_C64;
  size_t amp_bytes = 8;
  void* state = nullptr;
  bool owns_state = false;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  Ctrl* ctrl = nullptr;
  DTrace* trace = nullptr;
  DevBuf<double> partials;
  DevBuf<double> params;
  DevBuf<double> sample_buf;
  DevBuf<uint64_t> sample_out;
  DevBuf<double> exp_partials;
  DevBuf<double> exp_out;
  unsigned* exp_ticket = nullptr;
  std::vector<double> dense;  // host copy for planning
  uint64_t dense_hash = 0;
  svp::Tuning tune;
  std::unordered_map<uint64_t, std::unique_ptr<sv_program>> cache;
  std::unordered_set<sv_program*> prepared;  // programs handed out by sv_prepare, not yet freed
  // pass timing
  bool profiling = false;
  std::vector<cudaEvent_t> events;
  size_t ev_used = 0;
  unsigned long long* work = nullptr;  // device work counters of the profiled launches (svk::PassArgs::work)
  bool use_cache = true;
  bool use_jit = false;
  bool dense_tc = true;  // dense four-qubit gates on the tensor cores where the kernel supports it
  std::unique_ptr<svb::Work, void (*)(svb::Work*)> branch{nullptr, svb::work_free};  // shot-branching scratch
};

namespace {

sv_status upload_plan(cudaStream_t s, size_t amp_bytes, sv_program* p) {
  const svp::Plan& P = p->plan;
  SV_CUDA(p->passes.upload(P.passes, s));
  SV_CUDA(p->gates.upload(P.gates, s));
  SV_CUDA(p->stages.upload(P.stages, s));
  SV_CUDA(p->scalars.upload(P.scalars, s));
  SV_CUDA(p->init.upload(P.init_items, s));
  SV_CUDA(p->jobs.upload(P.jobs, s));
  SV_CUDA(p->consts.upload(P.consts, s));
  SV_CUDA(p->mats.reserve(size_t(std::max<uint32_t>(P.n_mat, 1)) * amp_bytes));
  SV_CUDA(p->flags.reserve(std::max<uint32_t>(P.n_flags, 1)));
  SV_CUDA(cudaMemsetAsync(p->flags.p, 0, std::max<uint32_t>(P.n_flags, 1), s));
  // the host copies above read pageable vectors; finish them before the plan can change
  SV_CUDA(cudaStreamSynchronize(s));
  return SV_OK;
}

sv_status upload_program(sv_state* h, sv_program* p) { return upload_plan(h->stream, h->amp_bytes, p); }

int pass_grid(sv_state* h, int m) {
  int per_sm = 1;
  if (svk::pass_occupancy(h->dtype, m, &per_sm) != cudaSuccess) {
    cudaGetLastError();  // clear the non-sticky error of the failed query
    return -1;
  }
  const uint64_t tiles = 1ull << (h->n_int - m);
  const uint64_t want = uint64_t(h->sms) * uint64_t(per_sm);
  return int(std::min<uint64_t>(tiles, want));
}

sv_status launch_program(sv_state* h, sv_program* p, const double* dev_params, size_t n_params, uint64_t seed,
                         uint64_t stream_id, uint64_t shot) {
  const svp::Plan& P = p->plan;
  if (n_params < P.n_params_needed)
    return fail(SV_ERR_ARG, "program references " + std::to_string(P.n_params_needed) + " parameters, got " +
                                std::to_string(n_params));
  if (P.n_params_needed && !dev_params) return fail(SV_ERR_ARG, "params is NULL");
  cudaStream_t s = h->stream;
  SV_CUDA(cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), s));
  svk::PrepArgs pa{};
  pa.jobs = p->jobs.p;
  pa.njobs = int(P.jobs.size());
  pa.params = dev_params;
  pa.n_params = n_params;
  pa.consts = p->consts.p;
  pa.mats = p->mats.p;
  pa.ctrl = h->ctrl;
  pa.init = p->init.p;
  pa.ninit = int(P.init_items.size());
  pa.flags = p->flags.p;
  pa.seed = seed;
  pa.stream = stream_id;
  pa.shot = shot;
  SV_CUDA(svk::launch_prep(h->dtype, pa, s));
  if (!P.gen_init) SV_CUDA(svk::launch_init_state(h->dtype, h->state, 1ull << h->n_int, h->sms, s));
  if (h->use_jit && !p->jit_tried) {
    p->jit_tried = true;
    std::string err;
    if (svj::compile(P, p->jit, err) != SV_OK) p->jit.reset();  // generic kernels remain
  }
  const svj::JitModule* jm = h->use_jit ? p->jit.get() : nullptr;
  if (!P.passes.empty()) {
    int grid = pass_grid(h, P.m);
    if (jm && P.jit_min_blocks > 0)  // specialised kernels compiled for that many CTAs per SM
      grid = int(std::min<uint64_t>(1ull << (h->n_int - P.m), uint64_t(h->sms) * uint64_t(P.jit_min_blocks)));
    if (grid < 1) return fail(SV_ERR_CUDA, "pass kernel configuration failed for tile bits " + std::to_string(P.m));
    SV_CUDA(h->partials.reserve(size_t(grid) * 16));
    svk::PassArgs a{};
    a.state = h->state;
    a.passes = p->passes.p;
    a.gates = p->gates.p;
    a.stages = p->stages.p;
    a.scalars = p->scalars.p;
    a.mats = p->mats.p;
    a.flags = p->flags.p;
    a.ctrl = h->ctrl;
    a.trace = h->trace;
    a.partials = h->partials.p;
    a.n = h->n_int;
    a.dense_tc = h->dense_tc ? 1 : 0;
    a.work = h->profiling ? h->work : nullptr;
    for (size_t i = 0; i < P.passes.size(); ++i) {
      a.gen_init = (P.gen_init && i == 0) ? 1 : 0;
      if (h->profiling) {
        while (h->events.size() < h->ev_used + 2) {
          cudaEvent_t e;
          SV_CUDA(cudaEventCreate(&e));
          h->events.push_back(e);
        }
        SV_CUDA(cudaEventRecord(h->events[h->ev_used], s));
      }
      if (jm) {
        std::string err;
        const sv_status st = svj::launch(*jm, int(i), a, grid, s, err);
        if (st != SV_OK) return fail(st, err);
      } else {
        SV_CUDA(svk::launch_pass(h->dtype, a, int(i), grid, P.m, s, P.passes[i].dense != 0, P.passes[i].proj != 0));
      }
      if (h->profiling) {
        SV_CUDA(cudaEventRecord(h->events[h->ev_used + 1], s));
        h->ev_used += 2;
      }
    }
  }
  return SV_OK;
}

sv_status check_status(sv_state* h) {
  int32_t st = 0;
  cudaError_t e = cudaMemcpyAsync(&st, &h->ctrl->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  if (st == SV_ERR_NUMERIC) return fail(SV_ERR_NUMERIC, "a measurement saw a zero-norm state");
  if (st != 0) return fail(sv_status(st), "device reported an error");
  return SV_OK;
}

sv_status get_program(sv_state* h, const sv_op* ops, size_t n_ops, sv_program** out) {
  uint64_t key = fnv1a(ops, n_ops * sizeof(sv_op));
  key = fnv1a(&h->dense_hash, sizeof(h->dense_hash), key);
  key = fnv1a(&h->tune, sizeof(h->tune), key);
  auto it = h->cache.find(key);
  if (it != h->cache.end() && !h->use_cache) {
    cudaStreamSynchronize(h->stream);
    h->cache.erase(it);
    it = h->cache.end();
  }
  if (it != h->cache.end()) {
    *out = it->second.get();
    return SV_OK;
  }
  std::unique_ptr<sv_program> p(new sv_program());
  p->owner = h;
  std::string err;
  sv_status st = svp::build_plan(h->n, h->dtype, ops, n_ops, h->dense.empty() ? nullptr : h->dense.data(),
                                 h->dense.size() / 2, h->tune, p->plan, err);
  if (st != SV_OK) return fail(st, err);
  st = upload_program(h, p.get());
  if (st != SV_OK) return st;
  p->cached = true;
  if (h->cache.size() > 256) h->cache.clear();
  *out = p.get();
  h->cache[key] = std::move(p);
  return SV_OK;
}

bool has_draws(const sv_op* ops, size_t n_ops) {
  for (size_t i = 0; i < n_ops; ++i)
    if (ops[i].kind == SV_MEASURE || ops[i].kind == SV_RESET) return true;
  return false;
}

sv_status sample_current(sv_state* h, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                         uint64_t* dev_out) {
  const uint64_t nb = svk::sample_blocks(h->n_int), nr = svk::sample_runs(h->n_int);
  SV_CUDA(h->sample_buf.reserve(nr + 2 * nb + 1));
  svk::SampleArgs a{};
  a.state = h->state;
  a.n = h->n_int;
  a.n_logical = h->n;
  a.run_cum = h->sample_buf.p;
  a.block_sums = h->sample_buf.p + nr;
  a.block_prefix = h->sample_buf.p + nr + nb;
  a.shots = shots;
  a.seed = seed;
  a.stream = stream_id;
  a.shot0 = shot0;
  a.out = dev_out;
  SV_CUDA(svk::launch_sample(h->dtype, a, h->sms, h->stream));
  return SV_OK;
}

}  // namespace

extern "C" {

const char* sv_last_error(void) { return g_err.c_str(); }

const char* sv_version(void) { return "libsv 0.1 (sm_103a)"; }

sv_status sv_create(int n, sv_dtype dtype, void* dev_buf, size_t bytes, sv_state** out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > 34) return fail(SV_ERR_ARG, "n must be in 1..34");
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  std::unique_ptr<sv_state> h(new sv_state());
  h->n = n;
  h->n_int = std::max(n, 10);  // small states are padded with qubits that stay |0>
  h->dtype = dtype;
  h->amp_bytes = dtype == SV_C64 ? 8 : 16;
  const size_t need = (size_t(1) << h->n_int) * h->amp_bytes;
  SV_CUDA(cudaGetDevice(&h->device));
  SV_CUDA(cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device));
  if (dev_buf) {
    if (bytes < need) return fail(SV_ERR_ARG, "dev_buf smaller than 2^max(n,10) amplitudes");
    if (reinterpret_cast<uintptr_t>(dev_buf) % 16) return fail(SV_ERR_ARG, "dev_buf must be 16-byte aligned");
    h->state = dev_buf;
  } else {
    cudaError_t e = cudaMalloc(&h->state, need);
    if (e != cudaSuccess) return fail(SV_ERR_OOM, std::string("state allocation: ") + cudaGetErrorString(e));
    h->owns_state = true;
  }
  if (cudaMalloc(&h->ctrl, sizeof(Ctrl)) != cudaSuccess ||
      cudaMalloc(&h->trace, sizeof(DTrace) * svp::MAX_TRACE) != cudaSuccess ||
      cudaMalloc(&h->exp_ticket, sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&h->work, sizeof(unsigned long long) * SV_WORK_COUNTERS) != cudaSuccess) {
    if (h->owns_state) cudaFree(h->state);
    return fail(SV_ERR_OOM, "control block allocation");
  }
  SV_CUDA(cudaMemset(h->ctrl, 0, sizeof(Ctrl)));
  SV_CUDA(cudaMemset(h->exp_ticket, 0, sizeof(unsigned)));
  SV_CUDA(cudaMemset(h->work, 0, sizeof(unsigned long long) * SV_WORK_COUNTERS));
  SV_CUDA(svk::launch_init_state(h->dtype, h->state, 1ull << h->n_int, h->sms, nullptr));
  SV_CUDA(cudaDeviceSynchronize());
  *out = h.release();
  return SV_OK;
}

sv_status sv_destroy(sv_state* h) {
  if (!h) return SV_OK;
  cudaStreamSynchronize(h->stream);
  h->cache.clear();
  // programs prepared for this state stay valid for sv_program_free only
  for (sv_program* p : h->prepared) p->owner = nullptr;
  h->prepared.clear();
  if (h->owns_state && h->state) cudaFree(h->state);
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->trace) cudaFree(h->trace);
  if (h->exp_ticket) cudaFree(h->exp_ticket);
  if (h->work) cudaFree(h->work);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  delete h;
  return SV_OK;
}

sv_status sv_bind_stream(sv_state* h, void* cuda_stream) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  h->stream = static_cast<cudaStream_t>(cuda_stream);
  return SV_OK;
}

sv_status sv_set_dense_pool(sv_state* h, const double* pool, size_t n_complex) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (n_complex && !pool) return fail(SV_ERR_ARG, "pool is NULL");
  h->dense.assign(pool, pool + 2 * n_complex);
  h->dense_hash = fnv1a(h->dense.data(), h->dense.size() * sizeof(double), 7);
  return SV_OK;
}

sv_status sv_set_tuning(sv_state* h, int tile_bits, int low_bits, int max_pass_gates) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (tile_bits && (tile_bits < 10 || tile_bits > svp::MAX_TILE_BITS)) return fail(SV_ERR_ARG, "tile_bits in 10..14");
  if (low_bits && (low_bits < 2 || low_bits > 14)) return fail(SV_ERR_ARG, "low_bits in 2..14");
  if (tile_bits && low_bits && tile_bits - low_bits > 9) return fail(SV_ERR_ARG, "tile_bits - low_bits <= 9");
  if (!tile_bits && low_bits && 12 - low_bits > 9) return fail(SV_ERR_ARG, "tile_bits - low_bits <= 9");
  if (max_pass_gates < 0 || max_pass_gates > svp::MAX_PASS_GATES) return fail(SV_ERR_ARG, "max_pass_gates in 0..128");
  h->tune.tile_bits = tile_bits;
  h->tune.low_bits = low_bits ? low_bits : -1;
  h->tune.max_pass_gates = max_pass_gates;
  return SV_OK;
}

sv_status sv_set_jit_blocks(sv_state* h, int blocks_per_sm) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (blocks_per_sm < 0 || blocks_per_sm > 4) return fail(SV_ERR_ARG, "blocks_per_sm in 0..4");
  h->tune.jit_min_blocks = blocks_per_sm;
  return SV_OK;
}

sv_status sv_set_tile_select(sv_state* h, int closure) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  h->tune.tile_select = closure ? 1 : 0;
  return SV_OK;
}

sv_status sv_set_stage_pairs(sv_state* h, int mode) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (mode < 0 || mode > 2) return fail(SV_ERR_ARG, "stage pair mode is 0, 1 or 2");
  h->tune.stage_pairs = mode;
  return SV_OK;
}

sv_status sv_prepare(sv_state* h, const sv_op* ops, size_t n_ops, sv_program** out) {
  if (!h || !out) return fail(SV_ERR_ARG, "null argument");
  sv_program* cached = nullptr;
  sv_status st = get_program(h, ops, n_ops, &cached);
  if (st != SV_OK) return st;
  // hand out a private copy so that sv_program_free never touches the cache
  std::unique_ptr<sv_program> p(new sv_program());
  p->owner = h;
  p->plan = cached->plan;
  st = upload_program(h, p.get());
  if (st != SV_OK) return st;
  h->prepared.insert(p.get());
  *out = p.release();
  return SV_OK;
}

sv_status sv_plan_info(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                       size_t n_complex, int tile_bits, int low_bits, int max_pass_gates, sv_program_stats* out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  svp::Tuning t;
  t.tile_bits = tile_bits;
  t.low_bits = low_bits ? low_bits : -1;
  t.max_pass_gates = max_pass_gates;
  svp::Plan P;
  std::string err;
  sv_status st = svp::build_plan(n, dtype, ops, n_ops, dense_pool, n_complex, t, P, err);
  if (st != SV_OK) return fail(st, err);
  *out = P.stats;
  return SV_OK;
}

sv_status sv_program_free(sv_program* p) {
  if (!p) return SV_OK;
  if (p->cached) return fail(SV_ERR_ARG, "program belongs to a cache");
  if (p->owner) {  // null once its state was destroyed (which waited for the state's work)
    cudaStreamSynchronize(p->owner->stream);
    p->owner->prepared.erase(p);
  }
  delete p;
  return SV_OK;
}

sv_status sv_program_info(const sv_program* p, sv_program_stats* out) {
  if (!p || !out) return fail(SV_ERR_ARG, "null argument");
  *out = p->plan.stats;
  out->specialised = p->jit ? 1 : 0;
  out->compile_seconds = p->jit ? p->jit->compile_seconds : 0.0;
  return SV_OK;
}

sv_status sv_set_jit(sv_state* h, int enable) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  h->use_jit = enable != 0;
  return SV_OK;
}

sv_status sv_set_dense_tc(sv_state* h, int enable) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  h->dense_tc = enable != 0;
  return SV_OK;
}

sv_status sv_jit_check(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                       size_t n_complex, char* log, size_t log_len) {
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  svp::Plan P;
  std::string err;
  sv_status st = svp::build_plan(n, dtype, ops, n_ops, dense_pool, dense_pool ? n_complex : 0, svp::Tuning{}, P, err);
  if (st == SV_OK) {
    std::vector<char> cubin;
    st = svj::compile_cubin(P, cubin, err, &err);
  }
  if (log && log_len) {
    const size_t k = std::min(err.size(), log_len - 1);
    std::memcpy(log, err.data(), k);
    log[k] = 0;
  }
  if (st != SV_OK) return fail(st, err);
  return SV_OK;
}

sv_status sv_jit_check_adjoint(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                               size_t n_complex, char* log, size_t log_len) {
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  svp::Tuning t;
  t.tile_bits = svk::BATCH_TILE_BITS;
  t.min_qubits = svk::BATCH_TILE_BITS;
  svp::Plan F, B;
  std::string err;
  sv_status st = svp::build_adjoint_plan(n, dtype, ops, n_ops, dense_pool, dense_pool ? n_complex : 0, t, F, B, err);
  if (st == SV_OK) {
    std::vector<char> cubin;
    st = svj::compile_adjoint_cubin(F, B, cubin, err, &err);
  }
  if (log && log_len) {
    const size_t k = std::min(err.size(), log_len - 1);
    std::memcpy(log, err.data(), k);
    log[k] = 0;
  }
  if (st != SV_OK) return fail(st, err);
  return SV_OK;
}

sv_status sv_jit_check_batch(sv_dtype dtype, size_t n_progs, const int* n, const sv_op* const* ops,
                             const size_t* n_ops, char* log, size_t log_len) {
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  if (!n_progs || !n || !ops || !n_ops) return fail(SV_ERR_ARG, "null or empty program arrays");
  std::vector<svp::Plan> plans(n_progs);
  std::vector<const svp::Plan*> pp;
  std::string err;
  sv_status st = SV_OK;
  for (size_t k = 0; k < n_progs && st == SV_OK; ++k) {
    svp::Tuning t;
    t.tile_bits = svk::BATCH_TILE_BITS;
    t.min_qubits = svk::BATCH_TILE_BITS;
    st = svp::build_plan(n[k], dtype, ops[k], n_ops[k], nullptr, 0, t, plans[k], err);
    pp.push_back(&plans[k]);
  }
  if (st == SV_OK) {
    std::vector<char> cubin;
    st = svj::compile_batch_cubin(pp, cubin, err, &err);
  }
  if (log && log_len) {
    const size_t k = std::min(err.size(), log_len - 1);
    std::memcpy(log, err.data(), k);
    log[k] = 0;
  }
  if (st != SV_OK) return fail(st, err);
  return SV_OK;
}

sv_status sv_launch(sv_state* h, sv_program* p, const double* dev_params, size_t n_params, uint64_t seed,
                    uint64_t stream_id, uint64_t shot) {
  if (!h || !p) return fail(SV_ERR_ARG, "null argument");
  if (p->owner != h) return fail(SV_ERR_ARG, "program prepared for another state");
  return launch_program(h, p, dev_params, n_params, seed, stream_id, shot);
}

sv_status sv_run(sv_state* h, const sv_op* ops, size_t n_ops, const double* params, size_t n_params, uint64_t seed,
                 uint64_t stream_id, uint64_t shot, uint64_t* creg_out) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (n_ops && !ops) return fail(SV_ERR_ARG, "ops is NULL");
  if (n_params && !params) return fail(SV_ERR_ARG, "params is NULL");
  sv_program* p = nullptr;
  sv_status st = get_program(h, ops, n_ops, &p);
  if (st != SV_OK) return st;
  if (n_params) {
    SV_CUDA(h->params.reserve(n_params));
    SV_CUDA(cudaMemcpyAsync(h->params.p, params, n_params * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  st = launch_program(h, p, n_params ? h->params.p : nullptr, n_params, seed, stream_id, shot);
  if (st != SV_OK) return st;
  if (creg_out) {
    SV_CUDA(cudaMemcpyAsync(creg_out, &h->ctrl->creg, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
    return check_status(h);
  }
  return SV_OK;
}

sv_status sv_get_creg(sv_state* h, uint64_t* creg) {
  if (!h || !creg) return fail(SV_ERR_ARG, "null argument");
  SV_CUDA(cudaMemcpyAsync(creg, &h->ctrl->creg, sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
  return check_status(h);
}

sv_status sv_get_trace(sv_state* h, sv_draw* out, size_t max, size_t* n_out) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  Ctrl c;
  SV_CUDA(cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  SV_CUDA(cudaStreamSynchronize(h->stream));
  const size_t k = std::min<size_t>(std::min<size_t>(c.n_trace, svp::MAX_TRACE), max);
  if (n_out) *n_out = c.m;
  if (k && out) {
    static_assert(sizeof(sv_draw) == sizeof(DTrace), "trace layout");
    SV_CUDA(cudaMemcpyAsync(out, h->trace, k * sizeof(DTrace), cudaMemcpyDeviceToHost, h->stream));
    SV_CUDA(cudaStreamSynchronize(h->stream));
  }
  return SV_OK;
}

sv_status sv_sample_state(sv_state* h, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                          uint64_t* out) {
  if (!h || (shots && !out)) return fail(SV_ERR_ARG, "null argument");
  if (!shots) return SV_OK;
  SV_CUDA(h->sample_out.reserve(shots));
  sv_status st = sample_current(h, shots, seed, stream_id, shot0, h->sample_out.p);
  if (st != SV_OK) return st;
  SV_CUDA(cudaMemcpyAsync(out, h->sample_out.p, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
  SV_CUDA(cudaStreamSynchronize(h->stream));
  return SV_OK;
}

sv_status sv_sample_state_device(sv_state* h, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                                 uint64_t* dev_out) {
  if (!h || (shots && !dev_out)) return fail(SV_ERR_ARG, "null argument");
  if (!shots) return SV_OK;
  if (h->profiling) {
    while (h->events.size() < h->ev_used + 2) {
      cudaEvent_t e;
      SV_CUDA(cudaEventCreate(&e));
      h->events.push_back(e);
    }
    SV_CUDA(cudaEventRecord(h->events[h->ev_used], h->stream));
  }
  const sv_status st = sample_current(h, shots, seed, stream_id, shot0, dev_out);
  if (st != SV_OK) return st;
  if (h->profiling) {
    SV_CUDA(cudaEventRecord(h->events[h->ev_used + 1], h->stream));
    h->ev_used += 2;
  }
  return SV_OK;
}

sv_status sv_sample(sv_state* h, const sv_op* ops, size_t n_ops, const double* params, size_t n_params,
                    uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t* creg_out, uint64_t* bits_out) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (!shots) return SV_OK;
  sv_program* p = nullptr;
  sv_status st = get_program(h, ops, n_ops, &p);
  if (st != SV_OK) return st;
  if (n_params) {
    SV_CUDA(h->params.reserve(n_params));
    SV_CUDA(cudaMemcpyAsync(h->params.p, params, n_params * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  const double* dp = n_params ? h->params.p : nullptr;
  if (!has_draws(ops, n_ops)) {
    st = launch_program(h, p, dp, n_params, seed, stream_id, 0);
    if (st != SV_OK) return st;
    if (creg_out) std::fill(creg_out, creg_out + shots, 0ull);
    if (bits_out) return sv_sample_state(h, shots, seed, stream_id, 0, bits_out);
    return check_status(h);
  }
  // one trajectory per shot; records gathered on the device
  SV_CUDA(h->sample_out.reserve(2 * shots));
  uint64_t* d_creg = h->sample_out.p;
  uint64_t* d_bits = h->sample_out.p + shots;
  for (uint64_t s = 0; s < shots; ++s) {
    st = launch_program(h, p, dp, n_params, seed, stream_id, s);
    if (st != SV_OK) return st;
    SV_CUDA(cudaMemcpyAsync(d_creg + s, &h->ctrl->creg, sizeof(uint64_t), cudaMemcpyDeviceToDevice, h->stream));
    if (bits_out) {
      st = sample_current(h, 1, seed, stream_id, s, d_bits + s);
      if (st != SV_OK) return st;
    }
  }
  if (creg_out)
    SV_CUDA(cudaMemcpyAsync(creg_out, d_creg, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
  if (bits_out)
    SV_CUDA(cudaMemcpyAsync(bits_out, d_bits, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream));
  return check_status(h);
}

sv_status sv_sample_branched(sv_state* h, const sv_op* ops, size_t n_ops, const double* params, size_t n_params,
                             uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t* creg_out,
                             sv_branch_stats* stats) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (shots && !creg_out) return fail(SV_ERR_ARG, "creg_out is NULL");
  if (n_ops && !ops) return fail(SV_ERR_ARG, "ops is NULL");
  if (n_params && !params) return fail(SV_ERR_ARG, "params is NULL");
  if (stats) *stats = sv_branch_stats{shots, 0, 0, 0};
  if (!shots) return SV_OK;
  sv_program* p = nullptr;
  sv_status st = get_program(h, ops, n_ops, &p);
  if (st != SV_OK) return st;
  if (n_params) {
    SV_CUDA(h->params.reserve(n_params));
    SV_CUDA(cudaMemcpyAsync(h->params.p, params, n_params * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  const double* dp = n_params ? h->params.p : nullptr;
  if (!h->branch) h->branch.reset(svb::work_new());
  size_t cap = 0;
  for (const svp::DScalar& x : p->plan.scalars) cap += (x.kind == svp::S_MEASURE || x.kind == svp::S_RESET) ? 1 : 0;
  cap = std::min<size_t>(cap, svp::MAX_TRACE);
  std::vector<DTrace> tr;
  // representatives run one after another on this state, each a full sv_launch
  svb::Runner run = [&](const std::vector<svb::RepReq>& reps, std::vector<svb::RepOut>& outs,
                        std::string& err) -> sv_status {
    outs.assign(reps.size(), svb::RepOut());
    for (size_t k = 0; k < reps.size(); ++k) {
      sv_status rs = launch_program(h, p, dp, n_params, seed, stream_id, reps[k].shot);
      if (rs != SV_OK) {
        err = g_err;
        return rs;
      }
      Ctrl c;
      cudaError_t e = cudaMemcpyAsync(&c, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream);
      tr.resize(cap);  // the program's draw items bound the draws a trajectory executes
      if (e == cudaSuccess && cap)
        e = cudaMemcpyAsync(tr.data(), h->trace, cap * sizeof(DTrace), cudaMemcpyDeviceToHost, h->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
      const size_t nk = std::min<uint64_t>(c.m, cap);
      if (e != cudaSuccess) {
        err = std::string("representative record: ") + cudaGetErrorString(e);
        return SV_ERR_CUDA;
      }
      svb::RepOut& o = outs[k];
      o.creg = c.creg;
      o.status = c.status;
      o.m = c.m;
      o.draws.resize(nk);
      for (size_t d = 0; d < nk; ++d) o.draws[d] = svk::BrDraw{tr[d].p0, tr[d].p1, tr[d].outcome, -1};
    }
    return SV_OK;
  };
  std::string err;
  st = svb::sample(h->branch.get(), h->stream, h->sms, {stream_id}, {shots}, seed, 0, run, creg_out, stats, err);
  if (st != SV_OK) return fail(st, err);
  return SV_OK;
}

sv_status sv_expval(sv_state* h, const sv_pauli* terms, size_t n_terms, double* total, double* per_term) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (n_terms && !terms) return fail(SV_ERR_ARG, "terms is NULL");
  const uint64_t lim = h->n >= 64 ? ~0ull : ((1ull << h->n) - 1);
  for (size_t t = 0; t < n_terms; ++t)
    if ((terms[t].x_mask | terms[t].z_mask) & ~lim) return fail(SV_ERR_ARG, "Pauli term acts on a qubit >= n");
  // group by X mask, in first-appearance order
  std::vector<uint64_t> keys;
  std::map<uint64_t, std::vector<size_t>> groups;
  for (size_t t = 0; t < n_terms; ++t) {
    auto it = groups.find(terms[t].x_mask);
    if (it == groups.end()) keys.push_back(terms[t].x_mask);
    groups[terms[t].x_mask].push_back(t);
  }
  std::vector<size_t> order;
  for (uint64_t x : keys)
    for (size_t t : groups[x]) order.push_back(t);
  const size_t nt = order.size();
  SV_CUDA(h->exp_out.reserve(std::max<size_t>(nt, 1)));
  const int grid = std::max(1, std::min(h->sms * 8, int((1ull << h->n_int) / 256)));
  SV_CUDA(h->exp_partials.reserve(size_t(grid) * 32));
  size_t slot = 0;
  for (uint64_t x : keys) {
    const size_t cnt = groups[x].size();
    // index bits of i behind the seven low bits of the pair index (bit h, the top bit of x, skipped)
    const int hbit = x ? 63 - __builtin_clzll(x) : 64;
    const uint64_t lmask = hbit < 7 ? (0xFFull & ~(1ull << hbit)) : 0x7Full;
    const std::vector<size_t>& g = groups[x];
    for (size_t c = 0; c < cnt; c += svk::EXPVAL_TERMS) {  // at most 16 terms per launch
      svk::ExpvalArgs a{};
      a.state = h->state;
      a.n = h->n_int;
      a.x_mask = x;
      a.nterms = int(std::min<size_t>(svk::EXPVAL_TERMS, cnt - c));
      for (int t = 0; t < svk::EXPVAL_TERMS; ++t) {
        a.zw[t] = 0;  // unused slot: summed, never written out
        a.zh7[t] = 0;
        if (t >= a.nterms) continue;
        const uint64_t z = terms[g[c + size_t(t)]].z_mask;
        uint32_t zl = 0, k = 0;
        for (int b = 0; b < 8; ++b)
          if ((lmask >> b) & 1) zl |= uint32_t((z >> b) & 1) << (k++);
        // phase i^q of the term (q = |x & z| mod 4): odd q takes the imaginary
        // part of the transform, q >= 2 flips the sign
        const uint32_t q = uint32_t(__builtin_popcountll(x & z) & 3);
        a.zw[t] = (zl + ((q & 1) ? 128u : 0u)) | ((q >> 1) << 8);
        // bits of z above the block's index bits (bit hbit < 7 of the first
        // index is always 0, so it drops out); n <= 34 keeps this in 32 bits
        a.zh7[t] = uint32_t((z & ~lmask) >> 7);
      }
      a.partials = h->exp_partials.p;
      a.out = h->exp_out.p + slot + c;
      a.ticket = h->exp_ticket;
      SV_CUDA(svk::launch_expval_group(h->dtype, a, grid, h->stream));
    }
    slot += cnt;
  }
  std::vector<double> vals(nt);
  if (nt) SV_CUDA(cudaMemcpyAsync(vals.data(), h->exp_out.p, nt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  SV_CUDA(cudaStreamSynchronize(h->stream));
  double tot = 0;
  std::vector<double> per(n_terms, 0.0);
  for (size_t k = 0; k < nt; ++k) per[order[k]] = vals[k];
  for (size_t t = 0; t < n_terms; ++t) tot += terms[t].coeff * per[t];
  if (total) *total = tot;
  if (per_term) std::copy(per.begin(), per.end(), per_term);
  return SV_OK;
}

// ------------------------------------------------------------------ batched execution

}  // extern "C"

struct sv_batch {
  sv_dtype dtype = SV_C64;
  size_t amp_bytes = 8;
  int sms = 0, grid = 0;
  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<std::unique_ptr<sv_program>> progs;
  std::vector<svk::BatchProg> hprogs;
  std::vector<uint32_t> prog_nint, prog_flags;
  DevBuf<svk::BatchProg> d_progs;
  DevBuf<svk::BatchItem> d_items;
  DevBuf<unsigned char> slots;
  DevBuf<uint8_t> fslots;
  DevBuf<Ctrl> ctrls;
  DevBuf<unsigned> queue;
  DevBuf<int> status;
  DevBuf<uint64_t> cregs;
  DevBuf<double> prm;
  Ctrl* prep_ctrl = nullptr;
  size_t n_items = 0;
  uint64_t slot_amps = 0;
  uint32_t slot_flags = 0;
  cudaGraphExec_t gexec = nullptr;
  uint64_t gkey = 0;
  // shot branching
  std::vector<uint32_t> prog_draws;  // draw items of each program (a bound on the draws a trajectory executes)
  std::vector<svk::BatchItem> items_host;  // staging of the last quick item upload
  int tune_low = 0, tune_gates = 0;           // planner tuning of programs added from now on (0: default)
  DevBuf<unsigned long long> work;            // device work counters while profiling (sv_batch_profile)
  bool profiling = false;
  bool use_jit = false;                       // the kernel specialised to the batch's programs (sv_batch_set_jit)
  std::shared_ptr<svj::JitKernel> jit;        // built for the first jit_nprogs programs
  size_t jit_nprogs = 0;
  DevBuf<DTrace> tslots;
  DevBuf<svk::BrDraw> tout;
  DevBuf<uint64_t> mout;
  std::unique_ptr<svb::Work, void (*)(svb::Work*)> branch{nullptr, svb::work_free};
  ~sv_batch() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (prep_ctrl) cudaFree(prep_ctrl);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (own) cudaStreamDestroy(own);
  }
};

extern "C" {

sv_status sv_batch_create(sv_dtype dtype, void* cuda_stream, sv_batch** out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  std::unique_ptr<sv_batch> b(new sv_batch());
  b->dtype = dtype;
  b->amp_bytes = dtype == SV_C64 ? 8 : 16;
  int dev = 0;
  SV_CUDA(cudaGetDevice(&dev));
  SV_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
  b->user = static_cast<cudaStream_t>(cuda_stream);
  SV_CUDA(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
  SV_CUDA(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
  SV_CUDA(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
  if (cudaMalloc(&b->prep_ctrl, sizeof(Ctrl)) != cudaSuccess) return fail(SV_ERR_OOM, "batch control block");
  int per_sm = 1;
  if (svk::batch_occupancy(dtype, &per_sm) != cudaSuccess) {
    cudaGetLastError();
    return fail(SV_ERR_CUDA, "batched kernel configuration failed");
  }
  b->grid = b->sms * per_sm;
  *out = b.release();
  return SV_OK;
}

sv_status sv_batch_add_program(sv_batch* b, int n, const sv_op* ops, size_t n_ops, const double* params,
                               size_t n_params, const double* dense_pool, size_t n_complex, uint32_t* prog_id) {
  if (!b || !prog_id) return fail(SV_ERR_ARG, "null argument");
  if (n_params && !params) return fail(SV_ERR_ARG, "params is NULL");
  std::unique_ptr<sv_program> p(new sv_program());
  svp::Tuning t;
  t.tile_bits = svk::BATCH_TILE_BITS;
  t.min_qubits = svk::BATCH_TILE_BITS;
  if (b->tune_low) t.low_bits = b->tune_low;
  t.max_pass_gates = b->tune_gates;
  std::string err;
  sv_status st = svp::build_plan(n, b->dtype, ops, n_ops, dense_pool, dense_pool ? n_complex : 0, t, p->plan, err);
  if (st != SV_OK) return fail(st, err);
  const svp::Plan& P = p->plan;
  if (n_params < P.n_params_needed) return fail(SV_ERR_ARG, "program references more parameters than given");
  st = upload_plan(b->own, b->amp_bytes, p.get());
  if (st != SV_OK) return st;
  if (n_params) {
    SV_CUDA(b->prm.reserve(n_params));
    SV_CUDA(cudaMemcpyAsync(b->prm.p, params, n_params * sizeof(double), cudaMemcpyHostToDevice, b->own));
  }
  SV_CUDA(cudaMemsetAsync(b->prep_ctrl, 0, sizeof(Ctrl), b->own));
  svk::PrepArgs pa{};
  pa.jobs = p->jobs.p;
  pa.njobs = int(P.jobs.size());
  pa.params = n_params ? b->prm.p : nullptr;
  pa.n_params = n_params;
  pa.consts = p->consts.p;
  pa.mats = p->mats.p;
  pa.ctrl = b->prep_ctrl;
  pa.init = p->init.p;
  pa.ninit = 0;
  pa.flags = p->flags.p;
  SV_CUDA(svk::launch_prep(b->dtype, pa, b->own));
  int32_t pst = 0;
  SV_CUDA(cudaMemcpyAsync(&pst, &b->prep_ctrl->status, sizeof(pst), cudaMemcpyDeviceToHost, b->own));
  SV_CUDA(cudaStreamSynchronize(b->own));
  if (pst) return fail(SV_ERR_ARG, "parameter index out of range");
  svk::BatchProg bp{};
  bp.passes = p->passes.p;
  bp.gates = p->gates.p;
  bp.stages = p->stages.p;
  bp.scalars = p->scalars.p;
  bp.mats = p->mats.p;
  bp.init = p->init.p;
  bp.npasses = uint32_t(P.passes.size());
  bp.ninit = uint32_t(P.init_items.size());
  *prog_id = uint32_t(b->progs.size());
  b->hprogs.push_back(bp);
  b->prog_nint.push_back(uint32_t(P.n_int));
  b->prog_flags.push_back(std::max<uint32_t>(P.n_flags, 1));
  uint32_t nd = 0;
  for (const svp::DScalar& x : P.scalars) nd += (x.kind == svp::S_MEASURE || x.kind == svp::S_RESET) ? 1u : 0u;
  b->prog_draws.push_back(nd);
  b->progs.push_back(std::move(p));
  SV_CUDA(b->d_progs.upload(b->hprogs, b->own));
  SV_CUDA(cudaStreamSynchronize(b->own));
  return SV_OK;
}

}  // extern "C"

namespace {
// quick: no wait for the upload and no device-memory query while the slots already fit
sv_status batch_items(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids, const uint64_t* shots,
                      size_t n_items, bool quick) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  if (n_items && (!prog_ids || !stream_ids || !shots)) return fail(SV_ERR_ARG, "null item arrays");
  if (n_items >= (size_t(1) << 32)) return fail(SV_ERR_ARG, "too many items");
  std::vector<svk::BatchItem> items(n_items);
  uint64_t max_nint = 0;
  uint32_t max_flags = 1;
  for (size_t i = 0; i < n_items; ++i) {
    if (prog_ids[i] >= b->progs.size()) return fail(SV_ERR_ARG, "unknown program id");
    svk::BatchItem& it = items[i];
    it.prog = prog_ids[i];
    it.n_int = b->prog_nint[prog_ids[i]];
    it.stream = stream_ids[i];
    it.shot = shots[i];
    it.out = uint32_t(i);
    max_nint = std::max<uint64_t>(max_nint, it.n_int);
    max_flags = std::max(max_flags, b->prog_flags[prog_ids[i]]);
  }
  // longest trajectories first, so that the tail of the launch is short
  std::stable_sort(items.begin(), items.end(),
                   [](const svk::BatchItem& x, const svk::BatchItem& y) { return x.n_int > y.n_int; });
  const uint64_t slot_amps = n_items ? (1ull << max_nint) : 1;
  const size_t need = size_t(b->grid) * slot_amps * b->amp_bytes;
  if (!(quick && need <= b->slots.n)) {
    size_t free_b = 0, total_b = 0;
    SV_CUDA(cudaMemGetInfo(&free_b, &total_b));
    if (need > b->slots.n && need - b->slots.n > free_b)
      return fail(SV_ERR_OOM, "batch work space exceeds free device memory");
  }
  if (cudaSuccess != b->slots.reserve(need)) return fail(SV_ERR_OOM, "batch state slots");
  SV_CUDA(b->fslots.reserve(size_t(b->grid) * max_flags));
  SV_CUDA(b->ctrls.reserve(size_t(b->grid)));
  SV_CUDA(b->queue.reserve(1));
  SV_CUDA(b->status.reserve(1));
  SV_CUDA(b->cregs.reserve(std::max<size_t>(n_items, 1)));
  if (quick) {  // the staging vector must outlive the copy: keep it in the handle
    b->items_host.swap(items);
    SV_CUDA(b->d_items.upload(b->items_host, b->own));
  } else {
    SV_CUDA(b->d_items.upload(items, b->own));
    SV_CUDA(cudaStreamSynchronize(b->own));
  }
  b->n_items = n_items;
  b->slot_amps = slot_amps;
  b->slot_flags = max_flags;
  return SV_OK;
}

// The batch kernel of the next launch: with sv_batch_set_jit(1), the one
// specialised to the handle's programs (built again when programs were added;
// if it cannot be built, the generic one), else the generic one.
sv_status batch_kernel(sv_batch* b, const svj::JitKernel** out) {
  *out = nullptr;
  if (!b->use_jit || b->progs.empty()) return SV_OK;
  if (!b->jit || b->jit_nprogs != b->progs.size()) {
    std::vector<const svp::Plan*> plans;
    for (const auto& p : b->progs) plans.push_back(&p->plan);
    std::string err;
    std::shared_ptr<svj::JitKernel> k;
    if (svj::compile_batch(plans, svk::batch_smem_bytes(b->dtype), k, err) != SV_OK) {
      b->jit.reset();
      b->jit_nprogs = b->progs.size();  // not retried until programs change
      return SV_OK;
    }
    uint32_t base = 0;
    for (size_t i = 0; i < b->hprogs.size(); ++i) {
      b->hprogs[i].jit_base = base;
      base += b->hprogs[i].npasses;
    }
    SV_CUDA(b->d_progs.upload(b->hprogs, b->own));
    b->jit = k;
    b->jit_nprogs = b->progs.size();
  }
  *out = b->jit.get();
  return SV_OK;
}

cudaError_t launch_batch_kernel(sv_batch* b, const svj::JitKernel* k, svk::BatchArgs& a) {
  if (!k) return svk::launch_batch(b->dtype, a, b->grid, b->own);
  std::string err;
  const int grid = std::min(b->grid, b->sms * k->per_sm);
  if (svj::launch_single(*k, &a, grid, b->own, err) != SV_OK) {
    g_err = err;
    return cudaErrorLaunchFailure;
  }
  return cudaSuccess;
}
}  // namespace

extern "C" {

sv_status sv_batch_set_items(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids, const uint64_t* shots,
                             size_t n_items) {
  return batch_items(b, prog_ids, stream_ids, shots, n_items, false);
}

sv_status sv_batch_launch(sv_batch* b, uint64_t seed) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  svk::BatchArgs a{};
  a.items = b->d_items.p;
  a.n_items = uint32_t(b->n_items);
  a.progs = b->d_progs.p;
  a.state_slots = b->slots.p;
  a.slot_amps = b->slot_amps;
  a.flag_slots = b->fslots.p;
  a.slot_flags = b->slot_flags;
  a.ctrls = b->ctrls.p;
  a.queue = b->queue.p;
  a.seed = seed;
  a.creg_out = b->cregs.p;
  a.status_out = b->status.p;
  a.work = b->profiling ? b->work.p : nullptr;
  const svj::JitKernel* jk = nullptr;
  sv_status kst = batch_kernel(b, &jk);
  if (kst != SV_OK) return kst;
  uint64_t key = fnv1a(&a, sizeof(a));
  key = fnv1a(&b->grid, sizeof(b->grid), key);
  key = fnv1a(&jk, sizeof(jk), key);
  if (!b->gexec || key != b->gkey) {
    if (b->gexec) {
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
    }
    cudaGraph_t g = nullptr;
    SV_CUDA(cudaStreamBeginCapture(b->own, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->queue.p, 0, sizeof(unsigned), b->own);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status.p, 0, sizeof(int), b->own);
    if (e == cudaSuccess) e = launch_batch_kernel(b, jk, a);
    cudaError_t e2 = cudaStreamEndCapture(b->own, &g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(e != cudaSuccess ? e : e2, "batch graph capture");
    }
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph instantiate");
    b->gkey = key;
  }
  SV_CUDA(cudaEventRecord(b->ev_in, b->user));
  SV_CUDA(cudaStreamWaitEvent(b->own, b->ev_in, 0));
  SV_CUDA(cudaGraphLaunch(b->gexec, b->own));
  SV_CUDA(cudaEventRecord(b->ev_out, b->own));
  SV_CUDA(cudaStreamWaitEvent(b->user, b->ev_out, 0));
  return SV_OK;
}

sv_status sv_batch_set_jit(sv_batch* b, int enable) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  b->use_jit = enable != 0;
  return SV_OK;
}

sv_status sv_batch_jit_info(sv_batch* b, int* specialised, double* compile_seconds) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  const svj::JitKernel* k = (b->use_jit && b->jit && b->jit_nprogs == b->progs.size()) ? b->jit.get() : nullptr;
  if (specialised) *specialised = k ? 1 : 0;
  if (compile_seconds) *compile_seconds = k ? k->compile_seconds : 0.0;
  return SV_OK;
}

sv_status sv_batch_profile(sv_batch* b, int enable) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  if (enable) {
    SV_CUDA(b->work.reserve(SV_WORK_COUNTERS));
    SV_CUDA(cudaMemsetAsync(b->work.p, 0, sizeof(unsigned long long) * SV_WORK_COUNTERS, b->own));
  }
  b->profiling = enable != 0;
  return SV_OK;
}

sv_status sv_batch_work(sv_batch* b, sv_work_counts* out) {
  if (!b || !out) return fail(SV_ERR_ARG, "null argument");
  *out = sv_work_counts{};
  if (!b->work.p) return SV_OK;
  unsigned long long w[SV_WORK_COUNTERS];
  SV_CUDA(cudaMemcpyAsync(w, b->work.p, sizeof(w), cudaMemcpyDeviceToHost, b->own));
  SV_CUDA(cudaStreamSynchronize(b->own));
  out->bytes_read = w[0];
  out->bytes_written = w[1];
  out->gates = w[2];
  out->draws = w[3];
  out->passes = w[4];
  out->updates = w[5];
  return SV_OK;
}

sv_status sv_batch_results(sv_batch* b, uint64_t* creg_out) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  int st = 0;
  if (b->n_items && creg_out)
    SV_CUDA(cudaMemcpyAsync(creg_out, b->cregs.p, b->n_items * sizeof(uint64_t), cudaMemcpyDeviceToHost, b->own));
  SV_CUDA(cudaMemcpyAsync(&st, b->status.p, sizeof(int), cudaMemcpyDeviceToHost, b->own));
  SV_CUDA(cudaStreamSynchronize(b->own));
  if (st == SV_ERR_NUMERIC) return fail(SV_ERR_NUMERIC, "a trajectory met a zero-norm state");
  if (st) return fail(sv_status(st), "device reported an error");
  return SV_OK;
}

sv_status sv_batch_run(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids, const uint64_t* shots,
                       size_t n_items, uint64_t seed, uint64_t* creg_out) {
  sv_status st = sv_batch_set_items(b, prog_ids, stream_ids, shots, n_items);
  if (st != SV_OK) return st;
  st = sv_batch_launch(b, seed);
  if (st != SV_OK) return st;
  return sv_batch_results(b, creg_out);
}

sv_status sv_batch_set_tuning(sv_batch* b, int low_bits, int max_pass_gates) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  if (low_bits && (low_bits < 3 || low_bits > svk::BATCH_TILE_BITS))
    return fail(SV_ERR_ARG, "low_bits in 3..12 (tile_bits - low_bits <= 9)");
  if (max_pass_gates < 0 || max_pass_gates > svp::MAX_PASS_GATES) return fail(SV_ERR_ARG, "max_pass_gates in 0..128");
  b->tune_low = low_bits;
  b->tune_gates = max_pass_gates;
  return SV_OK;
}

sv_status sv_batch_sample_branched(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids,
                                   const uint64_t* n_shots, size_t n_requests, uint64_t seed, uint64_t* creg_out,
                                   sv_branch_stats* stats) {
  if (!b) return fail(SV_ERR_ARG, "null handle");
  if (n_requests && (!prog_ids || !stream_ids || !n_shots)) return fail(SV_ERR_ARG, "null request arrays");
  if (n_requests >= (size_t(1) << 32)) return fail(SV_ERR_ARG, "too many requests");
  uint64_t total = 0;
  uint32_t cap = 1;
  for (size_t r = 0; r < n_requests; ++r) {
    if (prog_ids[r] >= b->progs.size()) return fail(SV_ERR_ARG, "unknown program id");
    total += n_shots[r];
    cap = std::max(cap, std::min<uint32_t>(b->prog_draws[prog_ids[r]], svp::MAX_TRACE));
  }
  if (stats) *stats = sv_branch_stats{total, 0, 0, 0};
  if (total && !creg_out) return fail(SV_ERR_ARG, "creg_out is NULL");
  if (!total) return SV_OK;
  if (!b->branch) b->branch.reset(svb::work_new());
  SV_CUDA(b->tslots.reserve(size_t(b->grid) * svp::MAX_TRACE));
  std::vector<uint32_t> ip;
  std::vector<uint64_t> is, ish, ic, im;
  std::vector<svk::BrDraw> itr;
  // the representatives of one round run together in one persistent launch
  svb::Runner run = [&](const std::vector<svb::RepReq>& reps, std::vector<svb::RepOut>& outs,
                        std::string& err) -> sv_status {
    const size_t k = reps.size();
    ip.resize(k);
    is.resize(k);
    ish.resize(k);
    for (size_t i = 0; i < k; ++i) {
      ip[i] = prog_ids[reps[i].req];
      is[i] = stream_ids[reps[i].req];
      ish[i] = reps[i].shot;
    }
    sv_status rs = batch_items(b, ip.data(), is.data(), ish.data(), k, true);
    if (rs != SV_OK) {
      err = g_err;
      return rs;
    }
    cudaError_t e = b->tout.reserve(k * size_t(cap));
    if (e == cudaSuccess) e = b->mout.reserve(k);
    svk::BatchArgs a{};
    a.items = b->d_items.p;
    a.n_items = uint32_t(k);
    a.progs = b->d_progs.p;
    a.state_slots = b->slots.p;
    a.slot_amps = b->slot_amps;
    a.flag_slots = b->fslots.p;
    a.slot_flags = b->slot_flags;
    a.ctrls = b->ctrls.p;
    a.queue = b->queue.p;
    a.seed = seed;
    a.creg_out = b->cregs.p;
    a.status_out = b->status.p;
    a.trace_slots = b->tslots.p;
    a.trace_out = b->tout.p;
    a.trace_cap = cap;
    a.m_out = b->mout.p;
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_in, b->user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->own, b->ev_in, 0);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->queue.p, 0, sizeof(unsigned), b->own);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->status.p, 0, sizeof(int), b->own);
    const svj::JitKernel* jk = nullptr;
    if (batch_kernel(b, &jk) != SV_OK) {
      err = g_err;
      return SV_ERR_CUDA;
    }
    if (e == cudaSuccess) e = launch_batch_kernel(b, jk, a);
    ic.resize(k);
    im.resize(k);
    itr.resize(k * size_t(cap));
    int bst = 0;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ic.data(), b->cregs.p, k * sizeof(uint64_t), cudaMemcpyDeviceToHost, b->own);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(im.data(), b->mout.p, k * sizeof(uint64_t), cudaMemcpyDeviceToHost, b->own);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(itr.data(), b->tout.p, itr.size() * sizeof(svk::BrDraw), cudaMemcpyDeviceToHost, b->own);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bst, b->status.p, sizeof(int), cudaMemcpyDeviceToHost, b->own);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->own);
    if (e != cudaSuccess) {
      err = std::string("batched representatives: ") + cudaGetErrorString(e);
      return SV_ERR_CUDA;
    }
    outs.assign(k, svb::RepOut());
    for (size_t i = 0; i < k; ++i) {
      svb::RepOut& o = outs[i];
      o.creg = ic[i];
      o.status = bst;  // the launch reports its first failing trajectory
      o.m = im[i];
      const size_t nk = std::min<uint64_t>(im[i], cap);
      o.draws.assign(itr.begin() + i * size_t(cap), itr.begin() + i * size_t(cap) + nk);
    }
    return SV_OK;
  };
  std::vector<uint64_t> rstream(stream_ids, stream_ids + n_requests), rshots(n_shots, n_shots + n_requests);
  std::string err;
  // one resident wave of the batched kernel seeds the first round
  sv_status st = svb::sample(b->branch.get(), b->own, b->sms, rstream, rshots, seed, uint64_t(b->grid), run, creg_out,
                             stats, err);
  if (st != SV_OK) return fail(st, err);
  return SV_OK;
}

sv_status sv_batch_destroy(sv_batch* b) {
  if (!b) return SV_OK;
  cudaStreamSynchronize(b->own);
  delete b;
  return SV_OK;
}

// ------------------------------------------------------------------ adjoint gradients

}  // extern "C"

struct sv_grad {
  sv_dtype dtype = SV_C64;
  size_t amp_bytes = 8;
  int sms = 0, grid = 0;
  cudaStream_t stream = nullptr;
  sv_program fwd, bwd;
  uint32_t n_params_needed = 0, ngroups = 0, nterms = 0;
  DevBuf<unsigned char> fmats, bmats, slots;
  DevBuf<uint64_t> hx, hz;
  DevBuf<uint32_t> hg0;
  DevBuf<double> hc;
  DevBuf<Ctrl> ctrls;
  DevBuf<uint8_t> fslots;
  DevBuf<unsigned> queue;
  bool use_jit = true;                     // the kernel specialised to this program (sv_grad_set_jit)
  bool jit_tried = false;
  std::shared_ptr<svj::JitAdjoint> jit;    // compiled at the first run; null: the generic kernel runs
};

extern "C" {

sv_status sv_grad_create(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                         size_t n_complex, const sv_pauli* terms, size_t n_terms, void* cuda_stream, sv_grad** out) {
  if (!out) return fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (dtype != SV_C64 && dtype != SV_C128) return fail(SV_ERR_ARG, "unknown dtype");
  if (n_terms && !terms) return fail(SV_ERR_ARG, "terms is NULL");
  const uint64_t lim = n >= 64 ? ~0ull : ((1ull << n) - 1);
  for (size_t t = 0; t < n_terms; ++t)
    if ((terms[t].x_mask | terms[t].z_mask) & ~lim) return fail(SV_ERR_ARG, "Pauli term acts on a qubit >= n");
  std::unique_ptr<sv_grad> g(new sv_grad());
  g->dtype = dtype;
  g->amp_bytes = dtype == SV_C64 ? 8 : 16;
  g->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  SV_CUDA(cudaGetDevice(&dev));
  SV_CUDA(cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev));
  svp::Tuning t;
  t.tile_bits = svk::BATCH_TILE_BITS;
  t.min_qubits = svk::BATCH_TILE_BITS;
  std::string err;
  sv_status st = svp::build_adjoint_plan(n, dtype, ops, n_ops, dense_pool, dense_pool ? n_complex : 0, t,
                                         g->fwd.plan, g->bwd.plan, err);
  if (st != SV_OK) return fail(st, err);
  st = upload_plan(g->stream, g->amp_bytes, &g->fwd);
  if (st != SV_OK) return st;
  st = upload_plan(g->stream, g->amp_bytes, &g->bwd);
  if (st != SV_OK) return st;
  g->n_params_needed = uint32_t(g->fwd.plan.n_params_needed);
  // Hamiltonian grouped by X mask: per term Z mask and coeff * i^{|x&z|}
  std::vector<uint64_t> keys;
  std::map<uint64_t, std::vector<size_t>> groups;
  for (size_t k = 0; k < n_terms; ++k) {
    if (!groups.count(terms[k].x_mask)) keys.push_back(terms[k].x_mask);
    groups[terms[k].x_mask].push_back(k);
  }
  std::vector<uint64_t> hx, hz;
  std::vector<uint32_t> hg0;
  std::vector<double> hc;
  for (uint64_t x : keys) {
    hx.push_back(x);
    hg0.push_back(uint32_t(hz.size()));
    for (size_t k : groups[x]) {
      hz.push_back(terms[k].z_mask);
      const int ph = __builtin_popcountll(x & terms[k].z_mask) & 3;
      const double c = terms[k].coeff;
      const double re[4] = {c, 0, -c, 0}, im[4] = {0, c, 0, -c};  // c * i^ph
      hc.push_back(re[ph]);
      hc.push_back(im[ph]);
    }
  }
  hg0.push_back(uint32_t(hz.size()));
  g->ngroups = uint32_t(hx.size());
  g->nterms = uint32_t(hz.size());
  SV_CUDA(g->hx.upload(hx, g->stream));
  SV_CUDA(g->hz.upload(hz, g->stream));
  SV_CUDA(g->hg0.upload(hg0, g->stream));
  SV_CUDA(g->hc.upload(hc, g->stream));
  SV_CUDA(cudaStreamSynchronize(g->stream));
  int per_sm = 1;
  if (svk::adjoint_occupancy(dtype, g->nterms, &per_sm) != cudaSuccess) {
    cudaGetLastError();
    return fail(SV_ERR_CUDA, "adjoint kernel configuration failed (too many Pauli terms?)");
  }
  g->grid = g->sms * per_sm;
  *out = g.release();
  return SV_OK;
}

sv_status sv_grad_run(sv_grad* g, const double* dev_params, size_t n_sets, size_t n_params, double* dev_val,
                      double* dev_grad) {
  if (!g) return fail(SV_ERR_ARG, "null handle");
  if (!n_sets) return SV_OK;
  if (n_params < g->n_params_needed) return fail(SV_ERR_ARG, "n_params below the largest parameter index used");
  if (n_params > size_t(svp::MAX_ADJ_PARAMS)) return fail(SV_ERR_ARG, "at most 1024 parameters");
  if ((g->n_params_needed && !dev_params) || !dev_val || (n_params && !dev_grad))
    return fail(SV_ERR_ARG, "null device array");
  if (n_sets >= (size_t(1) << 31)) return fail(SV_ERR_ARG, "too many parameter sets");
  const svp::Plan& F = g->fwd.plan;
  const svp::Plan& B = g->bwd.plan;
  const uint64_t fstride = std::max<uint32_t>(F.n_mat, 1), bstride = std::max<uint32_t>(B.n_mat, 1);
  if (g->fmats.reserve(n_sets * fstride * g->amp_bytes) != cudaSuccess ||
      g->bmats.reserve(n_sets * bstride * g->amp_bytes) != cudaSuccess)
    return fail(SV_ERR_OOM, "per-set gate matrices");
  if (g->use_jit && !g->jit_tried) {
    g->jit_tried = true;
    std::string err;
    if (svj::compile_adjoint(F, B, svk::adjoint_smem_bytes(g->dtype, g->nterms), g->jit, err) != SV_OK)
      g->jit.reset();  // the generic kernel remains
  }
  const svj::JitAdjoint* jk = g->use_jit ? g->jit.get() : nullptr;
  const int resident = jk ? g->sms * jk->per_sm : g->grid;
  const int grid = int(std::min<size_t>(size_t(resident), n_sets));
  const uint64_t slot = 1ull << F.n_int;
  if (g->slots.reserve(size_t(grid) * 2 * slot * g->amp_bytes) != cudaSuccess)
    return fail(SV_ERR_OOM, "phi / lambda work space");
  SV_CUDA(g->ctrls.reserve(size_t(grid)));
  SV_CUDA(g->fslots.reserve(size_t(grid)));
  SV_CUDA(g->queue.reserve(1));
  cudaStream_t s = g->stream;
  for (int which = 0; which < 2; ++which) {
    sv_program& p = which == 0 ? g->fwd : g->bwd;
    svk::PrepArgs pa{};
    pa.jobs = p.jobs.p;
    pa.njobs = int(p.plan.jobs.size());
    pa.params = dev_params;
    pa.n_params = n_params;
    pa.consts = p.consts.p;
    pa.mats = which == 0 ? g->fmats.p : g->bmats.p;
    pa.nsets = uint32_t(n_sets);
    pa.params_stride = n_params;
    pa.mats_stride = which == 0 ? fstride : bstride;
    if (pa.njobs) SV_CUDA(svk::launch_prep(g->dtype, pa, s));
  }
  SV_CUDA(cudaMemsetAsync(g->queue.p, 0, sizeof(unsigned), s));
  svk::AdjArgs a{};
  a.fwd.passes = g->fwd.passes.p;
  a.fwd.gates = g->fwd.gates.p;
  a.fwd.stages = g->fwd.stages.p;
  a.fwd.scalars = g->fwd.scalars.p;
  a.fwd.mats = g->fmats.p;
  a.f_npasses = uint32_t(F.passes.size());
  a.f_mat_stride = fstride;
  a.b_passes = g->bwd.passes.p;
  a.b_gates = g->bwd.gates.p;
  a.b_stages = g->bwd.stages.p;
  a.b_npasses = uint32_t(B.passes.size());
  a.b_mats = g->bmats.p;
  a.b_mat_stride = bstride;
  a.hx = g->hx.p;
  a.hg0 = g->hg0.p;
  a.ngroups = g->ngroups;
  a.hz = g->hz.p;
  a.hc = reinterpret_cast<const double2*>(g->hc.p);
  a.nterms = g->nterms;
  a.slots = g->slots.p;
  a.slot_amps = slot;
  a.ctrls = g->ctrls.p;
  a.flag_slots = g->fslots.p;
  a.slot_flags = 1;
  a.queue = g->queue.p;
  a.nsets = uint32_t(n_sets);
  a.n_params = uint32_t(n_params);
  a.n_int = F.n_int;
  a.val_out = dev_val;
  a.grad_out = dev_grad;
  if (jk) {
    std::string err;
    const sv_status st = svj::launch_adjoint(*jk, a, grid, s, err);
    if (st != SV_OK) return fail(st, err);
    return SV_OK;
  }
  SV_CUDA(svk::launch_adjoint(g->dtype, a, grid, s));
  return SV_OK;
}

sv_status sv_grad_set_jit(sv_grad* g, int enable) {
  if (!g) return fail(SV_ERR_ARG, "null handle");
  g->use_jit = enable != 0;
  return SV_OK;
}

sv_status sv_grad_info(const sv_grad* g, sv_grad_stats* out) {
  if (!g || !out) return fail(SV_ERR_ARG, "null argument");
  out->forward_passes = g->fwd.plan.passes.size();
  out->backward_passes = g->bwd.plan.passes.size();
  out->gates = g->fwd.plan.stats.gates;
  out->term_groups = g->ngroups;
  out->terms = g->nterms;
  out->state_qubits = uint32_t(g->fwd.plan.n_int);
  const svj::JitAdjoint* jk = g->use_jit ? g->jit.get() : nullptr;
  out->resident_sets = uint32_t(jk ? g->sms * jk->per_sm : g->grid);
  out->specialised = jk ? 1u : 0u;
  out->pad = 0;
  out->compile_seconds = jk ? jk->compile_seconds : 0.0;
  return SV_OK;
}

sv_status sv_grad_destroy(sv_grad* g) {
  if (!g) return SV_OK;
  cudaStreamSynchronize(g->stream);
  delete g;
  return SV_OK;
}

sv_status sv_expval_grad_batch(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* params,
                               size_t n_sets, size_t n_params, const sv_pauli* terms, size_t n_terms, double* val_out,
                               double* grad_out, void* cuda_stream) {
  if (n_sets && (!val_out || (n_params && (!params || !grad_out)))) return fail(SV_ERR_ARG, "null host array");
  sv_grad* g = nullptr;
  sv_status st = sv_grad_create(n, dtype, ops, n_ops, nullptr, 0, terms, n_terms, cuda_stream, &g);
  if (st != SV_OK) return st;
  std::unique_ptr<sv_grad, sv_status (*)(sv_grad*)> guard(g, sv_grad_destroy);
  DevBuf<double> dp, dv, dg;
  SV_CUDA(dp.reserve(std::max<size_t>(n_sets * n_params, 1)));
  SV_CUDA(dv.reserve(std::max<size_t>(n_sets, 1)));
  SV_CUDA(dg.reserve(std::max<size_t>(n_sets * n_params, 1)));
  cudaStream_t s = g->stream;
  if (n_sets * n_params)
    SV_CUDA(cudaMemcpyAsync(dp.p, params, n_sets * n_params * sizeof(double), cudaMemcpyHostToDevice, s));
  st = sv_grad_run(g, dp.p, n_sets, n_params, dv.p, dg.p);
  if (st != SV_OK) return st;
  if (n_sets) SV_CUDA(cudaMemcpyAsync(val_out, dv.p, n_sets * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (n_sets * n_params)
    SV_CUDA(cudaMemcpyAsync(grad_out, dg.p, n_sets * n_params * sizeof(double), cudaMemcpyDeviceToHost, s));
  SV_CUDA(cudaStreamSynchronize(s));
  return SV_OK;
}

sv_status sv_get_amplitudes(sv_state* h, void* host_dst, size_t first, size_t count) {
  if (!h || (count && !host_dst)) return fail(SV_ERR_ARG, "null argument");
  if (first + count > (size_t(1) << h->n) || first + count < first) return fail(SV_ERR_ARG, "range outside the state");
  SV_CUDA(cudaMemcpyAsync(host_dst, static_cast<char*>(h->state) + first * h->amp_bytes, count * h->amp_bytes,
                          cudaMemcpyDeviceToHost, h->stream));
  SV_CUDA(cudaStreamSynchronize(h->stream));
  return SV_OK;
}

sv_status sv_set_amplitudes(sv_state* h, const void* host_src, size_t first, size_t count) {
  if (!h || (count && !host_src)) return fail(SV_ERR_ARG, "null argument");
  if (first + count > (size_t(1) << h->n) || first + count < first) return fail(SV_ERR_ARG, "range outside the state");
  SV_CUDA(cudaMemcpyAsync(static_cast<char*>(h->state) + first * h->amp_bytes, host_src, count * h->amp_bytes,
                          cudaMemcpyHostToDevice, h->stream));
  SV_CUDA(cudaStreamSynchronize(h->stream));
  return SV_OK;
}

sv_status sv_state_buffer(sv_state* h, void** dev_ptr, size_t* bytes) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (dev_ptr) *dev_ptr = h->state;
  if (bytes) *bytes = (size_t(1) << h->n_int) * h->amp_bytes;
  return SV_OK;
}

sv_status sv_set_cache(sv_state* h, int enable) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  h->use_cache = enable != 0;
  return SV_OK;
}

sv_status sv_profile(sv_state* h, int enable) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (enable && !h->profiling)
    SV_CUDA(cudaMemsetAsync(h->work, 0, sizeof(unsigned long long) * SV_WORK_COUNTERS, h->stream));
  h->profiling = enable != 0;
  return SV_OK;
}

sv_status sv_profile_work(sv_state* h, sv_work_counts* out) {
  if (!h || !out) return fail(SV_ERR_ARG, "null argument");
  unsigned long long w[SV_WORK_COUNTERS];
  SV_CUDA(cudaMemcpyAsync(w, h->work, sizeof(w), cudaMemcpyDeviceToHost, h->stream));
  SV_CUDA(cudaStreamSynchronize(h->stream));
  out->bytes_read = w[0];
  out->bytes_written = w[1];
  out->gates = w[2];
  out->draws = w[3];
  out->passes = w[4];
  out->updates = w[5];
  return SV_OK;
}

sv_status sv_profile_read(sv_state* h, double* total_ms, uint64_t* launches, double* bytes) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  SV_CUDA(cudaStreamSynchronize(h->stream));
  double ms = 0;
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float t = 0;
    SV_CUDA(cudaEventElapsedTime(&t, h->events[i], h->events[i + 1]));
    ms += t;
  }
  sv_work_counts w{};
  const sv_status st = sv_profile_work(h, &w);
  if (st != SV_OK) return st;
  if (total_ms) *total_ms = ms;
  if (launches) *launches = h->ev_used / 2;
  if (bytes) *bytes = double(w.bytes_read) + double(w.bytes_written);
  h->ev_used = 0;
  SV_CUDA(cudaMemsetAsync(h->work, 0, sizeof(unsigned long long) * SV_WORK_COUNTERS, h->stream));
  return SV_OK;
}

sv_status sv_selftest_wait(sv_state* h, uint32_t polls) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  if (polls > (1u << 24)) return fail(SV_ERR_ARG, "polls must be at most 2^24");
  SV_CUDA(cudaMemsetAsync(&h->ctrl->status, 0, sizeof(int32_t), h->stream));
  SV_CUDA(svk::launch_wait_probe(polls, &h->ctrl->status, h->stream));
  const sv_status st = check_status(h);
  if (st == SV_ERR_TIMEOUT) g_err = "bounded device wait ran out (self test: nothing arrives at its mbarrier)";
  return st;
}

sv_status sv_sync(sv_state* h) {
  if (!h) return fail(SV_ERR_ARG, "null handle");
  SV_CUDA(cudaStreamSynchronize(h->stream));
  return SV_OK;
}

}  // extern "C"
