// kernels.h -- host-side launchers of the libsv kernels.
#pragma once
#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

#include "../../include/sv.h"
#include "sv_plan.h"

namespace svk {

struct PassArgs {
  void* state;
  const svp::DPass* passes;
  const svp::DGate* gates;
  const svp::DStage* stages;
  const svp::DScalar* scalars;
  const void* mats;
  uint8_t* flags;
  svp::Ctrl* ctrl;
  svp::DTrace* trace;
  double* partials;  // [grid][16]
  int n;             // simulated qubits
  int pass;          // pass index (specialised kernels select their stage program by it)
  int dense_tc;      // 1: dense four-qubit gates of complex64 2^12-amplitude tiles on the tensor cores
  int gen_init;      // 1: this launch is the program's first pass and generates |0...0> instead of loading it
  // work counters (nullable): [0] bytes of the state read, [1] bytes of it
  // written, [2] gate records executed (predicated-off ones excluded), [3]
  // draws executed, [4] passes that touched the state, [5] amplitude-gate
  // updates (executed gates and draws, 2^n each)
  unsigned long long* work;
};

struct PrepArgs {
  const svp::DJob* jobs;
  int njobs;
  const double* params;
  uint64_t n_params;
  const double* consts;
  void* mats;
  svp::Ctrl* ctrl;
  const svp::DScalar* init;
  int ninit;
  uint8_t* flags;
  uint64_t seed, stream, shot;
  uint32_t nsets;           // parameter sets (grid y); 0 or 1: one set
  uint64_t params_stride;   // doubles between parameter sets
  uint64_t mats_stride;     // complex entries between matrix sets
};

#ifndef __CUDACC_RTC__
cudaError_t launch_prep(int dtype, const PrepArgs& p, cudaStream_t s);
#endif
#ifndef __CUDACC_RTC__
cudaError_t launch_init_state(int dtype, void* state, uint64_t n_amp, int sms, cudaStream_t s);
// bounded-wait self test: a one-warp kernel whose mbarrier wait always runs out
cudaError_t launch_wait_probe(uint32_t polls, int32_t* status, cudaStream_t s);
#endif
#ifndef __CUDACC_RTC__
// dense: the pass holds a dense four-qubit gate (its tensor-core variant runs when a.dense_tc)
// proj: the pass may start with a measurement projector pending (its copy-pipelined variant runs)
cudaError_t launch_pass(int dtype, const PassArgs& a, int pi, int grid, int m, cudaStream_t s, bool dense, bool proj);
#endif
#ifndef __CUDACC_RTC__
cudaError_t pass_occupancy(int dtype, int m, int* blocks_per_sm);
#endif

// shot branching: the draws of one representative trajectory per outcome path,
// and the walk that routes every shot of a request down the tree of paths
struct BrDraw {
  double p0, p1;    // unnormalised outcome masses the draw compared against
  int32_t outcome;  // the representative's outcome
  int32_t child;    // path whose representative took the other outcome here (-1: none yet)
};
struct BrPath {
  uint32_t off, len;  // its draws: draws[off .. off + len)
  uint64_t creg;      // classical register at the end of the path
};

// persistent batched execution: one CTA runs one trajectory at a time
struct BatchProg {
  const svp::DPass* passes;
  const svp::DGate* gates;
  const svp::DStage* stages;
  const svp::DScalar* scalars;
  const void* mats;
  const svp::DScalar* init;
  uint32_t npasses, ninit;
  uint32_t jit_base;  // specialised batch kernels: the program's first pass in the module's pass numbering
  uint32_t pad;
};

struct BatchItem {
  uint32_t prog;    // index into the program table
  uint32_t n_int;   // simulated qubits (>= 12)
  uint64_t stream;  // Philox stream of the trajectory
  uint64_t shot;
  uint32_t out;     // output slot
  uint32_t pad;
};

struct BatchArgs {
  const BatchItem* items;
  uint32_t n_items;
  const BatchProg* progs;
  void* state_slots;  // [grid][slot_amps] amplitudes
  uint64_t slot_amps;
  uint8_t* flag_slots;  // [grid][slot_flags]
  uint32_t slot_flags;
  svp::Ctrl* ctrls;     // [grid]
  unsigned* queue;      // next item (reset to 0 before the launch)
  uint64_t seed;
  uint64_t* creg_out;   // [n_items], indexed by BatchItem::out
  int* status_out;      // first nonzero trajectory status
  // draw records (shot branching; trace_out == nullptr: none are kept)
  svp::DTrace* trace_slots;  // [grid][MAX_TRACE] per-CTA scratch
  BrDraw* trace_out;         // [n_items][trace_cap]
  uint32_t trace_cap;
  uint64_t* m_out;           // [n_items] draws executed
  unsigned long long* work;  // work counters of PassArgs::work (nullable)
};
constexpr int BATCH_TILE_BITS = 12;
#ifndef __CUDACC_RTC__
cudaError_t launch_batch(int dtype, const BatchArgs& a, int grid, cudaStream_t s);
#endif
#ifndef __CUDACC_RTC__
cudaError_t batch_occupancy(int dtype, int* blocks_per_sm);
size_t batch_smem_bytes(int dtype);  // dynamic shared memory of a batch launch
#endif

// the walk over the shots of one or more requests (kern_branch.cu)
struct BranchArgs {
  const BrDraw* draws;
  const BrPath* paths;
  const uint64_t* req_begin;   // [nreq + 1] first shot (global index) of each request
  const uint64_t* req_stream;  // [nreq] Philox stream of each request
  const uint32_t* req_root;    // [nreq] first path of each request
  uint32_t nreq;
  uint64_t seed;
  uint64_t nshots;
  uint64_t* walk;      // [nshots] (path << 32) | depth, bit 31 set once the shot reached its path's end
  uint32_t* claim;     // [ndraws] smallest shot that left the tree at this draw (0xFFFFFFFF: none)
  uint32_t* fresh;     // [ndraws] draws claimed for the first time by this walk
  uint32_t* nfresh;
  uint64_t* creg_out;  // [nshots] (gather)
};
#ifndef __CUDACC_RTC__
cudaError_t launch_branch_init(const BranchArgs& a, int sms, cudaStream_t s);
cudaError_t launch_branch_walk(const BranchArgs& a, int sms, cudaStream_t s);
cudaError_t launch_branch_gather(const BranchArgs& a, int sms, cudaStream_t s);
#endif

// batched adjoint gradients: one CTA per parameter set (persistent)
struct AdjArgs {
  PassArgs fwd;  // forward plan (state, ctrl, flags, mats and n are set per CTA)
  uint32_t f_npasses;
  uint64_t f_mat_stride;  // complex entries per parameter set
  const svp::DPass* b_passes;
  const svp::DGate* b_gates;
  const svp::DStage* b_stages;
  uint32_t b_npasses;
  const void* b_mats;
  uint64_t b_mat_stride;
  const uint64_t* hx;   // [ngroups] X mask of each term group
  const uint32_t* hg0;  // [ngroups + 1] first term of each group
  uint32_t ngroups;
  const uint64_t* hz;   // [nterms] Z masks
  const double2* hc;    // [nterms] coefficient * i^{|x&z|}
  uint32_t nterms;
  void* slots;          // [grid][2][slot_amps]: phi, lambda
  uint64_t slot_amps;
  svp::Ctrl* ctrls;
  uint8_t* flag_slots;
  uint32_t slot_flags;
  unsigned* queue;
  uint32_t nsets, n_params;
  int n_int;
  double* val_out;   // [nsets]
  double* grad_out;  // [nsets][n_params]
};
#ifndef __CUDACC_RTC__
cudaError_t launch_adjoint(int dtype, const AdjArgs& a, int grid, cudaStream_t s);
#endif
#ifndef __CUDACC_RTC__
cudaError_t adjoint_occupancy(int dtype, uint32_t nterms, int* blocks_per_sm);
size_t adjoint_smem_bytes(int dtype, uint32_t nterms);  // dynamic shared memory of an adjoint launch
#endif

// terminal sampling: run sums and in-block prefixes -> block scan -> per-shot search
struct SampleArgs {
  const void* state;
  int n;                 // simulated qubits (>= 10)
  int n_logical;
  double* run_cum;       // [2^(n-5)] inclusive prefix of 32-amplitude run sums within each block
  double* block_sums;    // [nblocks]
  double* block_prefix;  // [nblocks] exclusive prefix; [nblocks] total at the end
  uint64_t shots, seed, stream, shot0;
  uint64_t* out;         // [shots]
};
#ifndef __CUDACC_RTC__
cudaError_t launch_sample(int dtype, const SampleArgs& a, int sms, cudaStream_t s);
#endif
#ifndef __CUDACC_RTC__
uint64_t sample_blocks(int n);
uint64_t sample_runs(int n);
#endif

// Pauli expectation values of one group of terms sharing an X mask.  The
// terms travel in the kernel's parameter block (warp-uniform operands): for
// term t with phase q = |x & z| mod 4 and zl its Z mask on the seven index bits
// a 128-pair block spans, zw[t] = (zl, or 128 + zl for odd q) | (q >> 1) << 8,
// and zh7[t] = the rest of its Z mask shifted down by 7.
constexpr int EXPVAL_TERMS = 16;
struct ExpvalArgs {
  const void* state;
  int n;
  uint64_t x_mask;
  uint32_t zh7[EXPVAL_TERMS];  // Z mask bits above bit 6 of the pair's first index, shifted down by 7
  uint32_t zw[EXPVAL_TERMS];   // bits 0..7: index of the term's transform value (Re: zl, Im: 128 + zl); bit 8: sign flip
  int nterms;               // <= 16
  double* partials;         // [grid][32]
  double* out;              // [nterms] (written by the last CTA)
  unsigned* ticket;
};
#ifndef __CUDACC_RTC__
cudaError_t launch_expval_group(int dtype, const ExpvalArgs& a, int grid, cudaStream_t s);
#endif

}  // namespace svk
