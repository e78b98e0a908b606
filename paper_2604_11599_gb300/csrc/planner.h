// planner.h -- lowering of the flat IR into passes, stages and scalar items.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sv.h"
#include "sv_plan.h"

namespace svp {

struct Tuning {
  int tile_bits = 12;      // m: qubits held by one shared-memory tile
  int low_bits = -1;       // L: contiguous low qubits of every tile (-1: per dtype)
  int max_pass_gates = 0;  // 0: up to MAX_PASS_GATES
  int min_qubits = 10;     // states are padded to at least this many qubits
  int tile_select = 1;     // 1: each tile's gathered qubits chosen for the gates they unlock; 0: first fit
  int jit_min_blocks = 0;  // specialised kernels: CTAs per SM they are compiled for (0: 2 complex64, 1 complex128)
  int stage_pairs = 0;     // complex64 stage packing: 0 fewest stages; 1 / 2: a stage without 16-byte pair
                           // accesses costs 3/2 / 2 times one with them (n=30 layered: 150.1 / 150.4 /
                           // 155.6 ms per step, so fewest stages is the default)
};

struct Plan {
  int n = 0;        // logical qubits
  int n_int = 0;    // simulated qubits (>= 4; extra qubits stay |0>)
  int dtype = 0;
  int m = 0, L = 0;
  int jit_min_blocks = 0;  // Tuning::jit_min_blocks
  std::vector<DPass> passes;
  std::vector<DGate> gates;
  std::vector<DStage> stages;
  std::vector<DScalar> scalars;      // phase items, referenced by passes
  std::vector<DScalar> init_items;   // COND evaluations before the first measurement
  std::vector<DJob> jobs;
  std::vector<double> consts;        // complex constant pool (re, im pairs)
  uint32_t n_mat = 0;                // complex entries in the matrix pool
  uint32_t n_flags = 0;
  uint32_t max_pass_mat = 0;
  uint32_t max_stages = 0;
  uint32_t max_gates = 0;
  uint32_t max_scalars = 0;
  uint32_t max_dots = 0;             // backward plans: derivative accumulators per pass
  bool needs_flush = false;
  bool gen_init = false;             // the first pass surely stores: it generates |0...0> itself (no init sweep)
  sv_program_stats stats{};
  uint64_t n_params_needed = 0;      // 1 + the largest parameter index referenced
};

// Builds the forward plan and the backward (adjoint) plan of a static program
// for gradients of <H>: `bwd` sweeps the reversed gate list with three gate
// register bits per stage, each parametrised gate preceded by its derivative
// accumulation items.  SV_ERR_UNSUPPORTED for programs with measurement,
// reset, COND or dense 4-qubit gates.
sv_status build_adjoint_plan(int n, int dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                             size_t dense_len, const Tuning& tune, Plan& fwd, Plan& bwd, std::string& err);

// Builds a plan; returns SV_OK or an error with a message in `err`.
sv_status build_plan(int n, int dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                     size_t dense_len, const Tuning& tune, Plan& out, std::string& err);

}  // namespace svp
