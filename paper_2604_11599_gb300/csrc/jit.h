// jit.h -- per-program specialisation of the pass kernel (NVRTC).
//
// A lowered program fixes, for every pass, its gate kinds, their register
// positions and the shared-memory addresses of every stage.  The specialiser
// writes one kernel per pass in which those are compile-time constants: no
// gate dispatch at run time, CX / X / SWAP become register renames and
// addresses fold into immediates.  Gate matrices and predicate flags remain
// run-time data, so the compiled module serves every parameter set and every
// trajectory of the program (compiled once, run many).
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "kernels.h"
#include "planner.h"

namespace svj {

struct JitModule {
  std::vector<void*> modules;      // CUmodule per chunk of passes
  std::vector<void*> functions;    // CUfunction of each pass
  std::vector<void*> functions_tc; // its tensor-core variant (passes with a dense gate), else null
  size_t smem = 0;                 // dynamic shared memory per launch
  double compile_seconds = 0;
  ~JitModule();
};

// Source text of the specialised module (for tests and inspection of the generator).
std::string generate_source(const svp::Plan& P);

// NVRTC only (no device needed): the module's cubin; with info, the ptxas
// resource report (registers, spills, stack) of every chunk is appended to it.
sv_status compile_cubin(const svp::Plan& P, std::vector<char>& cubin, std::string& err,
                        std::string* info = nullptr);

// compile_cubin + load into the current context.  Modules are cached for the
// process by device and generated source, so a program lowered again reuses
// its compiled kernels.
sv_status compile(const svp::Plan& P, std::shared_ptr<JitModule>& out, std::string& err);

sv_status launch(const JitModule& J, int pass, const svk::PassArgs& a, int grid, cudaStream_t s, std::string& err);

// The batched adjoint kernel specialised to one program: its forward passes'
// stage programs (CTA mode) and its backward passes' (phi / lambda groups,
// derivative accumulations) with every gate, register position and address a
// constant; the per-set matrices stay run-time data.
struct JitAdjoint {
  void* module = nullptr;  // CUmodule
  void* fn = nullptr;      // CUfunction sv_jit_adjoint
  size_t smem = 0;         // dynamic shared memory per launch
  int per_sm = 1;          // resident CTAs per SM (occupancy of the compiled kernel)
  double compile_seconds = 0;
  ~JitAdjoint();
};
std::string generate_adjoint_source(const svp::Plan& F, const svp::Plan& B);
// NVRTC only (no device needed), as compile_cubin
sv_status compile_adjoint_cubin(const svp::Plan& F, const svp::Plan& B, std::vector<char>& cubin, std::string& err,
                                std::string* info = nullptr);
// compiled and loaded; cached for the process by device, source and shared-memory size
sv_status compile_adjoint(const svp::Plan& F, const svp::Plan& B, size_t smem, std::shared_ptr<JitAdjoint>& out,
                          std::string& err);
sv_status launch_adjoint(const JitAdjoint& J, const svk::AdjArgs& a, int grid, cudaStream_t s, std::string& err);

// One specialised kernel in its own module.
struct JitKernel {
  void* module = nullptr;  // CUmodule
  void* fn = nullptr;      // CUfunction
  size_t smem = 0;         // dynamic shared memory per launch
  int per_sm = 1;          // resident CTAs per SM
  double compile_seconds = 0;
  ~JitKernel();
};
// The batched kernel specialised to a batch's programs (in the order given):
// each program's passes get their stage programs, numbered consecutively
// (BatchProg::jit_base is a program's first number).  Cached for the process by
// device, source and shared-memory size.
std::string generate_batch_source(const std::vector<const svp::Plan*>& plans);
// NVRTC only (no device needed), as compile_cubin
sv_status compile_batch_cubin(const std::vector<const svp::Plan*>& plans, std::vector<char>& cubin, std::string& err,
                              std::string* info = nullptr);
sv_status compile_batch(const std::vector<const svp::Plan*>& plans, size_t smem, std::shared_ptr<JitKernel>& out,
                        std::string& err);
// args: the address of the kernel's single parameter (e.g. an svk::BatchArgs)
sv_status launch_single(const JitKernel& K, void* args, int grid, cudaStream_t s, std::string& err);

}  // namespace svj
