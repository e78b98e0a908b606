// branch.h -- shot branching: every shot of a dynamic circuit with the
// number of trajectories actually simulated equal to the number of distinct
// outcome paths the shots take.
//
// Shot s of a request draws outcome o at its m-th measurement by comparing
// u(seed, stream, s, m) with p0 / (p0 + p1) of its own state (Sec. III-C:
// the outcome is decided at run time, not by pre-computed branches).  Two
// shots that took the same outcomes so far hold bit-identical states (the
// kernels are deterministic for a fixed program and outcome sequence), so at
// the next draw they compare their own u against the same (p0, p1).  One
// representative trajectory per path therefore gives (p0, p1) at every draw
// of every shot that follows it: a device walk replays each shot's draws
// against the recorded masses, finds where it leaves its path, and the shots
// that left a path at the same draw get one new representative (the smallest
// such shot), run in full on the same engine.  Every shot's record equals the
// record its own trajectory would give, bit for bit.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "kernels.h"

namespace svb {

struct RepReq {
  uint32_t req;   // request index
  uint64_t shot;  // shot counter within the request
};

struct RepOut {
  uint64_t creg = 0;
  int32_t status = 0;
  uint64_t m = 0;                   // draws executed
  std::vector<svk::BrDraw> draws;   // the first min(m, MAX_TRACE) of them
};

// Runs the representatives (each from |0...0>, its own Philox counter) on
// one engine and returns their records; the draws of out[k].draws must be
// those of reps[k] in execution order.
using Runner = std::function<sv_status(const std::vector<RepReq>& reps, std::vector<RepOut>& out, std::string& err)>;

struct Work;  // device scratch of the walk, reused across calls
Work* work_new();
void work_free(Work* w);

// req_stream[r], req_shots[r]: Philox stream and shot count of request r.
// seed_reps: representatives of the first round over all requests (shared
// in proportion to the shot counts, at least one each): an engine that runs
// them side by side (the batched launch) finds most paths in one round; an
// engine that runs them one after another passes 0.
// creg_out (host): the records of all shots, request by request.
sv_status sample(Work* w, cudaStream_t s, int sms, const std::vector<uint64_t>& req_stream,
                 const std::vector<uint64_t>& req_shots, uint64_t seed, uint64_t seed_reps, const Runner& run,
                 uint64_t* creg_out, sv_branch_stats* stats, std::string& err);

}  // namespace svb
