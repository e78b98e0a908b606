/*
 * sv.h -- C-ABI of libsv, a GB300 (sm_103a) state-vector simulator for dynamic
 * circuits: mid-circuit measurement, reset, if/else on classical predicates
 * and bounded loops, with feed-forward decided on the GPU.
 *
 * The operations follow the paper's statement of the problem (arXiv
 * 2604.11599): OpenQASM 3.0 programs with classical control (if/else and
 * loops with a fixed trip count) and mid-circuit measurement (Abstract);
 * `if` statements decided at run time from the measured bits, with no branch
 * simulated ahead of time (Sec. III-C); `input` parameters resolved at run
 * time so that a kernel is compiled once and run many times (Sec. III-D);
 * energies <H> for VQE (Sec. IV-A.2, IV-D); repeated shots (Sec. IV-C).
 *
 * Conventions (the paper is silent on them):
 *   - qubit q is bit q of the amplitude index (little-endian); classical bit
 *     j is bit j of a 64-bit register (creg); unwritten bits read 0;
 *   - amplitudes are interleaved (re, im): SV_C64 = 2 x float, SV_C128 =
 *     2 x double, 2^n of them, contiguous;
 *   - a measurement of qubit q draws u = Philox4x64-10(key = (seed,
 *     stream_id), counter = (shot, m, 0, 0)) word 0, u = (w >> 11) * 2^-53,
 *     where m counts the measure/reset ops executed so far in the
 *     trajectory; outcome = 1 iff u >= p0/(p0+p1); the state is projected
 *     and scaled by 1/sqrt(p_outcome);
 *   - a terminal sample of shot s uses counter (s, 2^32, 0, 0) and returns
 *     the smallest index i with CDF_i > u * CDF_last.
 *
 * Errors: every call returns an sv_status and never throws; sv_last_error()
 * gives a thread-local message for the last failing call on the calling
 * thread.  After a failed call the handle stays valid but the state's
 * contents are undefined.
 *
 * Streams: every call that touches the GPU is enqueued on the stream bound
 * with sv_bind_stream (default: the legacy default stream) and returns
 * without waiting, unless it has a host output (creg_out, sample output,
 * expectation values, amplitudes), in which case it waits for that output.
 */
#ifndef LIBSV_SV_H_
#define LIBSV_SV_H_

#ifndef __CUDACC_RTC__
#include <stddef.h>
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { SV_C64 = 0, SV_C128 = 1 } sv_dtype;

typedef enum {
  SV_OK = 0,
  SV_ERR_ARG = -1,          /* invalid argument or malformed op list          */
  SV_ERR_OOM = -2,          /* device or host allocation failed               */
  SV_ERR_CUDA = -3,         /* a CUDA call failed                             */
  SV_ERR_TIMEOUT = -4,      /* a bounded device wait ran out                  */
  SV_ERR_UNSUPPORTED = -5,  /* valid but not supported (e.g. unroll too large)*/
  SV_ERR_NUMERIC = -6       /* a measurement saw a zero-norm state            */
} sv_status;

/* op kinds of the flat IR */
enum { SV_GATE = 1, SV_DENSE = 2, SV_MEASURE = 3, SV_RESET = 4, SV_COND = 5, SV_LOOP = 6 };

/* standard gates (OpenQASM 3 stdgates meanings; Sec. III-B maps them one-to-one) */
enum {
  SV_I = 0, SV_H, SV_X, SV_Y, SV_Z, SV_S, SV_SDG, SV_T, SV_TDG, SV_SX, SV_RX, SV_RY, SV_RZ,
  SV_P, SV_U, SV_CX, SV_CY, SV_CZ, SV_SWAP, SV_CP, SV_CRX, SV_CRY, SV_CRZ, SV_CH, SV_CU,
  SV_GATE_COUNT
};

/*
 * One record of the flat, pre-order IR (120 bytes).
 *   GATE    gate on q[0..] (controlled gates: q[0] control, q[1] target).
 *           Angle i = pidx[i] >= 0 ? angle[i] * params[pidx[i]] : angle[i]
 *           (U / CU use angles theta, phi, lambda).
 *   DENSE   nq-qubit unitary on q[0..nq-1] (nq <= 4), row-major 2^nq x 2^nq
 *           complex128 matrix at element dense_off of the dense pool
 *           (sv_set_dense_pool); local bit r of its index is qubit q[r].
 *   MEASURE measure q[0] into classical bit cbit (< 64).
 *   RESET   measure q[0] (no classical write; it consumes a draw), then X if 1.
 *   COND    run the next then_len records iff (creg & mask) == value, else the
 *           else_len records after them (predicate read when the COND is reached).
 *   LOOP    run the next body_len records loop_k times.
 * Lengths count flat records, nested headers and bodies included.
 */
typedef struct sv_op {
  uint16_t kind;
  uint16_t gate;
  uint32_t cbit;
  int32_t q[8];
  int32_t pidx[3];
  uint32_t nq;
  double angle[3];
  uint64_t mask, value;
  uint32_t then_len, else_len;
  uint32_t loop_k, body_len;
  uint64_t dense_off;
} sv_op;

/* Pauli string: X on q iff bit q of x_mask, Z iff bit q of z_mask, Y iff both. */
typedef struct sv_pauli {
  uint64_t x_mask, z_mask;
  double coeff;
} sv_pauli;

/* one executed measure/reset of the last run (debug and parity record) */
typedef struct sv_draw {
  int32_t qubit, is_reset, outcome, pad;
  double p0, p1, u; /* p0, p1 as the device saw them (unnormalised) */
} sv_draw;

typedef struct sv_state sv_state;     /* opaque, library-owned */
typedef struct sv_program sv_program; /* opaque lowered program (plan) */

typedef struct sv_program_stats {
  uint64_t records;       /* IR records                                   */
  uint64_t unrolled_ops;  /* gate + measure + reset ops after unrolling   */
  uint64_t gates;         /* gates after unrolling (counted in updates/s) */
  uint64_t draws;         /* measure + reset ops after unrolling          */
  uint64_t passes;        /* state sweeps per run (without init)          */
  uint64_t stages;        /* register stages over all passes              */
  uint64_t flags;         /* device predicate slots                       */
  int32_t tile_bits, low_bits;
  uint64_t plan_bytes;    /* bytes of plan data copied to the device      */
  int32_t specialised;    /* 1: passes run as kernels compiled for this program (sv_set_jit) */
  double compile_seconds; /* time spent compiling them                    */
  uint64_t block_barriers; /* per tile, summed over passes: block-wide barriers after the tile
                              copy and after each stage                      */
  uint64_t warp_barriers;  /* the same steps where a warp barrier suffices (every warp keeps
                              to its own amplitudes across the step; checked at lowering)  */
  uint64_t kernels_per_run; /* kernel launches of one sv_launch: matrix preparation, a separate
                               |0...0> sweep unless the first pass generates it, the passes */
} sv_program_stats;

/* Shot branching (sv_sample_branched, sv_batch_sample_branched). */
typedef struct sv_branch_stats {
  uint64_t shots;       /* shots sampled                                           */
  uint64_t paths;       /* trajectories simulated: one per distinct outcome path   */
  uint64_t levels;      /* walk rounds (each finds the paths of the next depth)    */
  uint64_t max_draws;   /* most draws on one path                                  */
} sv_branch_stats;

#ifndef __CUDACC_RTC__ /* device code compiled at run time needs the types above only */

/*
 * Create a state of n qubits (1 <= n <= 34) in |0...0>: the amplitude vector
 * that state-vector simulation of a circuit evolves (Sec. II-C, CUDA-Q's
 * state-vector backends; Sec. IV-A.2, state vectors compared for validation).
 *   dev_buf  NULL: the library allocates 2^n amplitudes on the current device.
 *            Otherwise caller-owned device memory of `bytes` >= 2^max(n,10) *
 *            amplitude size, which must outlive the handle (e.g. a torch tensor).
 * On success *out receives the handle.  SV_ERR_ARG for bad n/dtype/size,
 * SV_ERR_OOM if allocation fails.
 */
sv_status sv_create(int n, sv_dtype dtype, void* dev_buf, size_t bytes, sv_state** out);

/* Release the handle and everything the library allocated for it (not dev_buf).
 * Resource management of this library; the paper has no counterpart. */
sv_status sv_destroy(sv_state* h);

/* Enqueue all later work of h on this cudaStream_t (NULL: legacy default stream).
 * Resource management of this library; the paper has no counterpart.
 * SV_ERR_ARG for a null handle. */
sv_status sv_bind_stream(sv_state* h, void* cuda_stream);

/* Copy a host complex128 pool (interleaved re, im; n_complex entries) used by DENSE ops. */
sv_status sv_set_dense_pool(sv_state* h, const double* pool, size_t n_complex);

/*
 * How the planner picks each pass's tile qubits (the L contiguous low qubits
 * plus m - L gathered ones; a pass runs the gates, in order, whose qubits are
 * all tile qubits).  1 (default): the gathered qubits are chosen one at a time
 * (a pair when no single qubit helps) for the number of further gates they let
 * the pass run, so a program needs fewer passes; 0: first fit in program
 * order.  Programs planned from now on use it.  SV_ERR_ARG for a null handle.
 */
sv_status sv_set_tile_select(sv_state* h, int closure);

/*
 * How the planner packs a complex64 pass's gates into register stages.  A
 * stage whose four register bits include the tile's lowest bit moves its
 * amplitudes through shared memory as 16-byte pairs, half the access
 * instructions of one without it.  0 (default): the packing with the fewest
 * stages; 1 / 2: packings compared at a cost of 3/2 / 2 for a stage without
 * pair accesses against one with them.  Programs planned from now on use it.
 * SV_ERR_ARG for a null handle or a mode outside 0..2.
 */
sv_status sv_set_stage_pairs(sv_state* h, int mode);

/*
 * CTAs per SM the specialised pass kernels are compiled for (their register
 * budget follows: 65,536 / (256 x blocks) per thread) and launched with; 0
 * (default) keeps 2 for complex64 and 1 for complex128.  Programs planned
 * from now on use it.  SV_ERR_ARG for a null handle or a value outside 0..4.
 */
sv_status sv_set_jit_blocks(sv_state* h, int blocks_per_sm);

/*
 * Lower an op list for this state's n and dtype.  The caller's ops are read
 * during the call only.  SV_ERR_ARG for a malformed list (qubit >= n,
 * duplicate qubits, cbit >= 64, lengths out of range, nesting > 64),
 * SV_ERR_UNSUPPORTED if the unrolled program exceeds 2^22 ops or 2^20 predicates.
 * The program belongs to the caller (sv_program_free).  It launches on this
 * state only; once the state is destroyed, freeing it is the one valid call
 * (sv_launch then reports SV_ERR_ARG).
 */
sv_status sv_prepare(sv_state* h, const sv_op* ops, size_t n_ops, sv_program** out);

/*
 * Host-only lowering (no device touched): validates an op list for n qubits
 * and reports the plan statistics the given tuning would produce (tile_bits,
 * low_bits, max_pass_gates as in sv_set_tuning; 0 = default).
 */
sv_status sv_plan_info(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                       size_t n_complex, int tile_bits, int low_bits, int max_pass_gates, sv_program_stats* out);
sv_status sv_program_free(sv_program* p);
sv_status sv_program_info(const sv_program* p, sv_program_stats* out);

/*
 * Run one trajectory of a prepared program from |0...0> on the bound stream,
 * with parameters already on the device (dev_params: n_params doubles, may be
 * NULL if the program has no parameter references).  Asynchronous.  A
 * trajectory applies the gates, measures mid-circuit (the state collapses onto
 * the outcome, Sec. II-C, Fig. 2), resets, and decides each `if` from the
 * measured bits when it is reached, with no branch simulated ahead of time
 * (Sec. III-C); loops repeat a fixed number of times (Abstract); angles may
 * reference run-time `input` parameters, so one lowered program serves every
 * parameter set (Sec. III-D).  SV_ERR_ARG for a null handle or program, a
 * program prepared for another state, or fewer parameters than the program
 * references; SV_ERR_CUDA if a launch fails.
 */
sv_status sv_launch(sv_state* h, sv_program* p, const double* dev_params, size_t n_params,
                    uint64_t seed, uint64_t stream_id, uint64_t shot);

/*
 * Prepare (cached by content) + copy params to the device + launch, then if
 * creg_out is non-NULL wait and write the classical register there.  One
 * trajectory of the dynamic circuit as in sv_launch (Sec. II-C Fig. 2,
 * Sec. III-C, Sec. III-D).  ops and params (host memory) are read during the
 * call only.  Errors: those of sv_prepare and sv_launch; with creg_out,
 * SV_ERR_NUMERIC if a measurement met a zero-norm state and SV_ERR_TIMEOUT if
 * a bounded device wait ran out.
 */
sv_status sv_run(sv_state* h, const sv_op* ops, size_t n_ops, const double* params, size_t n_params,
                 uint64_t seed, uint64_t stream_id, uint64_t shot, uint64_t* creg_out);

/* Classical register and draw record of the last run (waits for it). */
sv_status sv_get_creg(sv_state* h, uint64_t* creg);
sv_status sv_get_trace(sv_state* h, sv_draw* out, size_t max, size_t* n_out);

/*
 * `shots` shots of a program (repeated shots of a dynamic circuit, Sec. IV-C:
 * the conditional reset checked over 10^4 shots).  With MEASURE/RESET in the program, shot s runs
 * its own trajectory (counter shot = s) and creg_out[s] receives its
 * register; otherwise the program runs once.  bits_out (nullable) receives
 * one terminal sample per shot (counter (s, 2^32)).  Waits for the outputs.
 */
sv_status sv_sample(sv_state* h, const sv_op* ops, size_t n_ops, const double* params, size_t n_params,
                    uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t* creg_out,
                    uint64_t* bits_out);

/*
 * Shot branching: creg_out[s] (s < shots) receives exactly the register that
 * sv_sample on this state gives shot s, but only one trajectory runs per
 * distinct outcome path among the shots.  Shots that agree on their first k
 * outcomes hold the same state, so each of their next draws compares its own
 * Philox number with the same (p0, p1); a representative trajectory records
 * those masses and a device walk routes every shot down the tree of paths
 * (Sec. III-C: outcomes are still decided per shot at run time).  stats
 * (nullable) reports shots, paths, walk rounds and the longest path.
 * SV_ERR_UNSUPPORTED when a trajectory executes more than 4096 draws or
 * shots >= 2^32 - 1; SV_ERR_NUMERIC as for sv_run.  The state holds the last
 * representative's final state afterwards.  Device scratch (8 bytes per shot
 * plus 24 bytes per recorded draw) is allocated on first use, grows as needed
 * and is kept with the handle.  Waits for the output.
 */
sv_status sv_sample_branched(sv_state* h, const sv_op* ops, size_t n_ops, const double* params, size_t n_params,
                             uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t* creg_out,
                             sv_branch_stats* stats);

/* Terminal samples of the current state: out[s] for counter (shot0 + s, 2^32)
 * (measurement of every qubit at the end of a shot, Sec. IV-C).  out is a host
 * array of `shots` indices; waits for it.  SV_ERR_ARG for a null handle or
 * output. */
sv_status sv_sample_state(sv_state* h, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                          uint64_t* out);

/*
 * sv_sample_state with the samples left on the device: dev_out is a
 * caller-owned device array of `shots` uint64 indices.  Asynchronous on the
 * bound stream (for consumers on the GPU, e.g. a torch tensor); while
 * profiling (sv_profile) its kernels are timed as one launch.  The two-level
 * CDF scratch (8 bytes per 32 amplitudes plus 16 per 8,192) is allocated on
 * first use and kept with the handle.  SV_ERR_ARG for a null handle or
 * output, SV_ERR_CUDA on a launch error.
 */
sv_status sv_sample_state_device(sv_state* h, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                                 uint64_t* dev_out);

/*
 * <psi| sum_t coeff_t P_t |psi> of the current state (sums of 1,024 pairs in
 * the state precision, accumulated in double-float for complex64 and in FP64
 * for complex128, per-term results and the total in FP64): the
 * energy <H> of a Hamiltonian given as a Pauli sum, as in the VQE experiments
 * (Sec. II-D; Sec. IV-A.2, H = Z0 Z1; Sec. IV-D).  terms is a host array read
 * during the call; total (nullable) receives the sum, per_term (nullable,
 * n_terms host doubles) each <P_t>.  Waits for the result.  SV_ERR_ARG for a
 * null handle or terms, or a term on a qubit >= n.
 */
sv_status sv_expval(sv_state* h, const sv_pauli* terms, size_t n_terms, double* total, double* per_term);

/*
 * Pauli expectation values that allocate no device memory.  The paper has no
 * counterpart to this entry point; it exists for callers that cannot let a
 * library call cudaMalloc: applications whose device memory is entirely
 * handed out by their own allocator or a fixed pool, and latency-critical
 * loops that cannot afford cudaMalloc's implicit synchronisation with the
 * device.  sv_expval allocates its scratch; this variant keeps it in a
 * static array inside the library's device image instead (262,400 bytes on
 * every GPU that loads libsv, held until the process exits).
 *
 *   dev_state  device pointer to 2^n amplitudes of `dtype` (16-byte aligned),
 *              e.g. the buffer of a state created with sv_create; read only.
 *   terms      host array of n_terms Pauli strings, read during the call;
 *              n_terms <= 64 (larger requests return SV_ERR_ARG).
 *   dev_out    caller-owned device array of n_terms doubles; receives
 *              <P_t> for each term (no coefficient applied), in term order.
 *   cuda_stream  stream to enqueue on (NULL: legacy default stream).
 * Asynchronous: it returns once the work is enqueued.  The first call on a
 * device looks up the static array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.
 * The address is kept for the life of the process: do not call it again on a
 * device that was reset with cudaDeviceReset.  dev_state and dev_out must be
 * device (or managed) memory of the current device.
 * Every call shares the one array, so calls that overlap on the GPU (e.g.
 * on different streams) race and give wrong results; calls in stream order
 * are safe.  Errors: SV_ERR_ARG for bad n, dtype, pointers (null, not device
 * memory, or on another device), alignment or term count; SV_ERR_CUDA if a
 * launch fails (message in sv_last_error()).
 */
sv_status sv_expval_static(const void* dev_state, int n, sv_dtype dtype, const sv_pauli* terms, size_t n_terms,
                           double* dev_out, void* cuda_stream);

/*
 * Batched execution: many trajectories, of uneven qubit counts, in one
 * persistent kernel launch (replayed from a CUDA graph).  Each CTA of the
 * launch takes the next trajectory from a device work queue (longest first),
 * runs its whole program on a private state slot -- feed-forward decided on
 * the device -- and stores the classical register; trajectory t uses Philox
 * stream stream_ids[t] and shot shots[t], so its record equals that of
 * sv_run with the same (seed, stream_id, shot).  States are padded to at
 * least 12 qubits.
 *
 * sv_batch_create        handle for one dtype; work is enqueued on cuda_stream.
 * sv_batch_add_program   lowers an op list for n qubits with its parameters
 *                        (copied; n_params doubles) and optional dense pool;
 *                        *prog_id receives its index.
 * sv_batch_set_items     the batch: n_items trajectories (program, stream id,
 *                        shot); allocates the device work space (one state
 *                        slot of 2^max(n) amplitudes per resident CTA).
 * sv_batch_launch        asynchronous run of the current items.
 * sv_batch_results       waits and copies the n_items classical registers.
 * sv_batch_run           set_items + launch + results.
 * Errors: SV_ERR_ARG for bad ids or sizes, SV_ERR_OOM when the work space
 * does not fit, SV_ERR_NUMERIC if a trajectory met a zero-norm state.
 */
typedef struct sv_batch sv_batch;
sv_status sv_batch_create(sv_dtype dtype, void* cuda_stream, sv_batch** out);
sv_status sv_batch_add_program(sv_batch* b, int n, const sv_op* ops, size_t n_ops, const double* params,
                               size_t n_params, const double* dense_pool, size_t n_complex, uint32_t* prog_id);
sv_status sv_batch_set_items(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids, const uint64_t* shots,
                             size_t n_items);
sv_status sv_batch_launch(sv_batch* b, uint64_t seed);
sv_status sv_batch_results(sv_batch* b, uint64_t* creg_out);
sv_status sv_batch_run(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids, const uint64_t* shots,
                       size_t n_items, uint64_t seed, uint64_t* creg_out);
sv_status sv_batch_destroy(sv_batch* b);

/*
 * Planner tuning of the programs added to the batch after this call: the
 * tile is fixed at 2^12 amplitudes by the batched kernel; low_bits (3..12,
 * contiguous low qubits of a tile) and max_pass_gates (0..128, gates fused
 * into one pass) as in sv_set_tuning; 0 = default.  SV_ERR_ARG out of range.
 */
sv_status sv_batch_set_tuning(sv_batch* b, int low_bits, int max_pass_gates);


/*
 * Clifford fast path: programs whose gates are all Clifford (I, H, X, Y, Z,
 * S, SDG, SX, CX, CY, CZ, SWAP) with MEASURE, RESET, COND and LOOP records,
 * on 1 <= n <= 64 qubits, sampled by stabilizer tableaux (Aaronson and
 * Gottesman 2004) instead of state vectors: one warp per shot, 2n Pauli rows
 * in registers.  The paper's static suite is random Clifford circuits (Sec.
 * IV-A.2), run there on a stabilizer backend (Fig. 1c).
 *   sv_clifford_create   lowers the op list (COND to jumps, LOOP unrolled, at
 *                        most 2^24 instructions) and uploads it; work is
 *                        enqueued on cuda_stream (NULL: legacy default stream).
 *                        SV_ERR_UNSUPPORTED for a non-Clifford gate or a DENSE
 *                        record, SV_ERR_ARG for bad qubits, bits or lengths.
 *   sv_clifford_sample   creg_out[s] (host, `shots` entries) = the register of
 *                        shot shot0 + s; draw m of a shot uses Philox counter
 *                        (shot, m) as in sv_run, and a random outcome is 1 iff
 *                        u >= 1/2, so records equal sv_sample's except where the
 *                        state vector's rounded p0/(p0+p1) and 1/2 straddle u.
 *                        Waits for the output.
 *   sv_clifford_destroy  frees the handle.
 */
typedef struct sv_clifford sv_clifford;
sv_status sv_clifford_create(int n, const sv_op* ops, size_t n_ops, void* cuda_stream, sv_clifford** out);
sv_status sv_clifford_sample(sv_clifford* c, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                             uint64_t* creg_out);
sv_status sv_clifford_destroy(sv_clifford* c);

/*
 * Shot branching on the batched engine: n_requests requests, request r
 * running program prog_ids[r] with Philox stream stream_ids[r] for
 * n_shots[r] shots (counters 0 .. n_shots[r]-1).  creg_out receives the
 * records request after request (sum of n_shots entries), each equal to
 * the record sv_batch_run gives that (program, stream, shot).  The
 * representatives of each walk round run together in one persistent
 * launch.  Replaces the batch's current items.  Besides the walk's scratch,
 * the first call allocates 4,096 draw records per resident CTA (128 KiB each)
 * and keeps them with the handle.  Errors as for sv_sample_branched and
 * sv_batch_run.
 */
sv_status sv_batch_sample_branched(sv_batch* b, const uint32_t* prog_ids, const uint64_t* stream_ids,
                                   const uint64_t* n_shots, size_t n_requests, uint64_t seed, uint64_t* creg_out,
                                   sv_branch_stats* stats);

/*
 * Energies and adjoint gradients of <H> = sum_t coeff_t <psi(theta)|P_t|psi(theta)>
 * for many parameter sets of one static parameterised program (the VQE loop
 * of Sec. IV-D: one lowered program, new parameters each call).  The program
 * may contain gates and DENSE unitaries on <= 3 qubits only (no MEASURE,
 * RESET, COND); parameters enter angles as scale * theta[pidx].
 *
 * sv_grad_create   lowers the program for n qubits and copies the Pauli terms.
 * sv_grad_run      device pointers: params [P][n_params] doubles; writes
 *                  val [P] (energies) and grad [P][n_params] (dE/dtheta),
 *                  asynchronously on the handle's stream.  One persistent
 *                  launch: each CTA runs whole parameter sets (forward sweep,
 *                  lambda = H psi, backward sweep with the derivative
 *                  accumulations); per-warp derivative sums in
 *                  double-float (complex64) or FP64, gradient entries and
 *                  energies in FP64.
 * sv_expval_grad_batch  the same with host arrays, waiting for the result.
 * Errors: SV_ERR_ARG (bad sizes or masks, n_params below the largest index
 * referenced, more than 1024 parameters), SV_ERR_UNSUPPORTED (program with
 * measurement / control flow / 4-qubit dense gates), SV_ERR_OOM.
 */
typedef struct sv_grad sv_grad;
sv_status sv_grad_create(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                         size_t n_complex, const sv_pauli* terms, size_t n_terms, void* cuda_stream, sv_grad** out);
sv_status sv_grad_run(sv_grad* g, const double* dev_params, size_t n_sets, size_t n_params, double* dev_val,
                      double* dev_grad);
sv_status sv_grad_destroy(sv_grad* g);
/* 1 (default): sv_grad_run compiles, at its first call, a kernel specialised
 * to this program (every gate, register position and shared-memory address a
 * constant; the per-set matrices stay run-time data) and runs it; 0: the
 * generic kernel, which reads the gate records at run time.  If the
 * specialised kernel cannot be built the generic one runs.  SV_ERR_ARG for a
 * null handle. */
sv_status sv_grad_set_jit(sv_grad* g, int enable);
/* Shape of the work of one parameter set (for throughput and roofline
 * accounting): forward and backward state passes, gates, Pauli term groups
 * (one gather of the state each while lambda = H psi is formed), terms, the
 * state's qubits after padding, the parameter sets resident at once (one per
 * CTA, for the kernel the next run uses), whether that kernel is the
 * specialised one, and its compile time in seconds.  SV_ERR_ARG for a null
 * argument. */
typedef struct sv_grad_stats {
  uint64_t forward_passes, backward_passes, gates;
  uint32_t term_groups, terms, state_qubits, resident_sets;
  uint32_t specialised, pad;
  double compile_seconds;
} sv_grad_stats;
sv_status sv_grad_info(const sv_grad* g, sv_grad_stats* out);
sv_status sv_expval_grad_batch(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* params,
                               size_t n_sets, size_t n_params, const sv_pauli* terms, size_t n_terms, double* val_out,
                               double* grad_out, void* cuda_stream);

/* Copy amplitudes [first, first+count) to / from host memory (amplitude-size
 * elements: 8 bytes for SV_C64, 16 for SV_C128), waiting for the copy: the
 * state vector itself, which the paper's validation compares between
 * simulators (Sec. III-E, Sec. IV-A.2).  The host buffer is the caller's.
 * SV_ERR_ARG for a null handle or pointer or a range beyond 2^n. */
sv_status sv_get_amplitudes(sv_state* h, void* host_dst, size_t first, size_t count);
sv_status sv_set_amplitudes(sv_state* h, const void* host_src, size_t first, size_t count);

/* Device pointer and byte size of the state (for zero-copy views). */
sv_status sv_state_buffer(sv_state* h, void** dev_ptr, size_t* bytes);

/* Planner tuning: tile bits (10..14), contiguous low bits (2..tile), max gates per pass; 0 = default. */
sv_status sv_set_tuning(sv_state* h, int tile_bits, int low_bits, int max_pass_gates);

/*
 * Kernel timing and work counts of the state-sweep passes.  While enabled,
 * every pass launch is bracketed by CUDA events on the bound stream, and the
 * pass kernels themselves count on the device what they did: bytes of the
 * state read (tiles copied in; tiles that a pending projector zeroes, and the
 * first pass that generates |0...0>, read nothing), bytes written (tiles
 * stored; a pass whose gates were all predicated off, or a final flush with
 * no projector pending, writes nothing), gate records executed (gates of
 * not-taken if/else arms excluded), draws executed and passes that touched
 * the state.  sv_profile_read waits, then reports the summed event time (ms),
 * the number of pass launches and the bytes read + written, and resets the
 * timing and the counters.  sv_profile_work reads the counters without
 * resetting them.  Enabling zeroes the counters.  Errors: SV_ERR_ARG for a
 * null handle or output, SV_ERR_CUDA if a copy fails.
 */
#define SV_WORK_COUNTERS 8
typedef struct sv_work_counts {
  uint64_t bytes_read, bytes_written; /* state bytes moved by the pass kernels     */
  uint64_t gates;                     /* gate records executed                       */
  uint64_t draws;                     /* measure / reset draws executed              */
  uint64_t passes;                    /* pass launches that read or wrote the state  */
  uint64_t updates;                   /* amplitude-gate updates: (gates + draws) x 2^n */
} sv_work_counts;
sv_status sv_profile(sv_state* h, int enable);
sv_status sv_profile_read(sv_state* h, double* total_ms, uint64_t* launches, double* bytes);
sv_status sv_profile_work(sv_state* h, sv_work_counts* out);

/* Work counters of the batched launches (see sv_profile_work): while enabled,
 * every trajectory's passes count on the device the state bytes they read and
 * wrote (state slots, often resident in L2 for small n), the gate records and
 * draws they executed and the amplitude-gate updates (2^n per executed gate
 * or draw, n the trajectory's padded qubit count).  Enabling zeroes the
 * counters; sv_batch_work waits for the batch's stream and reads them.
 * SV_ERR_ARG for a null argument. */
sv_status sv_batch_profile(sv_batch* b, int enable);
sv_status sv_batch_work(sv_batch* b, sv_work_counts* out);

/* 1: launches run a kernel specialised to the handle's programs (every gate,
 * register position and shared-memory address of every pass a constant; the
 * per-program matrices and flags stay run-time data), compiled at the first
 * launch after programs were added (about 45 s for nine programs of 13-21
 * qubits with 228 passes in all, less for fewer or shorter programs; suited
 * to a fixed program set run many times, not to a serving loop that adds
 * programs as requests arrive); if it cannot be built the generic kernel
 * runs.  0 (default): the generic kernel, which reads the gate records at run
 * time.  sv_batch_jit_info: whether the next launch runs the specialised
 * kernel (built and current) and its compile time.  SV_ERR_ARG for a null
 * handle. */
sv_status sv_batch_set_jit(sv_batch* b, int enable);
sv_status sv_batch_jit_info(sv_batch* b, int* specialised, double* compile_seconds);

/*
 * Self test of the failure path of bounded device waits (the tensor-core
 * completion wait of the sweep kernels).  Runs that same wait -- mbarrier
 * try_wait polled at most `polls` times -- in a one-warp kernel on the bound
 * stream, on an mbarrier that nothing ever arrives at, so it always runs out.
 * The kernel issues no MMA and allocates no tensor memory; the outcome reaches
 * the caller exactly as a timed-out pass reports it: the control block's
 * status, read back by the host.  Returns SV_ERR_TIMEOUT (the expected
 * outcome; the handle stays usable and the next run starts clean),
 * SV_ERR_ARG for a null handle or polls > 2^24, SV_ERR_CUDA on a launch error.
 * The paper has no counterpart: it describes no device waits.
 */
sv_status sv_selftest_wait(sv_state* h, uint32_t polls);

/*
 * Program cache of sv_run / sv_sample (on by default): a repeated op list
 * reuses its lowered plan.  With the cache off every call lowers the list
 * and copies the plan to the device again.
 */
sv_status sv_set_cache(sv_state* h, int enable);

/*
 * Per-program specialisation of the sweep kernels (off by default).  With it
 * on, the first launch of a program compiles (NVRTC, sm_103a) one kernel per
 * pass in which gate kinds, register positions and shared-memory addresses
 * are constants; gate matrices and predicates stay run-time data.  If
 * compilation fails the program keeps the generic kernels and
 * sv_program_info reports specialised = 0.
 */
sv_status sv_set_jit(sv_state* h, int enable);

/*
 * Dense four-qubit unitaries (DENSE records on 4 qubits) on the tensor cores
 * (on by default).  Applies to complex64 states swept in 2^12-amplitude tiles
 * (the default), generic and specialised kernels: each such gate becomes a
 * 2^(n-4) x 32 by 32 x 32 real product (the 32 x 32 real form of the 16 x 16
 * complex unitary) on kind::tf32 MMAs, each operand split into a TF32 high
 * and low part with three products accumulated in FP32 (FP32-level accuracy).
 * Off, or in other configurations, the gate runs on the FP32 / FP64 pipes.
 * The paper gives no kernel for dense gates; this is a GB300 design choice.
 * SV_ERR_ARG for a NULL handle.  A tensor-core completion wait that runs out
 * makes the run report SV_ERR_TIMEOUT.
 */
sv_status sv_set_dense_tc(sv_state* h, int enable);

/*
 * Host-only check of the specialiser (no device touched): lowers the op list
 * and compiles its specialised module to a cubin.  The first log_len - 1 bytes
 * of the compiler log are copied to log (nullable): on failure the errors, on
 * success the ptxas resource report (registers, spill bytes, stack) of every
 * compiled chunk.
 */
sv_status sv_jit_check(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                       size_t n_complex, char* log, size_t log_len);
/* The same for the adjoint kernel specialised to a program (sv_grad_run's
 * default): lowers the forward and backward plans and compiles the module.
 * Errors as sv_grad_create's lowering, or SV_ERR_CUDA with the compiler log. */
sv_status sv_jit_check_adjoint(int n, sv_dtype dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                               size_t n_complex, char* log, size_t log_len);
/* The same for the batched kernel specialised to n_progs programs (as
 * sv_batch_set_jit builds it): program k has n[k] qubits and ops[k] (n_ops[k]
 * records, no dense gates), all lowered with the batched engine's 2^12-amplitude
 * tiles.  Host arrays, read during the call.  SV_ERR_ARG for empty or null
 * arrays or a malformed program, SV_ERR_CUDA with the compiler log. */
sv_status sv_jit_check_batch(sv_dtype dtype, size_t n_progs, const int* n, const sv_op* const* ops,
                             const size_t* n_ops, char* log, size_t log_len);

/* Wait for all work of h.  Resource management of this library; the paper
 * has no counterpart.  SV_ERR_CUDA if earlier asynchronous work failed. */
sv_status sv_sync(sv_state* h);

/* Thread-local message of the last error on this thread ("" if none). */
const char* sv_last_error(void);

/* Library version string. */
const char* sv_version(void);

#endif /* __CUDACC_RTC__ */

#ifdef __cplusplus
}
#endif

#endif /* LIBSV_SV_H_ */
