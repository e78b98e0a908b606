// sv_plan.h -- plan records shared by the host planner and the CUDA kernels.
//
// A program (the flat IR of include/sv.h) is lowered once into:
//   * matrix jobs   -- one per gate, evaluated on the device from the run-time
//                      parameters (OpenQASM `input` values, Sec. III-D), so a
//                      plan is compiled once and run with many parameter sets;
//   * passes        -- sweeps over the whole state.  A pass holds a tile of 2^m
//                      amplitudes (m tile qubits: the L lowest qubits plus m-L
//                      gathered higher ones) in shared memory, applies every gate
//                      of the pass in register-resident stages of four qubits,
//                      and optionally accumulates the |amp|^2 table of up to four
//                      measured qubits for the measurement group that follows;
//   * scalar items  -- measure / reset / cond-evaluation records run by one
//                      thread after a pass (the device-side feed-forward of
//                      Sec. III-C: predicates are read from the classical record
//                      on the GPU, never on the host).
#pragma once
#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

namespace svp {

enum OpCode : uint8_t {
  OP_NONE = 0,
  OP_U,     // general 2x2 complex on p0: 4 complex
  OP_R,     // real 2x2 on p0: [r00 r01; r10 r11] stored as 4 complex (re only)
  OP_RX,    // [c, -is; -is, c]: stored as (c, s)
  OP_D,     // diag(d0, d1) on p0: 2 complex
  OP_X,     // swap halves of p0
  OP_CU,    // control p0, target p1, 2x2 complex: 4 complex
  OP_CX,    // control p0, target p1
  OP_CZ,    // phase -1 where p0 and p1 are both 1
  OP_CD,    // control p0, target p1: diag(d0, d1) where control is 1: 2 complex
  OP_SWAP,  // swap p0 <-> p1
  OP_U4,    // dense 4x4 on (p0 = local bit 0, p1 = local bit 1): 16 complex
  OP_D16,   // dense 16x16 on the four register bits: 256 complex
  // adjoint (backward) stages only: Re <lambda| M |phi> with phi in registers 0..7 and
  // lambda in registers 8..15, accumulated for one gradient entry; M = dU/da * U^dagger
  OP_DOT,   // M (4 complex) on p0
  OP_CDOT,  // M on target p1 where control p0 is 1
  // forward plans only: one-qubit rotations with a scalar factor taken out, so
  // that one matrix entry per row is 1 (two FP operations per amplitude
  // instead of four); the pass multiplies the product of the factors of its
  // active gates into the state once, when it stores the tile
  OP_RXF,   // RX = f [1 -it; -it 1] (form 0) or f [u -i; -i u] (form 1): (k, form), (f)
  OP_RYF,   // RY = f [1 -t; t 1] (form 0) or f [u -1; 1 u] (form 1): (k, form), (f)
  OP_DZ,    // diag(d0, d1) = d0 diag(1, p): (p), (d0)
  OP_COUNT
};

#ifndef __CUDACC_RTC__
// number of complex matrix entries each op reads
static inline int op_mat_len(int op) {
  switch (op) {
    case OP_U: case OP_R: case OP_CU: case OP_DOT: case OP_CDOT: return 4;
    case OP_RX: case OP_D: case OP_CD: case OP_RXF: case OP_RYF: case OP_DZ: return 2;
    case OP_U4: return 16;
    case OP_D16: return 256;
    default: return 0;
  }
}
#endif

enum ScalarKind : uint8_t { S_MEASURE = 1, S_RESET = 2, S_COND = 3 };

enum JobKind : uint8_t {
  J_GATE = 1,   // gate matrix from its angles (adj = 1: its conjugate transpose)
  J_CONST = 2,  // copy from the constant pool
  J_DERIV = 3   // scale * (dU/d angle[slot]) * U^dagger of a one-qubit / controlled gate
};

constexpr int REG_BITS = 4;
constexpr int REG_N = 16;
constexpr int PASS_THREADS = 256;
constexpr int MAX_TILE_BITS = 14;
constexpr int MAX_GROUP_Q = 4;
constexpr int MAX_PASS_GATES = 128;
constexpr int MAX_PASS_MAT = 1024;  // complex entries staged in shared memory per pass (four dense 16 x 16)
constexpr int MAX_TRACE = 4096;     // draw records kept per trajectory
constexpr int ADJ_REG_BITS = 3;     // gate register bits of a backward stage (bit 3 selects phi / lambda)
constexpr int MAX_PASS_DOTS = 64;   // derivative accumulators per backward pass
constexpr int MAX_ADJ_PARAMS = 1024;

// gate as the kernel sees it: positions are register-bit indices (0..3) of its stage
struct DGate {
  uint16_t key;   // op * 16 + p0 * 4 + p1 (9 bits): one switch selects op and positions
  uint8_t op, p0, p1, pad0;
  uint16_t dslot; // OP_DOT / OP_CDOT: accumulator slot within the pass
  int32_t flag;   // -1: unconditional; else index into the flag array
  uint32_t mat;   // offset (complex entries) from the pass's matrix base
  uint32_t gidx;  // OP_DOT / OP_CDOT: gradient entry (parameter index)
  uint32_t pad3;
};
// a gate record in a kernel's shared list: key | active << SGK_ON_BIT | matrix offset << 16
constexpr uint32_t SGK_KEY = 0x1FFu;
constexpr int SGK_ON_BIT = 9;
constexpr uint32_t SGK_ON = 1u << SGK_ON_BIT;

// Register stage.  The tile is stored XOR-swizzled in shared memory (see
// tile_swizzle); because the swizzle is linear over GF(2), the address of a
// tile-local index is the XOR of the addresses of its set bits.  R[r] is the
// address of register bit r, E[k] that of group-index bit k.
struct DStage {
  uint16_t g0, ng;                       // gate range (pass-relative)
  uint16_t R[REG_BITS];
  uint16_t E[MAX_TILE_BITS - REG_BITS];  // E[5..7] select the warp (tiles of >= 12 bits)
  uint16_t bar;                          // 1: block barrier after the stage, 0: warp barrier suffices
  uint8_t Rb[REG_BITS];                  // the tile bits behind R and E (unswizzled)
  uint8_t Eb[MAX_TILE_BITS - REG_BITS];
};

// Shared-memory layout of a tile, in 16-byte granules (one complex128 or two
// complex64 amplitudes): granule g lives at g ^ fold(g >> 3), fold = XOR of
// the 3-bit groups, so the 8 granules of every 128-byte row are permuted by
// the higher index bits.  A = log2(amplitudes per granule) (1 for complex64,
// 0 for complex128); amplitude pairs of complex64 stay adjacent, so a
// 16-byte copy moves a granule verbatim.  The map is linear over GF(2).
#ifndef __CUDACC_RTC__
static inline uint32_t tile_swizzle(uint32_t x, int A) {
  uint32_t y = x >> (A + 3), f = 0;
  for (int k = 0; k < 5; ++k) {
    f ^= y & 7u;
    y >>= 3;
  }
  return x ^ (f << A);
}
#endif

struct DScalar {
  uint8_t kind;     // ScalarKind
  uint8_t tbit;     // MEASURE/RESET: bit of the qubit in the pass's group table
  uint16_t pad;
  int32_t flag;     // MEASURE/RESET: own flag; COND: parent flag (-1: none)
  int32_t f_then;   // COND: flag receiving the then-predicate
  int32_t f_else;   // COND: flag receiving the else-predicate (-1: none)
  uint32_t qubit;   // MEASURE/RESET: qubit (physical bit)
  uint32_t cbit;    // MEASURE: classical bit
  uint32_t pad2;
  uint64_t mask, value;  // COND predicate
};

struct DPass {
  uint32_t g0, ng;        // gates
  uint32_t s0, ns;        // stages
  uint32_t c0, nc;        // scalar items run after the pass
  uint32_t mat0, nmat;    // matrix range (complex entries) in the matrix pool
  uint8_t m, L;           // tile bits, contiguous low bits
  uint8_t gk;             // group table bits (0: no table)
  uint8_t kin;            // how many of the group bits are tile bits (table bits 0..kin-1)
  uint8_t group_always;   // 1: the table is needed whatever the flags say
  uint8_t flush;          // 1: final pass that only applies a pending projector
  uint8_t bar_in;         // 1: block barrier between the tile copy and the first stage
  uint8_t dense;          // 1: the pass holds a dense four-qubit gate (OP_D16)
  uint8_t proj;           // 1: a measurement projector may be pending when the pass starts
  uint8_t direct;         // 1: specialised kernels store the tile from the last stage's registers
  uint8_t pad[2];
  uint8_t tq[MAX_TILE_BITS];      // qubit at tile-local bit j (ascending for j >= L)
  uint8_t outer_gq[MAX_GROUP_Q];  // table bit kin+i <- qubit outer_gq[i] (outside the tile)
  uint16_t red_R[REG_BITS];       // reduction stage: register-bit addresses
  uint16_t red_E[MAX_TILE_BITS - REG_BITS];  // reduction stage: group-index-bit addresses
};

struct DJob {
  uint8_t kind;     // JobKind
  uint8_t op;       // OpCode the matrix is laid out for
  uint8_t gate;     // IR gate enum (J_GATE, J_DERIV)
  uint8_t adj;      // J_GATE: 1 = write the conjugate transpose
  
  int32_t pidx[3];
  double angle[3];
  uint32_t out;     // offset (complex entries) into the matrix pool
  uint32_t src;     // J_CONST: offset into the constant pool (complex entries)
  uint32_t len;     // J_CONST: entries to copy; J_DERIV: angle slot
  uint32_t pad2;
};

// per-trajectory control block on the device
struct Ctrl {
  uint64_t creg;
  uint64_t seed, stream, shot;
  uint64_t m;                 // draws executed
  uint64_t pm, pv, px;        // pending projector: a'[i] = ps * a[i ^ px] if ((i ^ px) & pm) == pv
  double ps;
  uint32_t ticket;            // last-CTA-done counter of the running pass
  int32_t status;             // 0 ok, else an sv_status
  uint32_t n_trace;
  uint32_t pad;
};

struct DTrace {
  int32_t qubit, is_reset, outcome, pad;
  double p0, p1, u;
};

}  // namespace svp
