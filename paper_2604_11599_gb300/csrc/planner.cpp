// planner.cpp -- lowering of the flat IR (include/sv.h) into device passes.
//
// 1. Unroll: COND/LOOP records are interpreted into a straight item list in
//    which every gate/measure/reset carries the predicate flag of its
//    enclosing branch and every COND becomes a flag-evaluation item.  The
//    flags are evaluated on the device from the classical register when the
//    COND is reached, so branches are decided by feed-forward on the GPU and
//    never duplicated into outcome-specific copies (Sec. III-C); loops
//    (Abstract: loops with a fixed trip count) are repeated.
// 2. Segment: a measurement group is a run of measure/reset items with no
//    gate between them on at most four distinct qubits.  The gates before a
//    group are swept in passes; the last pass also accumulates the group's
//    joint |amp|^2 table, and the group's draws, plus every COND evaluation
//    up to the next group (the register cannot change in between), run as
//    the scalar phase after that pass.
// 3. Fuse: gates are packed greedily (in dependency order) into passes whose
//    tile holds m qubits (the L lowest plus gathered higher ones), and each
//    pass into stages of four register qubits.
#include "planner.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

namespace svp {
namespace {

enum ItemKind { I_GATE = 0, I_MEAS, I_RESET, I_COND };

struct Item {
  ItemKind kind = I_GATE;
  int flag = -1;  // predicate flag of the enclosing branch; COND: parent flag
  // gates
  uint8_t op = OP_NONE;
  int nq = 0;
  int q[4] = {-1, -1, -1, -1};
  int gate = -1;  // IR gate, or -1 for a dense record
  int32_t pidx[3] = {-1, -1, -1};
  double angle[3] = {0, 0, 0};
  const double* dense = nullptr;  // row-major 2^k x 2^k complex (re, im)
  // measure / reset
  int qubit = -1;
  uint32_t cbit = 0;
  // cond
  int f_then = -1, f_else = -1;
  uint64_t mask = 0, value = 0;

  uint64_t qmask() const {
    uint64_t m = 0;
    for (int i = 0; i < nq; ++i) m |= 1ull << q[i];
    return m;
  }
};

int gate_qubits(int g) { return (g >= SV_CX && g <= SV_CU) ? 2 : 1; }

uint8_t gate_opcode(int g) {
  switch (g) {
    case SV_I: return OP_NONE;
    case SV_H: case SV_RY: return OP_R;
    case SV_X: return OP_X;
    case SV_Y: case SV_SX: case SV_U: return OP_U;
    case SV_RX: return OP_RX;
    case SV_Z: case SV_S: case SV_SDG: case SV_T: case SV_TDG: case SV_P: case SV_RZ: return OP_D;
    case SV_CX: return OP_CX;
    case SV_CZ: return OP_CZ;
    case SV_SWAP: return OP_SWAP;
    case SV_CY: case SV_CH: case SV_CRX: case SV_CRY: case SV_CU: return OP_CU;
    case SV_CP: case SV_CRZ: return OP_CD;
    default: return OP_COUNT;
  }
}

struct Unroller {
  const sv_op* ops = nullptr;
  size_t n_ops = 0;
  int n = 0;
  const double* pool = nullptr;
  size_t pool_len = 0;
  std::vector<Item> items;
  uint32_t n_flags = 0;
  uint64_t max_param = 0;
  sv_status st = SV_OK;
  std::string err;
  static constexpr size_t kMaxItems = size_t(1) << 22;
  static constexpr uint32_t kMaxFlags = 1u << 20;

  bool fail(sv_status s, const std::string& m) {
    if (st == SV_OK) {
      st = s;
      err = m;
    }
    return false;
  }
  bool qok(int32_t q) const { return q >= 0 && q < n; }

  bool walk(size_t begin, size_t end, int flag, int depth) {
    if (depth > 64) return fail(SV_ERR_ARG, "COND/LOOP nesting deeper than 64");
    size_t i = begin;
    while (i < end) {
      const sv_op& o = ops[i];
      switch (o.kind) {
        case SV_GATE: {
          if (o.gate >= SV_GATE_COUNT) return fail(SV_ERR_ARG, "unknown gate at record " + std::to_string(i));
          Item it;
          it.kind = I_GATE;
          it.flag = flag;
          it.gate = o.gate;
          it.op = gate_opcode(o.gate);
          it.nq = gate_qubits(o.gate);
          for (int k = 0; k < it.nq; ++k) {
            if (!qok(o.q[k])) return fail(SV_ERR_ARG, "qubit out of range at record " + std::to_string(i));
            it.q[k] = o.q[k];
          }
          if (it.nq == 2 && it.q[0] == it.q[1]) return fail(SV_ERR_ARG, "repeated qubit at record " + std::to_string(i));
          for (int k = 0; k < 3; ++k) {
            it.pidx[k] = o.pidx[k];
            it.angle[k] = o.angle[k];
            if (o.pidx[k] >= 0) max_param = std::max<uint64_t>(max_param, uint64_t(o.pidx[k]) + 1);
          }
          if (it.op != OP_NONE) items.push_back(it);
          ++i;
          break;
        }
        case SV_DENSE: {
          int k = int(o.nq);
          if (k < 1 || k > 8) return fail(SV_ERR_ARG, "dense record needs 1..8 qubits");
          if (k > 4) return fail(SV_ERR_UNSUPPORTED, "dense unitaries on more than 4 qubits");
          Item it;
          it.kind = I_GATE;
          it.flag = flag;
          it.nq = k;
          uint64_t seen = 0;
          for (int r = 0; r < k; ++r) {
            if (!qok(o.q[r]) || ((seen >> o.q[r]) & 1)) return fail(SV_ERR_ARG, "bad dense qubits at record " + std::to_string(i));
            seen |= 1ull << o.q[r];
            it.q[r] = o.q[r];
          }
          uint64_t need = (1ull << k) * (1ull << k);
          if (!pool || o.dense_off + need > pool_len) return fail(SV_ERR_ARG, "dense matrix outside the dense pool");
          it.dense = pool + 2 * o.dense_off;
          it.op = k == 1 ? OP_U : (k == 2 ? OP_U4 : OP_D16);
          items.push_back(it);
          ++i;
          break;
        }
        case SV_MEASURE:
        case SV_RESET: {
          if (!qok(o.q[0])) return fail(SV_ERR_ARG, "measured qubit out of range at record " + std::to_string(i));
          if (o.kind == SV_MEASURE && o.cbit >= 64) return fail(SV_ERR_ARG, "classical bit >= 64");
          Item it;
          it.kind = o.kind == SV_MEASURE ? I_MEAS : I_RESET;
          it.flag = flag;
          it.qubit = o.q[0];
          it.cbit = o.cbit;
          items.push_back(it);
          ++i;
          break;
        }
        case SV_COND: {
          size_t t0 = i + 1, t1 = t0 + o.then_len, e1 = t1 + o.else_len;
          if (e1 > end || t1 < t0 || e1 < t1) return fail(SV_ERR_ARG, "COND lengths exceed the enclosing block");
          if (n_flags + 2 > kMaxFlags) return fail(SV_ERR_UNSUPPORTED, "too many predicates after unrolling");
          Item it;
          it.kind = I_COND;
          it.flag = flag;
          it.f_then = int(n_flags++);
          it.f_else = o.else_len ? int(n_flags++) : -1;
          it.mask = o.mask;
          it.value = o.value;
          items.push_back(it);
          int ft = it.f_then, fe = it.f_else;
          if (!walk(t0, t1, ft, depth + 1)) return false;
          if (!walk(t1, e1, fe, depth + 1)) return false;
          i = e1;
          break;
        }
        case SV_LOOP: {
          size_t b0 = i + 1, b1 = b0 + o.body_len;
          if (b1 > end || b1 < b0) return fail(SV_ERR_ARG, "LOOP body exceeds the enclosing block");
          for (uint32_t r = 0; r < o.loop_k; ++r)
            if (!walk(b0, b1, flag, depth + 1)) return false;
          i = b1;
          break;
        }
        default:
          return fail(SV_ERR_ARG, "unknown record kind at record " + std::to_string(i));
      }
      if (items.size() > kMaxItems) return fail(SV_ERR_UNSUPPORTED, "unrolled program exceeds 2^22 ops");
    }
    return true;
  }
};

struct Segment {
  std::vector<int> gates;    // item indices
  std::vector<int> phase;    // scalar items after the last pass (program order)
  uint64_t group_q = 0;      // qubits of the group's measure/reset items
  bool has_group = false;
};

int popc(uint64_t v) { return __builtin_popcountll(v); }

// Orders the tile-local bits that receive thread-group index bits so that the
// first lanes of a warp hit distinct shared-memory banks under the swizzle.
// complex128 (A = 0): a quarter-warp (8 lanes x 16 B) is conflict-free when
// its three lane bits fall in distinct classes p mod 3.  complex64 (A = 1): a
// half-warp (16 lanes x 8 B) needs local bit 0 plus one bit of each class
// (p - 1) mod 3.
void order_thread_bits(const std::vector<int>& free_bits, int A, uint8_t* out) {
  std::vector<int> rest(free_bits);
  std::sort(rest.begin(), rest.end());
  std::vector<int> order;
  auto take = [&](auto pred) {
    for (size_t k = 0; k < rest.size(); ++k)
      if (pred(rest[k])) {
        order.push_back(rest[k]);
        rest.erase(rest.begin() + long(k));
        return;
      }
  };
  if (A == 1) take([](int p) { return p == 0; });
  for (int c = 0; c < 3; ++c)
    take([&](int p) { return A == 1 ? (p >= 1 && (p - 1) % 3 == c) : (p % 3 == c); });
  for (int b : rest) order.push_back(b);
  for (size_t k = 0; k < order.size() && k < MAX_TILE_BITS; ++k) out[k] = uint8_t(order[k]);
}

struct Builder {
  Plan& P;
  const std::vector<Item>& items;
  int B;  // log2 amplitudes per 16-byte granule (1: complex64, 0: complex128)
  int max_pass_gates;
  int tile_select = 1;  // Tuning::tile_select
  int reg_bits = REG_BITS;  // gate register bits per stage (ADJ_REG_BITS for backward plans)
  int stage_pairs = 0;       // complex64 stage packing weighs 16-byte pair accesses (Tuning::stage_pairs)
  bool adjoint = false;     // backward plan: derivative items, then U^dagger, per gate

  Builder(Plan& p, const std::vector<Item>& it, int b, int mpg) : P(p), items(it), B(b), max_pass_gates(mpg) {}

  // complex constant pool helpers
  uint32_t add_consts(const std::vector<double>& v) {
    uint32_t off = uint32_t(P.consts.size() / 2);
    P.consts.insert(P.consts.end(), v.begin(), v.end());
    return off;
  }

  void emit_job_deriv(const Item& it, int slot, uint32_t out) {
    DJob j{};
    j.kind = J_DERIV;
    j.op = OP_DOT;
    j.gate = uint8_t(it.gate);
    for (int k = 0; k < 3; ++k) {
      j.pidx[k] = it.pidx[k];
      j.angle[k] = it.angle[k];
    }
    j.len = uint32_t(slot);
    j.out = out;
    P.jobs.push_back(j);
  }

  // parametrised angle slots of a gate item (gradient entries)
  int n_dots(const Item& it) const {
    if (!adjoint || it.gate < 0) return 0;
    int d = 0;
    for (int k = 0; k < 3; ++k) d += it.pidx[k] >= 0;
    return d;
  }

  // The op a gate item runs as: forward plans take the factored rotations
  // (RX, RY and one-qubit diagonal gates), backward plans the plain ones.
  uint8_t op_of(const Item& it) const {
    if (adjoint || it.gate < 0 || it.nq != 1) return it.op;
    if (it.gate == SV_RX) return OP_RXF;
    if (it.gate == SV_RY) return OP_RYF;
    if (it.op == OP_D) return OP_DZ;
    return it.op;
  }

  void emit_job_gate(const Item& it, uint32_t out, uint8_t op) {
    DJob j{};
    j.kind = J_GATE;
    j.op = op;
    j.adj = adjoint ? 1 : 0;
    j.gate = uint8_t(it.gate);
    for (int k = 0; k < 3; ++k) {
      j.pidx[k] = it.pidx[k];
      j.angle[k] = it.angle[k];
    }
    j.out = out;
    P.jobs.push_back(j);
  }

  void emit_job_const(uint8_t op, const std::vector<double>& v, uint32_t out) {
    DJob j{};
    j.kind = J_CONST;
    j.op = op;
    j.src = add_consts(v);
    j.len = uint32_t(v.size() / 2);
    j.out = out;
    P.jobs.push_back(j);
  }

  // matrix entries of an item (with its derivative items in backward plans)
  int mat_len(const Item& it) const { return op_mat_len(op_of(it)) + 4 * n_dots(it); }

  // conjugate transpose of a row-major K x K complex matrix (re, im pairs)
  static std::vector<double> dagger(const double* m, int K) {
    std::vector<double> v(2 * K * K);
    for (int r = 0; r < K; ++r)
      for (int c = 0; c < K; ++c) {
        v[2 * (r * K + c)] = m[2 * (c * K + r)];
        v[2 * (r * K + c) + 1] = -m[2 * (c * K + r) + 1];
      }
    return v;
  }

  // Emit one pass: `chosen` gate items, tile bits `tq` (m entries), optional phase.
  void emit_pass(const std::vector<int>& chosen, const std::vector<int>& tq, const Segment* seg, bool flush) {
    const int m = int(tq.size());
    DPass ps{};
    ps.m = uint8_t(m);
    ps.L = uint8_t(P.L);
    for (int j = 0; j < m; ++j) ps.tq[j] = uint8_t(tq[j]);
    int loc[64];
    for (int q = 0; q < 64; ++q) loc[q] = -1;
    for (int j = 0; j < m; ++j) loc[tq[j]] = j;

    ps.g0 = uint32_t(P.gates.size());
    ps.s0 = uint32_t(P.stages.size());
    ps.mat0 = P.n_mat;
    uint32_t mat = 0;
    uint32_t dots = 0;

    // stages: four register bits each, dependency order preserved.  Two
    // packings are built and the one with fewer stages is kept (each stage
    // moves the tile through shared memory once): first fit in program order,
    // and one that gives each stage the register set (among all sets of
    // reg_bits of the remaining gates' local bits) under which the most
    // remaining gates can run.
    std::vector<uint32_t> stS;
    std::vector<std::vector<int>> stG;
    {
      std::vector<uint32_t> lmask(chosen.size());
      for (size_t i = 0; i < chosen.size(); ++i) {
        const Item& it = items[chosen[i]];
        uint32_t lm = 0;
        for (int k = 0; k < it.nq; ++k) lm |= 1u << loc[it.q[k]];
        lmask[i] = lm;
      }
      // gates (positions into chosen) that run under register set S, in order
      auto take = [&](const std::vector<int>& rem, uint32_t S, std::vector<int>& sg, std::vector<int>& left,
                      bool grow) -> uint32_t {
        uint32_t blocked = 0, used = 0;
        for (int i : rem) {
          const uint32_t lm = lmask[size_t(i)];
          const bool fits = grow ? popc(used | lm) <= reg_bits : (lm & ~S) == 0;
          if ((lm & blocked) || !fits) {
            blocked |= lm;
            left.push_back(i);
            continue;
          }
          used |= lm;
          sg.push_back(i);
        }
        return used;
      };
      // paired: only register sets that hold local bit 0 (a gate's or the
      // padding), so that complex64 stages move amplitude pairs as 16 bytes
      auto pack = [&](bool best, bool paired, std::vector<uint32_t>& oS, std::vector<std::vector<int>>& oG) {
        std::vector<int> rem(chosen.size());
        for (size_t i = 0; i < rem.size(); ++i) rem[i] = int(i);
        while (!rem.empty()) {
          std::vector<int> sg, left;
          uint32_t S = 0;
          if (!best) {
            S = take(rem, 0, sg, left, true);
          } else {
            uint32_t bits = 0;
            for (int i : rem) bits |= lmask[size_t(i)];
            if (paired) bits |= 1u;
            std::vector<int> bl;
            for (int j = 0; j < 32; ++j)
              if ((bits >> j) & 1) bl.push_back(j);
            const int k = std::min<int>(reg_bits, int(bl.size()));
            size_t bestn = 0, bestp = 0;
            uint32_t bestS = 0, bestSp = 0;
            std::vector<int> pick(static_cast<size_t>(k));
            for (int i = 0; i < k; ++i) pick[size_t(i)] = i;
            while (true) {  // every k-subset of the remaining gates' local bits
              uint32_t Sc = 0;
              for (int i : pick) Sc |= 1u << bl[size_t(i)];
              // take(rem, Sc, .., false), counted only
              size_t na = 0;
              uint32_t blocked = 0;
              for (int i : rem) {
                const uint32_t lm = lmask[size_t(i)];
                if ((lm & blocked) || (lm & ~Sc)) blocked |= lm;
                else ++na;
              }
              if (na > bestn) {
                bestn = na;
                bestS = Sc;
              }
              if ((Sc & 1u) && na > bestp) {
                bestp = na;
                bestSp = Sc;
              }
              int i = k - 1;
              while (i >= 0 && pick[size_t(i)] == int(bl.size()) - k + i) --i;
              if (i < 0) break;
              ++pick[size_t(i)];
              for (int j = i + 1; j < k; ++j) pick[size_t(j)] = pick[size_t(j - 1)] + 1;
            }
            // paired: the best set holding local bit 0, unless none runs a gate
            // (the next gate needs four other bits, e.g. a dense 4-qubit one)
            S = take(rem, (paired && bestp > 0) ? bestSp : bestS, sg, left, false);
          }
          for (int& i : sg) i = chosen[size_t(i)];
          rem.swap(left);
          oS.push_back(S);
          oG.push_back(sg);
        }
      };
      std::vector<uint32_t> s1, s2, s3;
      std::vector<std::vector<int>> g1, g2, g3;
      pack(false, false, s1, g1);
      if (!adjoint && s1.size() > 1) pack(true, false, s2, g2);
      // complex64: a stage whose register set holds local bit 0 moves its
      // amplitudes as 16-byte pairs (half the shared-memory instructions of a
      // stage without it), so packings are compared by that cost
      const bool pair_cost = B == 1 && !adjoint && stage_pairs > 0;
      if (pair_cost && s1.size() > 1) pack(true, true, s3, g3);
      auto cost = [&](const std::vector<uint32_t>& ss) {
        size_t c = 0;
        for (uint32_t S : ss)
          c += (!pair_cost || (S & 1u) || popc(S) < reg_bits) ? (stage_pairs == 2 ? 1 : 2) : 3 - (stage_pairs == 2 ? 1 : 0);
        return c;
      };
      stS = s1;
      stG = g1;
      if (!s2.empty() && (pair_cost ? cost(s2) < cost(stS) : s2.size() < stS.size())) {
        stS = s2;
        stG = g2;
      }
      if (!s3.empty() && cost(s3) < cost(stS)) {
        stS = s3;
        stG = g3;
      }
    }

    // Warp ownership.  With 2^m >= 16 * PASS_THREADS every thread holds one
    // group per 256, so the warp index (thread bits 5..7) is three group bits:
    // a warp touches only the amplitudes whose tile bits there equal its index.
    // The tile copies map thread bit t to tile bit t + B, so their warp bits are
    // B+5, B+6, B+7.  Two consecutive steps (copy, stages, copy back) with the
    // same ordered warp bits need only a warp barrier between them.
    const bool warp_local = !adjoint && m >= 12 && PASS_THREADS == 256;
    const int W0[3] = {B + 5, B + 6, B + 7};
    const uint32_t w0m = (1u << W0[0]) | (1u << W0[1]) | (1u << W0[2]);
    int Wcur[3] = {W0[0], W0[1], W0[2]};
    const int K = int(stS.size());
    std::vector<uint8_t> bar_before(size_t(K) + 1, 1);
    for (int si = 0; si < K; ++si) {
      const uint32_t S = stS[size_t(si)];
      const uint32_t wcm = (1u << Wcur[0]) | (1u << Wcur[1]) | (1u << Wcur[2]);
      // Lanes are conflict-free in shared memory when their bits reach every
      // class of the swizzle's 3-bit fold (complex64 8-byte accesses also
      // need local bit 0; with bit 0 a register bit, pairs move as 16 bytes).
      auto lanes_ok = [&](uint32_t fm, bool pairs) {
        bool cls[3] = {false, false, false};
        for (int j = 0; j < m; ++j)
          if ((fm >> j) & 1) {
            if (B == 0) cls[j % 3] = true;
            else if (j >= 1) cls[(j - 1) % 3] = true;
          }
        return cls[0] && cls[1] && cls[2] && (B == 0 || pairs || (fm & 1u));
      };
      const uint32_t all = (m >= 32) ? ~0u : ((1u << m) - 1u);
      // register bits: the stage's qubits, padded with local bit 0 when it is
      // free (complex64: amplitude pairs then share a 16-byte granule, so
      // specialised kernels move them with one access), then with the highest
      // other local bits that keep the lanes conflict-free and, where possible,
      // stay off the warp bits; ascending, so local bit 0 is register bit 0
      std::vector<int> reg;
      uint32_t rm = S;
      for (int j = 0; j < m; ++j)
        if ((S >> j) & 1) reg.push_back(j);
      if (B == 1 && !(S & 1u) && popc(S) < reg_bits) {
        reg.push_back(0);
        rm |= 1u;
      }
      for (int pass = 0; pass < 3; ++pass)
        for (int j = m - 1; j >= 1 && int(reg.size()) < reg_bits; --j) {
          if ((rm >> j) & 1) continue;
          const uint32_t r2 = rm | (1u << j);
          if (pass < 2 && !lanes_ok(all & ~r2 & ~(warp_local ? wcm : 0u), B == 1 && (r2 & 1u))) continue;
          if (pass == 0 && warp_local && (((wcm | w0m) >> j) & 1)) continue;
          reg.push_back(j);
          rm = r2;
        }
      std::sort(reg.begin(), reg.end());
      const bool pairs = B == 1 && (rm & 1u);
      const uint32_t fm = all & ~rm;
      const bool can_be_clean = lanes_ok(fm, pairs);

      // Direct store (the last stage of a pass without a measurement table
      // writes its registers to the state itself, specialised kernels): every
      // store instruction must write whole 128-byte lines (scattered 32-byte
      // sectors measured slower than the pass's own store phase).  The tile bits
      // `dwant` below a line (bits 0..2 + B, less register bit 0 when it holds
      // complex64 amplitude pairs) go to the first lanes; the warp bits avoid them.
      const bool dlast = !adjoint && si == K - 1 && !(seg && seg->has_group);
      std::vector<int> dwant;
      if (dlast) {  // the first lanes cover a 128-byte line: tile bits below 3 + B, minus register bit 0
        for (int b = (B == 1 && (rm & 1u)) ? 1 : 0; b < 3 + B; ++b) dwant.push_back(b);
      }
      bool dpossible = dlast;
      for (int b : dwant) dpossible = dpossible && !((rm >> b) & 1u);
      uint32_t dmask = 0;
      for (int b : dwant) dmask |= 1u << b;
      int W[3] = {-1, -1, -1};
      if (warp_local) {
        if (!(rm & wcm) && (!can_be_clean || lanes_ok(fm & ~wcm, pairs)) && !(dpossible && (wcm & dmask))) {
          for (int i = 0; i < 3; ++i) W[i] = Wcur[i];
          bar_before[size_t(si)] = 0;
        } else {
          // the triple that stays out of the following stages longest and keeps
          // the lanes conflict-free; ties go to the copies' warp bits, so the
          // run can end warp-locally
          int run[MAX_TILE_BITS] = {};
          for (int j = 0; j < m; ++j)
            while (si + 1 + run[j] < K && !((stS[size_t(si + 1 + run[j])] >> j) & 1)) ++run[j];
          int best = -1;
          uint32_t bestm = 0;
          for (int a = 0; a < m; ++a)
            for (int b = a + 1; b < m; ++b)
              for (int c = b + 1; c < m; ++c) {
                const uint32_t tm = (1u << a) | (1u << b) | (1u << c);
                if ((tm & rm) || (B == 1 && (tm & 1u))) continue;
                if (dpossible && (tm & dmask)) continue;
                if (can_be_clean && !lanes_ok(fm & ~tm, pairs)) continue;
                const int r = std::min(run[a], std::min(run[b], run[c]));
                const int score = 8 * r + (si + 1 + r == K && tm == w0m ? 4 : 0) + popc(tm & w0m);
                if (score > best) {
                  best = score;
                  bestm = tm;
                }
              }
          if (best < 0)  // cannot happen for m >= 12 (8 free bits); keep any three
            for (int j = m - 1; j >= 1 && popc(bestm) < 3; --j)
              if (!((rm >> j) & 1)) bestm |= 1u << j;
          if (bestm == w0m) {
            for (int i = 0; i < 3; ++i) W[i] = W0[i];
          } else {
            int i = 0;
            for (int j = 0; j < m; ++j)
              if ((bestm >> j) & 1) W[i++] = j;
          }
        }
        for (int i = 0; i < 3; ++i) Wcur[i] = W[i];
      }

      DStage st{};
      st.g0 = uint16_t(P.gates.size() - ps.g0);
      int rpos[MAX_TILE_BITS];
      for (int j = 0; j < MAX_TILE_BITS; ++j) rpos[j] = -1;
      for (int r = 0; r < reg_bits; ++r) {
        st.R[r] = uint16_t(tile_swizzle(1u << reg[size_t(r)], B));
        st.Rb[r] = uint8_t(reg[size_t(r)]);
        rpos[reg[size_t(r)]] = r;
      }
      std::vector<int> freeb;
      for (int j = 0; j < m; ++j)
        if (rpos[j] < 0 && !(warp_local && (j == W[0] || j == W[1] || j == W[2]))) freeb.push_back(j);
      uint8_t thr[MAX_TILE_BITS] = {};
      order_thread_bits(freeb, B, thr);
      std::vector<int> ebits;
      if (warp_local) {
        for (int k = 0; k < 5; ++k) ebits.push_back(thr[k]);
        for (int i = 0; i < 3; ++i) ebits.push_back(W[i]);
        for (size_t k = 5; k < freeb.size(); ++k) ebits.push_back(thr[k]);
      } else {
        for (size_t k = 0; k < freeb.size(); ++k) ebits.push_back(thr[k]);
      }
      if (dpossible) {
        const auto lanes_end = ebits.begin() + std::min<long>(5, long(ebits.size()));
        bool ok = true;
        for (int b : dwant) ok = ok && std::find(ebits.begin(), lanes_end, b) != lanes_end;
        if (ok) {  // those tile bits first, in order; the lane order is otherwise kept
          for (size_t i = 0; i < dwant.size(); ++i) {
            auto it = std::find(ebits.begin() + long(i), lanes_end, dwant[i]);
            std::rotate(ebits.begin() + long(i), it, it + 1);
          }
          ps.direct = 1;
        }
      }
      for (int k = 0; k < m - reg_bits; ++k) {
        st.E[k] = uint16_t(tile_swizzle(1u << ebits[size_t(k)], B));
        st.Eb[k] = uint8_t(ebits[size_t(k)]);
      }
      const std::vector<int>& sg = stG[size_t(si)];
      for (int idx : sg) {
        const Item& it = items[idx];
        // backward plans: derivative accumulations before the gate's U^dagger
        for (int k = 0; adjoint && it.gate >= 0 && k < 3; ++k) {
          if (it.pidx[k] < 0) continue;
          DGate d{};
          d.op = it.nq == 2 ? OP_CDOT : OP_DOT;
          d.flag = -1;
          d.p0 = uint8_t(rpos[loc[it.q[0]]]);
          d.p1 = it.nq > 1 ? uint8_t(rpos[loc[it.q[1]]]) : 0;
          d.key = uint16_t(d.op * 16 + d.p0 * 4 + d.p1);
          d.mat = mat;
          d.dslot = uint16_t(dots++);
          d.gidx = uint32_t(it.pidx[k]);
          emit_job_deriv(it, k, P.n_mat + mat);
          mat += 4;
          P.gates.push_back(d);
        }
        DGate g{};
        g.op = op_of(it);
        if (it.op == OP_D16) ps.dense = 1;
        g.flag = it.flag;
        g.p0 = uint8_t(rpos[loc[it.q[0]]]);
        g.p1 = it.nq > 1 ? uint8_t(rpos[loc[it.q[1]]]) : 0;
        g.key = uint16_t(g.op == OP_D16 ? OP_D16 * 16 : g.op * 16 + g.p0 * 4 + g.p1);
        g.mat = mat;
        const uint32_t out = P.n_mat + mat;
        if (it.gate >= 0) {
          emit_job_gate(it, out, g.op);
        } else if (it.op == OP_U || it.op == OP_U4) {
          const int K = it.op == OP_U ? 2 : 4;
          std::vector<double> v = adjoint ? dagger(it.dense, K) : std::vector<double>(it.dense, it.dense + 2 * K * K);
          emit_job_const(it.op, v, out);
        } else {  // OP_D16: expand onto the four register bits
          const int k = it.nq;
          int ri[4];
          uint32_t gm = 0;
          for (int r = 0; r < k; ++r) {
            ri[r] = rpos[loc[it.q[r]]];
            gm |= 1u << ri[r];
          }
          const int K = 1 << k;
          std::vector<double> du;
          const double* dm = it.dense;
          if (adjoint) {
            du = dagger(it.dense, K);
            dm = du.data();
          }
          std::vector<double> v(2 * 256, 0.0);
          for (int a = 0; a < 16; ++a)
            for (int b = 0; b < 16; ++b) {
              if ((a & ~gm) != (b & ~gm)) continue;
              int la = 0, lb = 0;
              for (int r = 0; r < k; ++r) {
                la |= ((a >> ri[r]) & 1) << r;
                lb |= ((b >> ri[r]) & 1) << r;
              }
              v[2 * (a * 16 + b)] = dm[2 * (la * K + lb)];
              v[2 * (a * 16 + b) + 1] = dm[2 * (la * K + lb) + 1];
            }
          emit_job_const(OP_D16, v, out);
        }
        mat += uint32_t(op_mat_len(g.op));
        P.gates.push_back(g);
      }
      st.ng = uint16_t(P.gates.size() - ps.g0 - st.g0);  // gate records, derivative items included
      st.bar = 1;
      P.stages.push_back(st);
    }
    // barrier flags: a block barrier wherever the warp bits change; after the
    // last stage unless it ends on the copies' warp bits without a group table
    const bool end_w0 = warp_local && K > 0 && Wcur[0] == W0[0] && Wcur[1] == W0[1] && Wcur[2] == W0[2];
    const bool tail_local = end_w0 && !(seg && seg->has_group);
    // a direct store leaves no shared-memory reader after the last stage; the
    // next tile's refill of this buffer then needs the last stage's warps to
    // own what they refill, or a block barrier when the tile lands
    bar_before[size_t(K)] = (tail_local || (ps.direct && warp_local)) ? 0 : 1;
    for (int si = 0; si < K; ++si) P.stages[ps.s0 + size_t(si)].bar = bar_before[size_t(si) + 1];
    ps.bar_in = K > 0 ? bar_before[0] : 1;
    if (ps.direct && !end_w0) ps.bar_in = 1;
    ps.ng = uint32_t(P.gates.size() - ps.g0);
    ps.ns = uint32_t(P.stages.size() - ps.s0);
    ps.nmat = mat;
    P.n_mat += mat;
    P.max_dots = std::max(P.max_dots, dots);
    P.max_pass_mat = std::max(P.max_pass_mat, mat);
    P.max_stages = std::max(P.max_stages, ps.ns);
    P.max_gates = std::max(P.max_gates, ps.ng);

    // group table and scalar phase
    ps.c0 = uint32_t(P.scalars.size());
    if (seg && seg->has_group) {
      // table bits: group qubits inside the tile first (they become the
      // reduction stage's register bits), then the ones outside
      std::vector<int> in_q, out_q;
      for (int q = 0; q < 64; ++q) {
        if (!((seg->group_q >> q) & 1)) continue;
        if (loc[q] >= 0) in_q.push_back(q);
        else out_q.push_back(q);
      }
      ps.kin = uint8_t(in_q.size());
      ps.gk = uint8_t(in_q.size() + out_q.size());
      int tbit[64];
      for (int q = 0; q < 64; ++q) tbit[q] = -1;
      uint32_t used = 0;
      std::vector<int> reg;
      for (size_t k = 0; k < in_q.size(); ++k) {
        tbit[in_q[k]] = int(k);
        reg.push_back(loc[in_q[k]]);
        used |= 1u << loc[in_q[k]];
      }
      for (size_t k = 0; k < out_q.size(); ++k) {
        tbit[out_q[k]] = int(in_q.size() + k);
        ps.outer_gq[k] = uint8_t(out_q[k]);
      }
      for (int j = m - 1; j >= 0 && int(reg.size()) < REG_BITS; --j)
        if (!((used >> j) & 1)) {
          reg.push_back(j);
          used |= 1u << j;
        }
      for (int r = 0; r < REG_BITS; ++r) ps.red_R[r] = uint16_t(tile_swizzle(1u << reg[r], B));
      std::vector<int> freeb;
      for (int j = 0; j < m; ++j)
        if (!((used >> j) & 1)) freeb.push_back(j);
      uint8_t thr[MAX_TILE_BITS] = {};
      order_thread_bits(freeb, B, thr);
      for (int k = 0; k < m - REG_BITS; ++k) ps.red_E[k] = uint16_t(tile_swizzle(1u << thr[k], B));

      // which flags are decided inside this phase
      std::vector<int> decided_here;
      bool always = false;
      for (int idx : seg->phase) {
        const Item& it = items[idx];
        DScalar s{};
        if (it.kind == I_COND) {
          s.kind = S_COND;
          s.flag = it.flag;
          s.f_then = it.f_then;
          s.f_else = it.f_else;
          s.mask = it.mask;
          s.value = it.value;
          decided_here.push_back(it.f_then);
          if (it.f_else >= 0) decided_here.push_back(it.f_else);
        } else {
          s.kind = it.kind == I_MEAS ? S_MEASURE : S_RESET;
          s.flag = it.flag;
          s.f_then = s.f_else = -1;
          s.qubit = uint32_t(it.qubit);
          s.cbit = it.cbit;
          s.tbit = uint8_t(tbit[it.qubit]);
          if (it.flag < 0 || std::find(decided_here.begin(), decided_here.end(), it.flag) != decided_here.end())
            always = true;
        }
        P.scalars.push_back(s);
      }
      ps.group_always = always ? 1 : 0;
    }
    ps.nc = uint32_t(P.scalars.size() - ps.c0);
    P.max_scalars = std::max(P.max_scalars, ps.nc);
    ps.flush = flush ? 1 : 0;
    P.passes.push_back(ps);
  }

  // Greedy fusion of a segment's gates into passes.
  // The passes of a segment, as (gates, tile qubits, last) in order; reads
  // the items and the tuning only, so segments can be planned concurrently.
  struct PassPick {
    std::vector<int> chosen, tq;
    bool last = false;
  };
  void emit_segment(const Segment& seg) {
    std::vector<PassPick> picks;
    plan_segment(seg, picks);
    emit_picks(seg, picks);
  }
  void emit_picks(const Segment& seg, const std::vector<PassPick>& picks) {
    for (const PassPick& pk : picks) emit_pass(pk.chosen, pk.tq, pk.last ? &seg : nullptr, false);
  }
  void plan_segment(const Segment& seg, std::vector<PassPick>& picks) const {
    const int n = P.n_int, m = P.m, L = P.L;
    const uint64_t low = (L >= 64) ? ~0ull : ((1ull << L) - 1);
    std::vector<int> rem(seg.gates);
    if (rem.empty()) {
      // a measurement group with no gate before it: an empty (read-only) pass
      std::vector<int> tq;
      uint64_t T = low;
      for (int q = 0; q < n && popc(T) < m; ++q) {
        if ((seg.group_q >> q) & 1) T |= 1ull << q;
      }
      for (int q = 0; q < n && popc(T) < m; ++q) T |= 1ull << q;
      for (int q = 0; q < n; ++q)
        if ((T >> q) & 1) tq.push_back(q);
      picks.push_back(PassPick{{}, tq, true});
      return;
    }
    const size_t cap = max_pass_gates > 0 ? size_t(max_pass_gates) : size_t(MAX_PASS_GATES);
    const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    // The gates (in order) a tile of qubits T runs: a gate runs when its qubits
    // are tile qubits and no earlier gate on one of them was left out; the
    // pass's record, matrix and derivative capacities bound it.  grow: first
    // fit, T takes the qubits of every gate that still fits in m.
    auto take = [&](const std::vector<int>& from, uint64_t& T, bool grow, std::vector<int>* chosen,
                    std::vector<int>* left) -> size_t {
      uint64_t blocked = 0;
      uint32_t mat = 0, dots = 0, recs = 0;
      size_t k = 0;
      for (int idx : from) {
        const Item& it = items[idx];
        const uint64_t qm = it.qmask();
        const uint32_t ml = uint32_t(mat_len(it));
        const uint32_t nd = uint32_t(n_dots(it));
        const bool fits = grow ? popc(T | qm) <= m : (qm & ~T) == 0;
        if ((qm & blocked) || !fits || recs + 1 + nd > cap || mat + ml > MAX_PASS_MAT || dots + nd > MAX_PASS_DOTS) {
          blocked |= qm;
          if (left) left->push_back(idx);
          continue;
        }
        if (grow) T |= qm;
        mat += ml;
        dots += nd;
        recs += 1 + nd;
        ++k;
        if (chosen) chosen->push_back(idx);
      }
      return k;
    };
    // Gates a tile T runs, for the searches below: the same rule as take(),
    // over per-gate masks and capacities gathered once per pass.
    std::vector<uint64_t> cq;
    std::vector<uint32_t> cml, cnd;
    auto prep = [&]() {
      cq.clear();
      cml.clear();
      cnd.clear();
      for (int idx : rem) {
        const Item& it = items[idx];
        cq.push_back(it.qmask());
        cml.push_back(uint32_t(mat_len(it)));
        cnd.push_back(uint32_t(n_dots(it)));
      }
    };
    auto count = [&](uint64_t T) -> size_t {
      uint64_t blocked = 0;
      uint32_t mat = 0, dots = 0, recs = 0;
      size_t k = 0;
      const size_t nr = cq.size();
      for (size_t i = 0; i < nr; ++i) {
        const uint64_t qm = cq[i];
        if ((qm & blocked) || (qm & ~T) || recs + 1 + cnd[i] > cap || mat + cml[i] > MAX_PASS_MAT ||
            dots + cnd[i] > MAX_PASS_DOTS) {
          blocked |= qm;
          // nothing further can run once every tile qubit is blocked: a later
          // gate either leaves the tile or touches a blocked qubit
          if ((blocked & T) == T) break;
          continue;
        }
        mat += cml[i];
        dots += cnd[i];
        recs += 1 + cnd[i];
        ++k;
      }
      return k;
    };
    // Beam search over the gathered qubits (width kBeam): grow every kept tile
    // by one qubit, keep the kBeam tiles that run the most gates (ties to the
    // lower qubit set); returns the best tile seen.
    auto beam = [&](uint64_t T0) -> uint64_t {
      constexpr size_t kBeam = 4;
      std::vector<uint64_t> cur{T0};
      uint64_t best = T0;
      size_t bestv = count(best);
      std::vector<std::pair<size_t, uint64_t>> nx;
      std::vector<uint64_t> cand;
      for (int step = popc(T0); step < m; ++step) {
        nx.clear();
        cand.clear();
        for (uint64_t X : cur)
          for (int q = 0; q < n; ++q) {
            if ((X >> q) & 1) continue;
            cand.push_back(X | (1ull << q));
          }
        // beams that differ in one qubit reach the same sets: count each once
        std::sort(cand.begin(), cand.end());
        cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
        for (uint64_t X2 : cand) nx.push_back({count(X2), X2});
        std::sort(nx.begin(), nx.end(), [](const std::pair<size_t, uint64_t>& a, const std::pair<size_t, uint64_t>& b) {
          return a.first > b.first || (a.first == b.first && a.second < b.second);
        });
        nx.erase(std::unique(nx.begin(), nx.end(),
                             [](const std::pair<size_t, uint64_t>& a, const std::pair<size_t, uint64_t>& b) {
                               return a.second == b.second;
                             }),
                 nx.end());
        cur.clear();
        for (size_t i = 0; i < nx.size() && cur.size() < kBeam; ++i) cur.push_back(nx[i].second);
        if (!nx.empty() && nx[0].first > bestv) {
          bestv = nx[0].first;
          best = nx[0].second;
        }
      }
      return best;
    };
    while (!rem.empty()) {
      uint64_t T = low;
      if (tile_select && popc(all) > m) {
        // gathered qubits chosen one at a time for the gates they let this
        // pass run (a pair when no single qubit adds any; else the qubits of
        // the first gate that still fits), ties to the lowest qubit
        prep();
        size_t have = count(T);
        while (popc(T) < m) {
          int bq = -1;
          size_t bv = 0;
          for (int q = 0; q < n; ++q) {
            if ((T >> q) & 1) continue;
            const size_t v = count(T | (1ull << q));
            if (v > bv) {
              bv = v;
              bq = q;
            }
          }
          if (bq >= 0 && bv > have) {
            T |= 1ull << bq;
            have = bv;
            continue;
          }
          uint64_t bp = 0;
          if (popc(T) + 2 <= m) {
            // No single qubit lets another gate run, so a pair can only do so
            // through a gate with exactly that pair outside the tile (every
            // other gate that would run is held by a blocker with both qubits
            // outside): only those pairs are counted, in the (a, b) order of an
            // exhaustive search, which they would win (count is monotone in T).
            std::vector<uint32_t> pairs;
            for (uint64_t qm : cq) {
              const uint64_t out = qm & ~T;
              if (popc(out) != 2) continue;
              const int a = __builtin_ctzll(out), b2 = 63 - __builtin_clzll(out);
              pairs.push_back(uint32_t(a) << 8 | uint32_t(b2));
            }
            std::sort(pairs.begin(), pairs.end());
            pairs.erase(std::unique(pairs.begin(), pairs.end()), pairs.end());
            for (uint32_t pr : pairs) {
              const uint64_t pm = (1ull << (pr >> 8)) | (1ull << (pr & 0xFF));
              const size_t v = count(T | pm);
              if (v > bv) {
                bv = v;
                bp = pm;
              }
            }
          }
          if (bp && bv > have) {
            T |= bp;
            have = bv;
            continue;
          }
          // nothing more runs with one or two more qubits: the qubits of the
          // first gate (in order) that fits, if any; else the tile is done
          bool grew = false;
          for (int idx : rem) {
            const uint64_t qm = items[idx].qmask();
            if ((qm & ~T) && popc(T | qm) <= m) {
              T |= qm;
              grew = true;
              break;
            }
          }
          if (!grew) break;
          have = count(T);
        }
        // the beam's tile when it lets this pass run more gates than the greedy one
        const uint64_t Tb = beam(low);
        if (count(Tb) > have) T = Tb;
      }
      std::vector<int> chosen, left;
      take(rem, T, !tile_select || popc(all) <= m, &chosen, &left);
      if (chosen.empty()) {  // cannot happen (the first gate always fits an empty tile); first fit
        left.clear();
        T = low;
        take(rem, T, true, &chosen, &left);
      }
      rem.swap(left);
      const bool last = rem.empty();
      if (last && seg.has_group) {
        // bring measured qubits into the tile when there is room
        for (int q = 0; q < n && popc(T) < m; ++q)
          if ((seg.group_q >> q) & 1) T |= 1ull << q;
      }
      for (int q = 0; q < n && popc(T) < m; ++q) T |= 1ull << q;
      std::vector<int> tq;
      for (int q = 0; q < n; ++q)
        if ((T >> q) & 1) tq.push_back(q);
      picks.push_back(PassPick{chosen, tq, last});
    }
  }
};

}  // namespace

// Checks the barrier flags of every pass against the thread -> amplitude maps
// of the kernels (the tile copy: 16-byte vector k of thread t at chunk
// (t >> vl) + (k << (VB - L)), offset (t & (2^vl - 1)) << B; a stage: group g
// of thread g mod 256 at XOR of E over the bits of g, its 16 amplitudes at
// XOR of R over the register index).  Every stage must touch each amplitude
// once, and wherever only a warp barrier separates two steps (copy -> first
// stage, stage -> stage, last stage -> copy back) both must give every
// amplitude to the same warp.  Returns the number of violations.
int check_barriers(const Plan& P, uint64_t* warp_syncs, uint64_t* block_syncs) {
  const int B = P.dtype == SV_C64 ? 1 : 0;
  int bad = 0;
  *warp_syncs = *block_syncs = 0;
  // warp that touches each tile address: in the tile copy (per tile geometry) and in each stage
  std::vector<int8_t> copy_own, first, prev, cur;
  std::vector<uint8_t> cnt;
  std::vector<uint32_t> base;
  int cm = -1, cL = -1;
  auto stage_own = [&](const DStage& st, int m, std::vector<int8_t>& own) {
    const uint32_t T = 1u << m;
    own.assign(T, int8_t(-1));
    cnt.assign(T, 0);
    uint32_t off[1 << REG_BITS];  // register offsets: XOR of R over the set bits of j
    off[0] = 0;
    for (int j = 1; j < (1 << REG_BITS); ++j) off[j] = off[j & (j - 1)] ^ st.R[__builtin_ctz(unsigned(j))];
    const int G = int(T >> REG_BITS);
    base.assign(size_t(G), 0);  // group bases: XOR of E over the set bits of g
    for (int g = 1; g < G; ++g) base[size_t(g)] = base[size_t(g & (g - 1))] ^ st.E[__builtin_ctz(unsigned(g))];
    for (int g = 0; g < G; ++g) {
      const int8_t w = int8_t((g % PASS_THREADS) >> 5);
      for (int j = 0; j < (1 << REG_BITS); ++j) {
        const uint32_t a = base[size_t(g)] ^ off[j];
        if (a >= T) {
          ++bad;
          continue;
        }
        if (cnt[a] < 255) ++cnt[a];
        own[a] = w;
      }
    }
    for (uint32_t a = 0; a < T; ++a) bad += cnt[a] != 1;
  };
  for (const DPass& ps : P.passes) {
    if (ps.ns == 0) continue;
    const int m = ps.m, L = ps.L, T = 1 << m;
    if (m != cm || L != cL) {
      copy_own.assign(size_t(T), int8_t(-1));
      const int VB = B ? 9 : 8, NVT = 1 << (m - VB), vl = B ? L - 1 : L;
      for (int t = 0; t < PASS_THREADS; ++t) {
        const uint32_t wv = uint32_t(t) & ((1u << vl) - 1u);
        const uint32_t woff = B ? (wv << 1) : wv;
        for (int k = 0; k < NVT; ++k) {
          const uint32_t ch = (uint32_t(t) >> vl) + (uint32_t(k) << (VB - L));
          const uint32_t a = tile_swizzle((ch << L) | woff, B);
          for (int e = 0; e <= B; ++e) copy_own[a ^ uint32_t(e)] = int8_t(t >> 5);
        }
      }
      cm = m;
      cL = L;
    }
    // every stage's map is checked; consecutive maps are compared where no block barrier separates them
    for (uint32_t si = 0; si < ps.ns; ++si) {
      stage_own(P.stages[ps.s0 + si], m, cur);
      if (si == 0) first = cur;
      else if (!P.stages[ps.s0 + si - 1].bar) bad += prev != cur;
      std::swap(prev, cur);
    }
    // prev: the last stage's map
    if (ps.bar_in) ++*block_syncs;
    else {
      ++*warp_syncs;
      bad += first != copy_own;
      // direct store: the refill of the previous tile's buffer follows its last stage
      if (ps.direct) bad += prev != copy_own;
    }
    for (uint32_t si = 0; si < ps.ns; ++si) {
      if (P.stages[ps.s0 + si].bar) ++*block_syncs;
      else ++*warp_syncs;
    }
    if (!P.stages[ps.s0 + ps.ns - 1].bar) {
      if (!ps.direct) bad += (prev != copy_own) || ps.gk != 0;
      else bad += ps.gk != 0;
    }
  }
  return bad;
}

sv_status build_plan(int n, int dtype, const sv_op* ops, size_t n_ops, const double* dense_pool, size_t dense_len,
                     const Tuning& tune, Plan& P, std::string& err) {
  P = Plan{};
  if (n < 1 || n > 34) {
    err = "n must be in 1..34";
    return SV_ERR_ARG;
  }
  if (n_ops && !ops) {
    err = "ops is NULL";
    return SV_ERR_ARG;
  }
  P.n = n;
  P.jit_min_blocks = tune.jit_min_blocks;
  P.n_int = std::max(n, std::max(tune.min_qubits, 10));  // small states are padded with qubits that stay |0>
  P.dtype = dtype;
  int tb = tune.tile_bits > 0 ? tune.tile_bits : 12;
  // shared-memory tile: 2^14 x 8 B (complex64) or 2^13 x 16 B (complex128) at most
  tb = std::min(std::max(tb, 10), dtype == SV_C64 ? MAX_TILE_BITS : MAX_TILE_BITS - 1);
  P.m = std::min(P.n_int, tb);
  // 2^3 contiguous amplitudes per gathered chunk (64 B for complex64, 128 B for complex128):
  // shorter runs leave more qubits to gather, so a tile fuses more gates (n=30 layered
  // program: 41 passes with 2^4-amplitude runs, 38 with 2^3, measured 6.37e12 -> 6.50e12
  // updates/s on one box)
  int lb = tune.low_bits > 0 ? tune.low_bits : 3;
  P.L = std::min(std::max(lb, 2), P.m);
  P.L = std::max(P.L, P.m - 9);  // at most 2^9 gathered chunks per tile
  P.L = std::min(P.L, dtype == SV_C64 ? 9 : 8);  // a warp-group of 256 threads covers whole chunks

  Unroller U;
  U.ops = ops;
  U.n_ops = n_ops;
  U.n = n;
  U.pool = dense_pool;
  U.pool_len = dense_pool ? dense_len : 0;
  if (!U.walk(0, n_ops, -1, 0)) {
    err = U.err;
    return U.st;
  }
  P.n_flags = U.n_flags;
  P.n_params_needed = U.max_param;

  // segmentation
  std::vector<Segment> segs(1);
  bool seen_group = false;
  uint64_t n_gates = 0, n_draws = 0;
  for (size_t i = 0; i < U.items.size(); ++i) {
    const Item& it = U.items[i];
    Segment* cur = &segs.back();
    switch (it.kind) {
      case I_GATE:
        ++n_gates;
        if (cur->has_group) {
          segs.emplace_back();
          cur = &segs.back();
        }
        cur->gates.push_back(int(i));
        break;
      case I_MEAS:
      case I_RESET: {
        ++n_draws;
        seen_group = true;
        const uint64_t qb = 1ull << it.qubit;
        if (cur->has_group && popc(cur->group_q | qb) > MAX_GROUP_Q) {
          segs.emplace_back();
          cur = &segs.back();
        }
        cur->has_group = true;
        cur->group_q |= qb;
        cur->phase.push_back(int(i));
        break;
      }
      case I_COND: {
        if (!seen_group) {
          DScalar s{};
          s.kind = S_COND;
          s.flag = it.flag;
          s.f_then = it.f_then;
          s.f_else = it.f_else;
          s.mask = it.mask;
          s.value = it.value;
          P.init_items.push_back(s);
        } else if (cur->has_group) {
          cur->phase.push_back(int(i));
        } else {
          segs[segs.size() - 2].phase.push_back(int(i));
        }
        break;
      }
    }
  }

  Builder b(P, U.items, dtype == SV_C64 ? 1 : 0, tune.max_pass_gates);
  b.tile_select = tune.tile_select;
  b.stage_pairs = tune.stage_pairs;
  {
    // tile selection per segment on worker threads (it dominates the host
    // time of a plan; segments are independent), passes emitted in order
    std::vector<const Segment*> todo;
    for (const Segment& s : segs)
      if (!(s.gates.empty() && !s.has_group)) todo.push_back(&s);
    std::vector<std::vector<Builder::PassPick>> picks(todo.size());
    size_t work = 0;
    for (const Segment* s : todo) work += s->gates.size();
    const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
    const size_t nt = std::min<size_t>({todo.size(), size_t(hw), 8});
    if (nt <= 1 || work < 256) {
      for (size_t i = 0; i < todo.size(); ++i) b.plan_segment(*todo[i], picks[i]);
    } else {
      std::atomic<size_t> next{0};
      auto worker = [&]() {
        for (size_t i; (i = next.fetch_add(1)) < todo.size();) b.plan_segment(*todo[i], picks[i]);
      };
      std::vector<std::thread> th;
      for (size_t t = 1; t < nt; ++t) th.emplace_back(worker);
      worker();
      for (std::thread& t : th) t.join();
    }
    for (size_t i = 0; i < todo.size(); ++i) b.emit_picks(*todo[i], picks[i]);
  }
  // A projector can still be pending at the end (a final measurement group,
  // or later passes whose gates were all predicated off): a flush pass
  // applies it.  When nothing is pending its CTAs return at once.
  if (n_draws > 0) {
    P.needs_flush = true;
    std::vector<int> tq;
    for (int q = 0; q < P.m; ++q) tq.push_back(q);
    b.emit_pass({}, tq, nullptr, true);
  }

  // Which passes can start with a measurement projector pending: one is left
  // by every pass whose scalar phase draws, and applied by the next pass that
  // stores the state (surely if it holds an unconditional gate, or flushes).
  {
    bool pending = false;
    for (DPass& d : P.passes) {
      d.proj = pending ? 1 : 0;
      bool draws = false, stores = d.flush != 0;
      for (uint32_t c = 0; c < d.nc; ++c) {
        const uint8_t k = P.scalars[d.c0 + c].kind;
        draws = draws || k == S_MEASURE || k == S_RESET;
      }
      for (uint32_t g = 0; g < d.ng && !stores; ++g) stores = P.gates[d.g0 + g].flag < 0;
      pending = draws || (pending && !stores);
    }
    // The first pass generates the initial state when it surely stores (an
    // unconditional gate): the tile holding index 0 starts as |0...0>, every
    // other tile is zero before and after the pass.  It runs as the variant
    // that handles per-tile zeroing.
    if (!P.passes.empty()) {
      DPass& d = P.passes[0];
      bool stores = false;
      for (uint32_t g = 0; g < d.ng && !stores; ++g) stores = P.gates[d.g0 + g].flag < 0;
      if (stores && d.ns > 0) {
        P.gen_init = true;
        d.proj = 1;
      }
    }
  }

  P.stats.kernels_per_run = 1 + (P.gen_init ? 0 : 1) + P.passes.size();
  P.stats.records = n_ops;
  P.stats.unrolled_ops = n_gates + n_draws;
  P.stats.gates = n_gates;
  P.stats.draws = n_draws;
  P.stats.passes = P.passes.size();
  P.stats.stages = P.stages.size();
  P.stats.flags = P.n_flags;
  P.stats.tile_bits = P.m;
  P.stats.low_bits = P.L;
  P.stats.plan_bytes = P.passes.size() * sizeof(DPass) + P.gates.size() * sizeof(DGate) +
                       P.stages.size() * sizeof(DStage) + (P.scalars.size() + P.init_items.size()) * sizeof(DScalar) +
                       P.jobs.size() * sizeof(DJob) + P.consts.size() * sizeof(double);
  const int bad = check_barriers(P, &P.stats.warp_barriers, &P.stats.block_barriers);
  if (bad) {
    err = "internal: " + std::to_string(bad) + " stage barrier flags fail the ownership check";
    return SV_ERR_UNSUPPORTED;
  }
  return SV_OK;
}

sv_status build_adjoint_plan(int n, int dtype, const sv_op* ops, size_t n_ops, const double* dense_pool,
                             size_t dense_len, const Tuning& tune, Plan& fwd, Plan& bwd, std::string& err) {
  sv_status st = build_plan(n, dtype, ops, n_ops, dense_pool, dense_len, tune, fwd, err);
  if (st != SV_OK) return st;
  if (fwd.stats.draws || fwd.n_flags) {
    err = "adjoint gradients need a program without measurement, reset or COND";
    return SV_ERR_UNSUPPORTED;
  }
  Unroller U;
  U.ops = ops;
  U.n_ops = n_ops;
  U.n = n;
  U.pool = dense_pool;
  U.pool_len = dense_pool ? dense_len : 0;
  if (!U.walk(0, n_ops, -1, 0)) {
    err = U.err;
    return U.st;
  }
  std::vector<Item> rev(U.items.rbegin(), U.items.rend());
  for (const Item& it : rev) {
    if (it.nq > ADJ_REG_BITS) {
      err = "adjoint gradients support dense unitaries on at most 3 qubits";
      return SV_ERR_UNSUPPORTED;
    }
    if (it.gate >= 0)
      for (int k = 0; k < 3; ++k)
        if (it.pidx[k] >= MAX_ADJ_PARAMS) {
          err = "adjoint gradients support at most 1024 parameters";
          return SV_ERR_UNSUPPORTED;
        }
  }
  bwd = Plan{};
  bwd.n = fwd.n;
  bwd.n_int = fwd.n_int;
  bwd.dtype = dtype;
  bwd.m = fwd.m;
  bwd.L = fwd.L;
  bwd.n_params_needed = fwd.n_params_needed;
  Builder b(bwd, rev, dtype == SV_C64 ? 1 : 0, tune.max_pass_gates);
  b.reg_bits = ADJ_REG_BITS;
  b.adjoint = true;
  Segment seg;
  for (size_t i = 0; i < rev.size(); ++i) seg.gates.push_back(int(i));
  if (!seg.gates.empty()) b.emit_segment(seg);
  bwd.stats.gates = fwd.stats.gates;
  bwd.stats.passes = bwd.passes.size();
  bwd.stats.stages = bwd.stages.size();
  bwd.stats.tile_bits = bwd.m;
  bwd.stats.low_bits = bwd.L;
  return SV_OK;
}

}  // namespace svp
