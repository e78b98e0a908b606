// kern_clifford.cu -- stabilizer-tableau fast path for Clifford programs.
//
// A program whose gates are Clifford (the paper's static suite is random
// Clifford circuits, Sec. IV-A.2, and it runs such programs on a stabilizer
// backend, Fig. 1c) keeps its state a stabilizer state through measurement,
// reset and feed-forward, so each shot is a tableau of 2n Pauli rows
// (Aaronson and Gottesman 2004: rows 0..n-1 destabilisers, n..2n-1
// stabilisers; x bits, z bits, sign) instead of 2^n amplitudes.  One warp
// runs one shot: with n <= 64 a row is one 64-bit x word and one z word, and
// lane l holds rows l, l+32, l+64, l+96 in registers.
//
// Gates conjugate every row (bit rules below).  Measuring qubit q:
//   random       some stabiliser p has x_q = 1 (the smallest such p): every
//                other row with x_q = 1 becomes its product with row p, the
//                destabiliser p-n takes row p, and row p becomes +-Z_q with
//                the drawn outcome as its sign;
//   deterministic the outcome is the sign of the product of the stabilisers
//                n+i whose destabiliser i has x_q = 1 (they commute, so the
//                warp multiplies them in a shuffle tree).
// Draws follow the state-vector engine's convention: the m-th measure/reset
// of shot s reads u(seed, stream, s, m); outcome 1 iff u >= p0/(p0+p1), which
// for a random stabiliser outcome (p0 = p1) is u >= 1/2.  Records therefore
// equal the state-vector engine's except where its rounded p0/(p0+p1) and 1/2
// straddle u.
//
// Feed-forward: COND records lower to a conditional jump over the then
// branch (and an unconditional jump over the else branch); LOOP records are
// unrolled.  No control decision leaves the warp.
#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sv.h"
#include "dev_common.cuh"

namespace svapi {
void set_last_error(const std::string& msg);
}

namespace svc {

enum COp : uint8_t { C_H = 1, C_S, C_SDG, C_SX, C_X, C_Y, C_Z, C_CX, C_CZ, C_SWAP, C_MEAS, C_RESET, C_COND, C_JUMP };

struct CInstr {
  uint8_t op, a, b, pad;
  uint32_t tgt;  // MEAS: classical bit; COND: next pc when the predicate fails; JUMP: next pc
  uint64_t mask, value;
};
static_assert(sizeof(CInstr) == 24, "instruction layout");

constexpr int CL_MAXQ = 64;
constexpr int CL_SLOTS = 4;  // 2n <= 128 rows over 32 lanes
constexpr uint32_t CL_MAX_INSTR = 1u << 24;

struct CliffArgs {
  const CInstr* prog;
  uint32_t len;
  int n;
  uint64_t seed, stream, shot0, shots;
  uint64_t* out;
};

struct Rows {
  uint64_t x[CL_SLOTS], z[CL_SLOTS];
  uint32_t r;  // bit k: sign of slot k
};

static __device__ __forceinline__ uint32_t bitq(uint64_t v, int q) { return uint32_t(v >> q) & 1u; }

// Sign of row_i * row_h (both Hermitian and commuting, or the result is not
// used): the exponent of i collected qubit by qubit is +1 for XY, YZ, ZX and
// -1 for YX, ZY, XZ (first factor row i); with the two signs it is 0 or 2 mod 4.
static __device__ __forceinline__ uint32_t product_sign(uint64_t hx, uint64_t hz, uint32_t hr, uint64_t ix,
                                                        uint64_t iz, uint32_t ir) {
  const uint64_t a = ix, b = iz, c = hx, d = hz;
  const uint64_t plus = (a & b & ~c & d) | (a & ~b & c & d) | (~a & b & c & ~d);
  const uint64_t minus = (a & b & c & ~d) | (a & ~b & ~c & d) | (~a & b & c & d);
  const int s = 2 * int(hr) + 2 * int(ir) + __popcll(plus) - __popcll(minus);
  return ((s & 3) == 2) ? 1u : 0u;
}

static __device__ __forceinline__ void set_sign(Rows& R, int k, uint32_t v) { R.r = (R.r & ~(1u << k)) | (v << k); }

static __device__ __forceinline__ void g_one(Rows& R, uint8_t op, int q) {
#pragma unroll
  for (int k = 0; k < CL_SLOTS; ++k) {
    const uint32_t xb = bitq(R.x[k], q), zb = bitq(R.z[k], q);
    switch (op) {
      case C_H: {  // X <-> Z, Y -> -Y
        R.r ^= (xb & zb) << k;
        const uint64_t d = uint64_t(xb ^ zb) << q;
        R.x[k] ^= d;
        R.z[k] ^= d;
      } break;
      case C_S:  // X -> Y, Y -> -X
        R.r ^= (xb & zb) << k;
        R.z[k] ^= uint64_t(xb) << q;
        break;
      case C_SDG:  // X -> -Y, Y -> X
        R.r ^= (xb & (zb ^ 1u)) << k;
        R.z[k] ^= uint64_t(xb) << q;
        break;
      case C_SX:  // Z -> -Y, Y -> Z
        R.r ^= (zb & (xb ^ 1u)) << k;
        R.x[k] ^= uint64_t(zb) << q;
        break;
      case C_X:
        R.r ^= zb << k;
        break;
      case C_Y:
        R.r ^= (xb ^ zb) << k;
        break;
      default:  // C_Z
        R.r ^= xb << k;
        break;
    }
  }
}

static __device__ __forceinline__ void g_two(Rows& R, uint8_t op, int a, int b) {
#pragma unroll
  for (int k = 0; k < CL_SLOTS; ++k) {
    const uint32_t xa = bitq(R.x[k], a), za = bitq(R.z[k], a), xb = bitq(R.x[k], b), zb = bitq(R.z[k], b);
    if (op == C_CX) {  // control a, target b
      R.r ^= (xa & zb & (xb ^ za ^ 1u)) << k;
      R.x[k] ^= uint64_t(xa) << b;
      R.z[k] ^= uint64_t(zb) << a;
    } else if (op == C_CZ) {
      R.r ^= (xa & xb & (za ^ zb)) << k;
      R.z[k] ^= (uint64_t(xb) << a) | (uint64_t(xa) << b);
    } else {  // C_SWAP
      const uint64_t dx = uint64_t(xa ^ xb), dz = uint64_t(za ^ zb);
      R.x[k] ^= (dx << a) | (dx << b);
      R.z[k] ^= (dz << a) | (dz << b);
    }
  }
}

static __device__ __forceinline__ int measure(Rows& R, int q, int n, int lane, const CliffArgs& A, uint64_t shot,
                                              uint64_t m) {
  constexpr unsigned full = 0xffffffffu;
  const int rows = 2 * n;
  uint32_t cand = 0xffffffffu;
#pragma unroll
  for (int k = 0; k < CL_SLOTS; ++k) {
    const int row = lane + 32 * k;
    if (row >= n && row < rows && bitq(R.x[k], q)) cand = min(cand, uint32_t(row));
  }
  const uint32_t p = __reduce_min_sync(full, cand);
  if (p != 0xffffffffu) {  // random outcome
    const int kp = int(p >> 5), lp = int(p & 31u);
    uint64_t sx = 0, sz = 0;
    uint32_t sr = 0;
#pragma unroll
    for (int k = 0; k < CL_SLOTS; ++k)
      if (k == kp) {
        sx = R.x[k];
        sz = R.z[k];
        sr = (R.r >> k) & 1u;
      }
    const uint64_t px = __shfl_sync(full, sx, lp), pz = __shfl_sync(full, sz, lp);
    const uint32_t pr = __shfl_sync(full, sr, lp);
#pragma unroll
    for (int k = 0; k < CL_SLOTS; ++k) {
      const int row = lane + 32 * k;
      if (row < rows && uint32_t(row) != p && bitq(R.x[k], q)) {
        set_sign(R, k, product_sign(R.x[k], R.z[k], (R.r >> k) & 1u, px, pz, pr));
        R.x[k] ^= px;
        R.z[k] ^= pz;
      }
    }
    const double u = svk::draw_uniform(A.seed, A.stream, shot, m);
    const uint32_t o = (u >= 0.5) ? 1u : 0u;
#pragma unroll
    for (int k = 0; k < CL_SLOTS; ++k) {
      const uint32_t row = uint32_t(lane + 32 * k);
      if (row == p - uint32_t(n)) {
        R.x[k] = px;
        R.z[k] = pz;
        set_sign(R, k, pr);
      }
      if (row == p) {
        R.x[k] = 0;
        R.z[k] = 1ull << q;
        set_sign(R, k, o);
      }
    }
    return int(o);
  }
  // deterministic outcome: destabilisers are rows < n <= 64, slots 0 and 1
  uint64_t dmask = 0;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int row = lane + 32 * k;
    const uint32_t bal = __ballot_sync(full, row < n && bitq(R.x[k], q));
    dmask |= uint64_t(bal) << (32 * k);
  }
  uint64_t ax = 0, az = 0;
  uint32_t ar = 0;
#pragma unroll
  for (int k = 0; k < CL_SLOTS; ++k) {
    const int row = lane + 32 * k;
    if (row >= n && row < rows && ((dmask >> (row - n)) & 1ull)) {
      ar = product_sign(ax, az, ar, R.x[k], R.z[k], (R.r >> k) & 1u);
      ax ^= R.x[k];
      az ^= R.z[k];
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t ox = __shfl_xor_sync(full, ax, off), oz = __shfl_xor_sync(full, az, off);
    const uint32_t orr = __shfl_xor_sync(full, ar, off);
    ar = product_sign(ax, az, ar, ox, oz, orr);
    ax ^= ox;
    az ^= oz;
  }
  return int(ar);
}

__global__ void __launch_bounds__(256) k_clifford(const CliffArgs A) {
  const int lane = int(threadIdx.x & 31u);
  const uint64_t w0 = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = (uint64_t(gridDim.x) * blockDim.x) >> 5;
  const int n = A.n;
  for (uint64_t s = w0; s < A.shots; s += nw) {
    Rows R;
    R.r = 0;
#pragma unroll
    for (int k = 0; k < CL_SLOTS; ++k) {
      const int row = lane + 32 * k;
      R.x[k] = row < n ? (1ull << row) : 0ull;
      R.z[k] = (row >= n && row < 2 * n) ? (1ull << (row - n)) : 0ull;
    }
    const uint64_t shot = A.shot0 + s;
    uint64_t creg = 0, m = 0;
    uint32_t pc = 0;
    while (pc < A.len) {
      const CInstr I = A.prog[pc++];
      switch (I.op) {
        case C_CX:
        case C_CZ:
        case C_SWAP:
          g_two(R, I.op, I.a, I.b);
          break;
        case C_MEAS:
        case C_RESET: {
          const int o = measure(R, I.a, n, lane, A, shot, m);
          ++m;
          if (I.op == C_MEAS) creg = (creg & ~(1ull << I.tgt)) | (uint64_t(o) << I.tgt);
          else if (o) g_one(R, C_X, I.a);
        } break;
        case C_COND:
          if ((creg & I.mask) != I.value) pc = I.tgt;
          break;
        case C_JUMP:
          pc = I.tgt;
          break;
        default:
          g_one(R, I.op, I.a);
          break;
      }
    }
    if (lane == 0) A.out[s] = creg;
  }
}

// ---------------------------------------------------------------- host lowering

struct Lowering {
  const sv_op* ops;
  int n;
  std::vector<CInstr> out;
  std::string err;

  bool emit(uint8_t op, int a, int b = 0) {
    if (out.size() >= CL_MAX_INSTR) {
      err = "Clifford program longer than 2^24 instructions after unrolling";
      return false;
    }
    CInstr I{};
    I.op = op;
    I.a = uint8_t(a);
    I.b = uint8_t(b);
    out.push_back(I);
    return true;
  }

  bool qubit_ok(int q) {
    if (q < 0 || q >= n) {
      err = "qubit " + std::to_string(q) + " out of range";
      return false;
    }
    return true;
  }

  sv_status gate(const sv_op& o) {
    const int q0 = o.q[0], q1 = o.q[1];
    switch (o.gate) {
      case SV_I:
        return qubit_ok(q0) ? SV_OK : SV_ERR_ARG;
      case SV_H: case SV_X: case SV_Y: case SV_Z: case SV_S: case SV_SDG: case SV_SX: {
        if (!qubit_ok(q0)) return SV_ERR_ARG;
        const uint8_t op = o.gate == SV_H ? C_H : o.gate == SV_X ? C_X : o.gate == SV_Y ? C_Y : o.gate == SV_Z ? C_Z
                         : o.gate == SV_S ? C_S : o.gate == SV_SDG ? C_SDG : C_SX;
        return emit(op, q0) ? SV_OK : SV_ERR_UNSUPPORTED;
      }
      case SV_CX: case SV_CY: case SV_CZ: case SV_SWAP: {
        if (!qubit_ok(q0) || !qubit_ok(q1)) return SV_ERR_ARG;
        if (q0 == q1) {
          err = "two-qubit gate on one qubit";
          return SV_ERR_ARG;
        }
        bool ok = true;
        if (o.gate == SV_CX) ok = emit(C_CX, q0, q1);
        else if (o.gate == SV_CZ) ok = emit(C_CZ, q0, q1);
        else if (o.gate == SV_SWAP) ok = emit(C_SWAP, q0, q1);
        else ok = emit(C_SDG, q1) && emit(C_CX, q0, q1) && emit(C_S, q1);  // CY = S_t CX S_t^dagger
        return ok ? SV_OK : SV_ERR_UNSUPPORTED;
      }
      default:
        err = "gate " + std::to_string(o.gate) + " is not in the Clifford set {I, H, X, Y, Z, S, SDG, SX, CX, CY, CZ, SWAP}";
        return SV_ERR_UNSUPPORTED;
    }
  }

  // Instructions the records [i0, i1) unroll to, saturating above the limit
  // (so that an oversized program is refused before anything is emitted).
  uint64_t count(size_t i0, size_t i1) const {
    uint64_t c = 0;
    for (size_t i = i0; i < i1 && c <= CL_MAX_INSTR;) {
      const sv_op& o = ops[i];
      if (o.kind == SV_COND) {
        const size_t t1 = i + 1 + o.then_len, e1 = t1 + o.else_len;
        if (e1 > i1) return c + 1;  // malformed: block() reports it
        c += 2 + count(i + 1, t1) + count(t1, e1);
        i = e1;
      } else if (o.kind == SV_LOOP) {
        const size_t b1 = i + 1 + o.body_len;
        if (b1 > i1) return c + 1;
        const uint64_t body = count(i + 1, b1);
        c += (body && o.loop_k > (CL_MAX_INSTR + 1) / body) ? uint64_t(CL_MAX_INSTR) + 1 : body * o.loop_k;
        i = b1;
      } else {
        c += (o.kind == SV_GATE && o.gate == SV_CY) ? 3 : 1;
        ++i;
      }
    }
    return std::min<uint64_t>(c, uint64_t(CL_MAX_INSTR) + 1);
  }

  sv_status block(size_t i0, size_t i1) {
    for (size_t i = i0; i < i1;) {
      const sv_op& o = ops[i];
      switch (o.kind) {
        case SV_GATE: {
          const sv_status s = gate(o);
          if (s != SV_OK) return s;
          ++i;
        } break;
        case SV_MEASURE:
        case SV_RESET: {
          if (!qubit_ok(o.q[0])) return SV_ERR_ARG;
          if (o.kind == SV_MEASURE && o.cbit >= 64) {
            err = "classical bit out of range";
            return SV_ERR_ARG;
          }
          if (!emit(o.kind == SV_MEASURE ? C_MEAS : C_RESET, o.q[0])) return SV_ERR_UNSUPPORTED;
          out.back().tgt = o.kind == SV_MEASURE ? o.cbit : 0u;
          ++i;
        } break;
        case SV_COND: {
          const size_t t0 = i + 1, t1 = t0 + o.then_len, e1 = t1 + o.else_len;
          if (e1 > i1) {
            err = "COND lengths run past the enclosing block";
            return SV_ERR_ARG;
          }
          if (!emit(C_COND, 0)) return SV_ERR_UNSUPPORTED;
          const size_t c = out.size() - 1;
          out[c].mask = o.mask;
          out[c].value = o.value;
          sv_status s = block(t0, t1);
          if (s != SV_OK) return s;
          if (o.else_len) {
            if (!emit(C_JUMP, 0)) return SV_ERR_UNSUPPORTED;
            const size_t j = out.size() - 1;
            out[c].tgt = uint32_t(out.size());
            s = block(t1, e1);
            if (s != SV_OK) return s;
            out[j].tgt = uint32_t(out.size());
          } else {
            out[c].tgt = uint32_t(out.size());
          }
          i = e1;
        } break;
        case SV_LOOP: {
          const size_t b0 = i + 1, b1 = b0 + o.body_len;
          if (b1 > i1) {
            err = "LOOP body runs past the enclosing block";
            return SV_ERR_ARG;
          }
          for (uint32_t k = 0; k < o.loop_k; ++k) {
            const sv_status s = block(b0, b1);
            if (s != SV_OK) return s;
          }
          i = b1;
        } break;
        case SV_DENSE:
          err = "DENSE records are not Clifford";
          return SV_ERR_UNSUPPORTED;
        default:
          err = "unknown record kind";
          return SV_ERR_ARG;
      }
    }
    return SV_OK;
  }
};

}  // namespace svc

struct sv_clifford {
  int n = 0, sms = 0, grid_max = 0;
  cudaStream_t stream = nullptr;
  svc::CInstr* prog = nullptr;
  uint32_t len = 0;
  uint64_t* out = nullptr;
  size_t out_cap = 0;
  ~sv_clifford() {
    if (prog) cudaFree(prog);
    if (out) cudaFree(out);
  }
};

namespace {
sv_status cl_fail(sv_status s, const std::string& msg) {
  svapi::set_last_error(msg);
  return s;
}
sv_status cl_cuda(cudaError_t e, const char* where) {
  return cl_fail(SV_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
}  // namespace

extern "C" {

sv_status sv_clifford_create(int n, const sv_op* ops, size_t n_ops, void* cuda_stream, sv_clifford** out) {
  if (!out) return cl_fail(SV_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (n < 1 || n > svc::CL_MAXQ) return cl_fail(SV_ERR_ARG, "the Clifford path takes 1 to 64 qubits");
  if (n_ops && !ops) return cl_fail(SV_ERR_ARG, "ops is NULL");
  svc::Lowering L{ops, n, {}, {}};
  if (L.count(0, n_ops) > svc::CL_MAX_INSTR)
    return cl_fail(SV_ERR_UNSUPPORTED, "Clifford program longer than 2^24 instructions after unrolling");
  const sv_status s = L.block(0, n_ops);
  if (s != SV_OK) return cl_fail(s, L.err);
  std::unique_ptr<sv_clifford> c(new sv_clifford());
  c->n = n;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cl_cuda(e, "device query");
  c->grid_max = c->sms * 8;  // 8 CTAs of 8 warps: 64 resident warps per SM
  c->len = uint32_t(L.out.size());
  if (c->len) {
    e = cudaMalloc(&c->prog, c->len * sizeof(svc::CInstr));
    if (e != cudaSuccess) return cl_fail(SV_ERR_OOM, "Clifford program");
    e = cudaMemcpyAsync(c->prog, L.out.data(), c->len * sizeof(svc::CInstr), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cl_cuda(e, "Clifford program upload");
  }
  *out = c.release();
  return SV_OK;
}

sv_status sv_clifford_sample(sv_clifford* c, uint64_t shots, uint64_t seed, uint64_t stream_id, uint64_t shot0,
                             uint64_t* creg_out) {
  if (!c) return cl_fail(SV_ERR_ARG, "null handle");
  if (shots && !creg_out) return cl_fail(SV_ERR_ARG, "creg_out is NULL");
  if (!shots) return SV_OK;
  if (shots > c->out_cap) {
    if (c->out) cudaFree(c->out);
    c->out = nullptr;
    c->out_cap = 0;
    if (cudaMalloc(&c->out, shots * sizeof(uint64_t)) != cudaSuccess) return cl_fail(SV_ERR_OOM, "record buffer");
    c->out_cap = shots;
  }
  svc::CliffArgs a{};
  a.prog = c->prog;
  a.len = c->len;
  a.n = c->n;
  a.seed = seed;
  a.stream = stream_id;
  a.shot0 = shot0;
  a.shots = shots;
  a.out = c->out;
  const uint64_t want = (shots + 7) / 8;
  const int grid = int(std::max<uint64_t>(1, std::min<uint64_t>(want, uint64_t(c->grid_max))));
  svc::k_clifford<<<grid, 256, 0, c->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(creg_out, c->out, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cl_cuda(e, "Clifford sampling");
  return SV_OK;
}

sv_status sv_clifford_destroy(sv_clifford* c) {
  if (!c) return SV_OK;
  cudaStreamSynchronize(c->stream);
  delete c;
  return SV_OK;
}

}  // extern "C"
