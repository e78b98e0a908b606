/*
 * sv_oracle.c -- FP64 reference simulator for dynamic circuits.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  The CUDA
 * product path never calls it, and it shares no code with that path: the only
 * thing in common is the byte layout of the op records (the input format).
 *
 * What it computes is the plain textbook definition of a state-vector
 * trajectory of a dynamic circuit, as the paper uses it: gates act on the
 * amplitude vector; a mid-circuit measurement projects the state onto the
 * observed outcome (Sec. II-C, Fig. 2 and its text); an `if` on classical
 * bits is decided from the measured record while the trajectory runs, not by
 * simulating every branch in advance (Sec. III-C); loops with a fixed trip
 * count are run by repetition (Abstract); runtime `input` parameters supply
 * angles (Sec. III-D).  Every
 * loop below is written for obviousness, not speed: one pass over the vector
 * per gate, FP64 complex arithmetic, sums in a fixed left-to-right chunked
 * order so that results do not depend on the thread count.
 *
 * Readings where the paper is silent (qubit order, outcome rule, the draw
 * key, renormalisation) are the ones listed in the design notes:
 *   - qubit q is bit q of the amplitude index, classical bit j is bit j of
 *     a 64-bit register;
 *   - u = Philox4x64-10(key = (seed, stream), ctr = (shot, m, 0, 0)) word 0,
 *     u = (w >> 11) * 2^-53, m = number of measure/reset ops executed
 *     before this one in the trajectory;
 *   - outcome = 1 iff u >= p0 / (p0 + p1);
 *   - collapse: zero the other half and scale by 1/sqrt(p_outcome).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ---------------------------------------------------------------- input format */

enum { K_GATE = 1, K_DENSE = 2, K_MEASURE = 3, K_RESET = 4, K_COND = 5, K_LOOP = 6 };

enum {
  G_I = 0, G_H, G_X, G_Y, G_Z, G_S, G_SDG, G_T, G_TDG, G_SX, G_RX, G_RY, G_RZ, G_P, G_U,
  G_CX, G_CY, G_CZ, G_SWAP, G_CP, G_CRX, G_CRY, G_CRZ, G_CH, G_CU, G_COUNT
};

typedef struct {
  uint16_t kind, gate;
  uint32_t cbit;
  int32_t q[8];
  int32_t pidx[3];
  uint32_t nq;
  double angle[3];
  uint64_t mask, value;
  uint32_t then_len, else_len, loop_k, body_len;
  uint64_t dense_off;
} orc_op;

_Static_assert(sizeof(orc_op) == 120, "op record layout");

typedef struct {
  uint64_t x_mask, z_mask;
  double coeff;
} orc_pauli;

typedef struct {
  int32_t qubit;    /* measured qubit                                  */
  int32_t is_reset; /* 1 for RESET, 0 for MEASURE                      */
  int32_t outcome;
  int32_t forced;   /* 1 if the outcome was imposed by the caller      */
  double p0, p1;    /* raw probabilities of bit = 0 / 1                */
  double u;         /* the uniform draw                                */
  double margin;    /* |u - p0/(p0+p1)|                                */
} orc_draw;

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_ZERO = -2 };

#define CHUNK 4096 /* fixed summation chunk (amplitudes) */
/* states below this size run their loops on one thread: the threads of a
 * parallel region cost more than the loop itself there (results do not
 * depend on the thread count: sums are chunked in a fixed order) */
#define OMP_MIN_AMPS (1ULL << 14)
#define OMP_MIN_CHUNKS 4

/* ---------------------------------------------------------------- Philox4x64-10 */
/*
 * Counter-based generator of Salmon, Moraes, Dror and Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3" (SC'11), Philox-4x64 with 10 rounds.  One round
 * multiplies words 0 and 2 of the counter by the two Philox multipliers,
 * and mixes the high halves with words 1 and 3 and the round key; the key is
 * bumped by the two Weyl constants between rounds.
 */
static const uint64_t PH_M0 = 0xD2E7470EE14C6C93ULL, PH_M1 = 0xCA5A826395121157ULL;
static const uint64_t PH_W0 = 0x9E3779B97F4A7C15ULL, PH_W1 = 0xBB67AE8584CAA73BULL;

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += PH_W0;
      k1 += PH_W1;
    }
    unsigned __int128 p0 = (unsigned __int128)PH_M0 * c0;
    unsigned __int128 p1 = (unsigned __int128)PH_M1 * c2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u in [0,1) with 53 random bits, drawn for (seed, stream, shot, m). */
double orc_uniform(uint64_t seed, uint64_t stream, uint64_t shot, uint64_t m) {
  uint64_t ctr[4] = {shot, m, 0, 0}, key[2] = {seed, stream}, w[4];
  orc_philox4x64_10(ctr, key, w);
  return (double)(w[0] >> 11) * 0x1.0p-53;
}

/* ---------------------------------------------------------------- gate matrices */
/*
 * The OpenQASM 3 standard-library meanings of the gates the transpiler maps
 * one-to-one (Sec. III-B).  Returns the 2x2 matrix m = [m00 m01; m10 m11]
 * acting on the target, and the gate's shape: 1 = one-qubit gate on q[0];
 * 2 = controlled gate (control q[0], target q[1], m applied where the
 * control bit is 1); 3 = SWAP(q[0], q[1]); 0 = unknown gate.
 */
int orc_gate_matrix(int gate, const double a[3], cplx m[4]) {
  const double r2 = 1.0 / sqrt(2.0);
  double c, s;
  switch (gate) {
    case G_I: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 1; return 1;
    case G_H: m[0] = r2; m[1] = r2; m[2] = r2; m[3] = -r2; return 1;
    case G_X: m[0] = 0; m[1] = 1; m[2] = 1; m[3] = 0; return 1;
    case G_Y: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0; return 1;
    case G_Z: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -1; return 1;
    case G_S: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = I; return 1;
    case G_SDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = -I; return 1;
    case G_T: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * M_PI / 4); return 1;
    case G_TDG: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(-I * M_PI / 4); return 1;
    case G_SX: /* sqrt(X) = (1/2)[1+i 1-i; 1-i 1+i] */
      m[0] = 0.5 * (1 + I); m[1] = 0.5 * (1 - I); m[2] = 0.5 * (1 - I); m[3] = 0.5 * (1 + I); return 1;
    case G_RX: /* exp(-i a X / 2) */
      c = cos(a[0] / 2); s = sin(a[0] / 2);
      m[0] = c; m[1] = -I * s; m[2] = -I * s; m[3] = c; return 1;
    case G_RY: /* exp(-i a Y / 2) */
      c = cos(a[0] / 2); s = sin(a[0] / 2);
      m[0] = c; m[1] = -s; m[2] = s; m[3] = c; return 1;
    case G_RZ: /* exp(-i a Z / 2) */
      m[0] = cexp(-I * a[0] / 2); m[1] = 0; m[2] = 0; m[3] = cexp(I * a[0] / 2); return 1;
    case G_P: /* diag(1, e^{i a}) */
      m[0] = 1; m[1] = 0; m[2] = 0; m[3] = cexp(I * a[0]); return 1;
    case G_U: /* U(theta, phi, lambda) */
      c = cos(a[0] / 2); s = sin(a[0] / 2);
      m[0] = c; m[1] = -cexp(I * a[2]) * s; m[2] = cexp(I * a[1]) * s; m[3] = cexp(I * (a[1] + a[2])) * c;
      return 1;
    case G_CX: orc_gate_matrix(G_X, a, m); return 2;
    case G_CY: orc_gate_matrix(G_Y, a, m); return 2;
    case G_CZ: orc_gate_matrix(G_Z, a, m); return 2;
    case G_CH: orc_gate_matrix(G_H, a, m); return 2;
    case G_CP: orc_gate_matrix(G_P, a, m); return 2;
    case G_CRX: orc_gate_matrix(G_RX, a, m); return 2;
    case G_CRY: orc_gate_matrix(G_RY, a, m); return 2;
    case G_CRZ: orc_gate_matrix(G_RZ, a, m); return 2;
    case G_CU: orc_gate_matrix(G_U, a, m); return 2;
    case G_SWAP: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 1; return 3;
    default: return 0;
  }
}

static int gate_qubits(int gate) {
  if (gate >= G_CX && gate <= G_CU) return 2;
  return 1;
}

/* ---------------------------------------------------------------- amplitude loops */

/* psi <- (one-qubit m on q) psi; where ctrl >= 0, only on indices whose ctrl bit is 1. */
static void apply_1q(cplx* psi, int n, int q, int ctrl, const cplx m[4]) {
  const uint64_t N = 1ULL << n, bq = 1ULL << q;
  const uint64_t bc = ctrl >= 0 ? 1ULL << ctrl : 0;
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_AMPS)
  for (uint64_t i = 0; i < N; ++i) {
    if (i & bq) continue;
    if (ctrl >= 0 && !(i & bc)) continue;
    uint64_t j = i | bq;
    cplx a = psi[i], b = psi[j];
    psi[i] = m[0] * a + m[1] * b;
    psi[j] = m[2] * a + m[3] * b;
  }
}

/* SWAP(a, b): exchange the amplitudes whose bits a and b differ. */
static void apply_swap(cplx* psi, int n, int a, int b) {
  const uint64_t N = 1ULL << n, ba = 1ULL << a, bb = 1ULL << b;
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_AMPS)
  for (uint64_t i = 0; i < N; ++i) {
    if ((i & ba) && !(i & bb)) {
      uint64_t j = (i ^ ba) | bb;
      cplx t = psi[i];
      psi[i] = psi[j];
      psi[j] = t;
    }
  }
}

/* dense 2^k x 2^k unitary on (q_0..q_{k-1}), local bit r <-> q_r, row-major. */
static void apply_dense(cplx* psi, int n, int k, const int32_t* qs, const cplx* u) {
  const uint64_t N = 1ULL << n, K = 1ULL << k;
  uint64_t qmask = 0;
  for (int r = 0; r < k; ++r) qmask |= 1ULL << qs[r];
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_AMPS)
  for (uint64_t base = 0; base < N; ++base) {
    if (base & qmask) continue;
    cplx v[256], w[256];
    uint64_t idx[256];
    for (uint64_t r = 0; r < K; ++r) {
      uint64_t i = base;
      for (int b = 0; b < k; ++b)
        if ((r >> b) & 1) i |= 1ULL << qs[b];
      idx[r] = i;
      v[r] = psi[i];
    }
    for (uint64_t r = 0; r < K; ++r) {
      cplx acc = 0;
      for (uint64_t c = 0; c < K; ++c) acc += u[r * K + c] * v[c];
      w[r] = acc;
    }
    for (uint64_t r = 0; r < K; ++r) psi[idx[r]] = w[r];
  }
}

/* Sum of |psi_i|^2 over indices whose bit q equals `bit` (q < 0: all), in a
 * fixed order: left to right inside each CHUNK, chunk sums left to right. */
static double prob_sum(const cplx* psi, int n, int q, int bit) {
  const uint64_t N = 1ULL << n;
  const uint64_t nchunks = (N + CHUNK - 1) / CHUNK;
  double* part = (double*)malloc(sizeof(double) * nchunks);
#pragma omp parallel for schedule(static) if (nchunks > OMP_MIN_CHUNKS)
  for (uint64_t c = 0; c < nchunks; ++c) {
    double s = 0;
    uint64_t lo = c * CHUNK, hi = lo + CHUNK < N ? lo + CHUNK : N;
    for (uint64_t i = lo; i < hi; ++i) {
      if (q >= 0 && (int)((i >> q) & 1) != bit) continue;
      s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    }
    part[c] = s;
  }
  double s = 0;
  for (uint64_t c = 0; c < nchunks; ++c) s += part[c];
  free(part);
  return s;
}

double orc_norm2(const cplx* psi, int n) { return prob_sum(psi, n, -1, 0); }

/* ---------------------------------------------------------------- interpreter */

typedef struct {
  int n;
  cplx* psi;
  const orc_op* ops;
  size_t n_ops;
  const double* params;
  size_t n_params;
  const cplx* pool;
  size_t pool_len;
  uint64_t seed, stream, shot;
  uint64_t creg;
  uint64_t m; /* executed draws so far */
  const int32_t* forced;
  size_t n_forced;
  orc_draw* draws;
  size_t max_draws;
  double* norms; /* optional: norm^2 after every executed op */
  size_t max_norms, n_norms;
  int depth;
  int err;
} orc_ctx;

static double resolve_angle(const orc_ctx* cx, const orc_op* op, int i) {
  if (op->pidx[i] >= 0) return op->angle[i] * cx->params[op->pidx[i]];
  return op->angle[i];
}

static void record_norm(orc_ctx* cx) {
  if (cx->norms && cx->n_norms < cx->max_norms) cx->norms[cx->n_norms] = orc_norm2(cx->psi, cx->n);
  cx->n_norms++;
}

/* Mid-circuit measurement of qubit q (Fig. 2): Born probabilities, one
 * Philox draw, collapse onto the outcome and renormalise.  Returns the outcome. */
static int measure(orc_ctx* cx, int q, int is_reset) {
  double p0 = prob_sum(cx->psi, cx->n, q, 0);
  double p1 = prob_sum(cx->psi, cx->n, q, 1);
  if (!(p0 + p1 > 0)) {
    cx->err = ORC_ERR_ZERO;
    return 0;
  }
  double u = orc_uniform(cx->seed, cx->stream, cx->shot, cx->m);
  double thr = p0 / (p0 + p1);
  int outcome = u >= thr ? 1 : 0;
  int forced = 0;
  if (cx->forced && cx->m < cx->n_forced && cx->forced[cx->m] >= 0) {
    outcome = cx->forced[cx->m] ? 1 : 0;
    forced = 1;
  }
  if (cx->draws && cx->m < cx->max_draws) {
    orc_draw* d = &cx->draws[cx->m];
    d->qubit = q; d->is_reset = is_reset; d->outcome = outcome; d->forced = forced;
    d->p0 = p0; d->p1 = p1; d->u = u; d->margin = fabs(u - thr);
  }
  cx->m++;
  double p = outcome ? p1 : p0;
  if (!(p > 0)) {
    cx->err = ORC_ERR_ZERO;
    return outcome;
  }
  const double scale = 1.0 / sqrt(p);
  const uint64_t N = 1ULL << cx->n;
  cplx* psi = cx->psi;
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_AMPS)
  for (uint64_t i = 0; i < N; ++i) {
    if ((int)((i >> q) & 1) == outcome) psi[i] *= scale;
    else psi[i] = 0;
  }
  return outcome;
}

static int valid_qubit(const orc_ctx* cx, int32_t q) { return q >= 0 && q < cx->n; }

static void exec_range(orc_ctx* cx, size_t begin, size_t end);

static void exec_op(orc_ctx* cx, size_t i, size_t* next) {
  const orc_op* op = &cx->ops[i];
  *next = i + 1;
  switch (op->kind) {
    case K_GATE: {
      double a[3];
      cplx m[4];
      for (int k = 0; k < 3; ++k) {
        if (op->pidx[k] >= 0 && (size_t)op->pidx[k] >= cx->n_params) { cx->err = ORC_ERR_ARG; return; }
        a[k] = resolve_angle(cx, op, k);
      }
      int shape = orc_gate_matrix(op->gate, a, m);
      int nq = gate_qubits(op->gate);
      if (shape == 0 || op->gate >= G_COUNT) { cx->err = ORC_ERR_ARG; return; }
      for (int k = 0; k < nq; ++k)
        if (!valid_qubit(cx, op->q[k])) { cx->err = ORC_ERR_ARG; return; }
      if (nq == 2 && op->q[0] == op->q[1]) { cx->err = ORC_ERR_ARG; return; }
      if (shape == 1) apply_1q(cx->psi, cx->n, op->q[0], -1, m);
      else if (shape == 2) apply_1q(cx->psi, cx->n, op->q[1], op->q[0], m);
      else apply_swap(cx->psi, cx->n, op->q[0], op->q[1]);
      record_norm(cx);
      return;
    }
    case K_DENSE: {
      int k = (int)op->nq;
      if (k < 1 || k > 8) { cx->err = ORC_ERR_ARG; return; }
      uint64_t seen = 0;
      for (int r = 0; r < k; ++r) {
        if (!valid_qubit(cx, op->q[r]) || (seen >> op->q[r]) & 1) { cx->err = ORC_ERR_ARG; return; }
        seen |= 1ULL << op->q[r];
      }
      uint64_t need = (1ULL << k) * (1ULL << k);
      if (!cx->pool || op->dense_off + need > cx->pool_len) { cx->err = ORC_ERR_ARG; return; }
      apply_dense(cx->psi, cx->n, k, op->q, cx->pool + op->dense_off);
      record_norm(cx);
      return;
    }
    case K_MEASURE: {
      if (!valid_qubit(cx, op->q[0]) || op->cbit >= 64) { cx->err = ORC_ERR_ARG; return; }
      int o = measure(cx, op->q[0], 0);
      cx->creg = (cx->creg & ~(1ULL << op->cbit)) | ((uint64_t)o << op->cbit);
      record_norm(cx);
      return;
    }
    case K_RESET: {
      if (!valid_qubit(cx, op->q[0])) { cx->err = ORC_ERR_ARG; return; }
      int o = measure(cx, op->q[0], 1);
      if (o) {
        cplx x[4] = {0, 1, 1, 0};
        apply_1q(cx->psi, cx->n, op->q[0], -1, x);
      }
      record_norm(cx);
      return;
    }
    case K_COND: {
      /* Sec. III-C: the predicate is read from the classical record *now*. */
      size_t t0 = i + 1, t1 = t0 + op->then_len, e1 = t1 + op->else_len;
      if (e1 > cx->n_ops) { cx->err = ORC_ERR_ARG; return; }
      *next = e1;
      if ((cx->creg & op->mask) == op->value) exec_range(cx, t0, t1);
      else exec_range(cx, t1, e1);
      return;
    }
    case K_LOOP: {
      size_t b0 = i + 1, b1 = b0 + op->body_len;
      if (b1 > cx->n_ops) { cx->err = ORC_ERR_ARG; return; }
      *next = b1;
      for (uint32_t r = 0; r < op->loop_k && !cx->err; ++r) exec_range(cx, b0, b1);
      return;
    }
    default:
      cx->err = ORC_ERR_ARG;
      return;
  }
}

static void exec_range(orc_ctx* cx, size_t begin, size_t end) {
  if (++cx->depth > 64) { cx->err = ORC_ERR_ARG; cx->depth--; return; }
  size_t i = begin;
  while (i < end && !cx->err) {
    size_t next;
    exec_op(cx, i, &next);
    i = next;
  }
  cx->depth--;
}

/*
 * One trajectory from |0...0>.  psi (2^n complex128) is written by the call.
 * forced[m] >= 0 imposes the outcome of draw m (used to follow another
 * simulator's record through a near-threshold draw); draws[] receives one
 * record per executed measure/reset; norms[] the squared norm after every
 * executed gate/measure/reset.  Returns ORC_OK or an error code.
 */
int orc_run(int n, const void* ops, size_t n_ops, const double* params, size_t n_params,
            const cplx* pool, size_t pool_len, uint64_t seed, uint64_t stream, uint64_t shot,
            const int32_t* forced, size_t n_forced, cplx* psi, uint64_t* creg_out,
            orc_draw* draws, size_t max_draws, size_t* n_draws,
            double* norms, size_t max_norms, size_t* n_norms) {
  if (n < 1 || n > 34 || !psi) return ORC_ERR_ARG;
  orc_ctx cx;
  memset(&cx, 0, sizeof cx);
  cx.n = n; cx.psi = psi; cx.ops = (const orc_op*)ops; cx.n_ops = n_ops;
  cx.params = params; cx.n_params = params ? n_params : 0;
  cx.pool = pool; cx.pool_len = pool ? pool_len : 0;
  cx.seed = seed; cx.stream = stream; cx.shot = shot;
  cx.forced = forced; cx.n_forced = forced ? n_forced : 0;
  cx.draws = draws; cx.max_draws = draws ? max_draws : 0;
  cx.norms = norms; cx.max_norms = norms ? max_norms : 0;
  const uint64_t N = 1ULL << n;
#pragma omp parallel for schedule(static) if (N >= OMP_MIN_AMPS)
  for (uint64_t i = 0; i < N; ++i) psi[i] = 0;
  psi[0] = 1;
  exec_range(&cx, 0, n_ops);
  if (creg_out) *creg_out = cx.creg;
  if (n_draws) *n_draws = cx.m;
  if (n_norms) *n_norms = cx.n_norms;
  return cx.err;
}

/* ---------------------------------------------------------------- terminal sampling */
/*
 * Terminal samples from |psi|^2: CDF c_i = sum_{j<=i} |psi_j|^2 accumulated
 * left to right; shot s draws u = uniform(seed, stream, shot0 + s, m_index)
 * and returns the smallest i with c_i > u * c_{N-1}.  margin[s] is the
 * distance of u * c_{N-1} to the nearest CDF boundary, over c_{N-1}.
 */
int orc_sample(int n, const cplx* psi, uint64_t shots, uint64_t seed, uint64_t stream,
               uint64_t shot0, uint64_t m_index, uint64_t* out, double* margin) {
  if (n < 1 || n > 34) return ORC_ERR_ARG;
  const uint64_t N = 1ULL << n;
  double* cdf = (double*)malloc(sizeof(double) * N);
  if (!cdf) return ORC_ERR_ARG;
  double acc = 0;
  for (uint64_t i = 0; i < N; ++i) {
    acc += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    cdf[i] = acc;
  }
  const double total = cdf[N - 1];
  for (uint64_t s = 0; s < shots; ++s) {
    double t = orc_uniform(seed, stream, shot0 + s, m_index) * total;
    uint64_t lo = 0, hi = N - 1; /* invariant: answer in [lo, hi] */
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      if (cdf[mid] > t) hi = mid;
      else lo = mid + 1;
    }
    out[s] = lo;
    if (margin) {
      double d = cdf[lo] - t;
      if (lo > 0 && t - cdf[lo - 1] < d) d = t - cdf[lo - 1];
      margin[s] = d / total;
    }
  }
  free(cdf);
  return ORC_OK;
}

/* ---------------------------------------------------------------- Pauli expectation */
/*
 * <psi| P |psi> for each Pauli string P (X on qubit q iff bit q of x_mask, Z
 * iff bit q of z_mask, Y iff both), by applying the one-qubit Pauli
 * matrices to a copy and taking the inner product (the energy <H> checked
 * in the paper's VQE experiment, Sec. IV-A.2 and Sec. IV-D).  per_term[t]
 * receives the real part; *total the coefficient-weighted sum.
 */
int orc_expval(int n, const cplx* psi, const void* terms_v, size_t n_terms, double* per_term,
               double* total) {
  if (n < 1 || n > 34) return ORC_ERR_ARG;
  const orc_pauli* terms = (const orc_pauli*)terms_v;
  const uint64_t N = 1ULL << n;
  cplx* phi = (cplx*)malloc(sizeof(cplx) * N);
  if (!phi) return ORC_ERR_ARG;
  const uint64_t nchunks = (N + CHUNK - 1) / CHUNK;
  double* part = (double*)malloc(sizeof(double) * nchunks);
  const cplx PX[4] = {0, 1, 1, 0}, PY[4] = {0, -I, I, 0}, PZ[4] = {1, 0, 0, -1};
  double tot = 0;
  for (size_t t = 0; t < n_terms; ++t) {
    memcpy(phi, psi, sizeof(cplx) * N);
    for (int q = 0; q < n; ++q) {
      int x = (terms[t].x_mask >> q) & 1, z = (terms[t].z_mask >> q) & 1;
      if (x && z) apply_1q(phi, n, q, -1, PY);
      else if (x) apply_1q(phi, n, q, -1, PX);
      else if (z) apply_1q(phi, n, q, -1, PZ);
    }
    if ((terms[t].x_mask | terms[t].z_mask) >> n) { free(phi); free(part); return ORC_ERR_ARG; }
#pragma omp parallel for schedule(static) if (nchunks > OMP_MIN_CHUNKS)
    for (uint64_t c = 0; c < nchunks; ++c) {
      double s = 0;
      uint64_t lo = c * CHUNK, hi = lo + CHUNK < N ? lo + CHUNK : N;
      for (uint64_t i = lo; i < hi; ++i) s += creal(conj(psi[i]) * phi[i]);
      part[c] = s;
    }
    double e = 0;
    for (uint64_t c = 0; c < nchunks; ++c) e += part[c];
    if (per_term) per_term[t] = e;
    tot += terms[t].coeff * e;
  }
  if (total) *total = tot;
  free(phi);
  free(part);
  return ORC_OK;
}

/* ---------------------------------------------------------------- misc */

void orc_set_threads(int k) {
#ifdef _OPENMP
  if (k > 0) omp_set_num_threads(k);
#else
  (void)k;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
