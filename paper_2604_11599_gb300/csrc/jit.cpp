// jit.cpp -- NVRTC specialisation of the pass kernel for one lowered program.
#include "jit.h"

#include <cuda.h>
#include <nvrtc.h>

#include <chrono>
#include <functional>
#include <map>
#include <mutex>
#include <sstream>
#include <thread>

#include "jit_headers.inc"

namespace svj {

namespace {

const char* op_template(int op) {
  switch (op) {
    case svp::OP_U: return "g_u";
    case svp::OP_R: return "g_r";
    case svp::OP_RX: return "g_rx";
    case svp::OP_RXF: return "g_rxf";
    case svp::OP_RYF: return "g_ryf";
    case svp::OP_DZ: return "g_dz";
    case svp::OP_D: return "g_d";
    case svp::OP_X: return "g_x";
    case svp::OP_CU: return "g_cu";
    case svp::OP_CX: return "g_cx";
    case svp::OP_CZ: return "g_cz";
    case svp::OP_CD: return "g_cd";
    case svp::OP_SWAP: return "g_swap";
    case svp::OP_U4: return "g_u4";
    case svp::OP_D16: return "d16_apply";
    default: return nullptr;
  }
}

bool two_qubit(int op) {
  return op == svp::OP_CU || op == svp::OP_CX || op == svp::OP_CZ || op == svp::OP_CD || op == svp::OP_SWAP ||
         op == svp::OP_U4;
}

// one straight-line stage program per pass (struct <prefix><pass>).  Without
// direct_ok the last stage of a direct pass writes the tile back to shared
// memory like any other, behind a block barrier (kernels whose tile loop
// stores from shared memory: the CTA-mode forward passes of the adjoint).
void emit_stages(std::ostringstream& o, const svp::Plan& P, size_t pi, const char* prefix = "JS",
                 bool direct_ok = true, bool inline_run = true) {
  const svp::DPass& d = P.passes[pi];
  const int GB = P.m - svp::REG_BITS;
  o << "struct " << prefix << pi << " {\n"
    << "  template <typename T, int M, bool TC>\n"
    << "  static __device__ " << (inline_run ? "__forceinline__" : "__noinline__")
    << " void run(const PassArgs& A, const DPass& sp, const uint32_t* sgk,\n"
    << "                                             const typename CxT<T>::V* smat, typename CxT<T>::V* tb,\n"
    << "                                             TcCtx& tc, const uint64_t base, const typename CxT<T>::V fT,\n"
    << "                                             const bool fscale, const ProjFold& pj) {\n"
    << "    using V = typename CxT<T>::V;\n"
    << "    const int tid = threadIdx.x;\n";
  for (uint32_t si = 0; si < d.ns; ++si) {
    const svp::DStage& st = P.stages[d.s0 + si];
    uint32_t off[16];
    off[0] = 0;
    for (int j = 1; j < 16; ++j) off[j] = off[j & (j - 1)] ^ st.R[__builtin_ctz(unsigned(j))];
    // one group per thread (2^(m-4) == threads): straight-line code, so the
    // group base -- a function of the thread index only -- can stay out of the tile loop
    if ((1 << GB) == svp::PASS_THREADS) o << "    {\n      const int grp = tid;\n";
    else o << "    for (int grp = tid; grp < " << (1 << GB) << "; grp += " << svp::PASS_THREADS << ") {\n";
    o << "      uint32_t b = 0;\n";
    for (int k = 0; k < GB; ++k) o << "      if (grp & " << (1 << k) << ") b ^= " << st.E[k] << "u;\n";
    // complex64 with register bit 0 on tile bit 0: amplitude pairs share a
    // 16-byte granule (the swizzle never touches bit 0), one access per pair
    const bool pairs = P.dtype == SV_C64 && st.R[0] == 1;
    o << "      V a[16];\n";
    if (pairs) {
      for (int j = 0; j < 16; j += 2)
        o << "      { const float4 q = *reinterpret_cast<const float4*>(tb + (b ^ " << off[j] << "u)); a[" << j
          << "] = make_float2(q.x, q.y); a[" << j + 1 << "] = make_float2(q.z, q.w); }\n";
    } else {
      for (int j = 0; j < 16; ++j) o << "      a[" << j << "] = tb[b ^ " << off[j] << "u];\n";
    }
    if (d.proj && si == 0) {
      // the pending projector, on the loaded amplitudes: register j of group grp is
      // tile index li(grp) ^ loff[j]; kept iff ((t ^ px) & pm) == pv, scaled by ps
      uint32_t loff[16];
      loff[0] = 0;
      for (int j = 1; j < 16; ++j) loff[j] = loff[j & (j - 1)] ^ (1u << st.Rb[__builtin_ctz(unsigned(j))]);
      o << "      if (pj.on) {\n        uint32_t li = 0;\n";
      for (int k = 0; k < GB; ++k) o << "        if (grp & " << (1 << k) << ") li |= " << (1u << st.Eb[k]) << "u;\n";
      if (P.dtype == SV_C64 && st.Rb[0] == 0) {  // amplitude pairs in registers: a flip of tile bit 0 swaps them
        o << "        if (pj.swap0) {\n";
        for (int j = 0; j < 16; j += 2) o << "          { const V t = a[" << j << "]; a[" << j << "] = a[" << j + 1 << "]; a[" << j + 1 << "] = t; }\n";
        o << "        }\n";
      }
      o << "        const auto ps = decltype(a[0].x)(pj.ps);\n";
      for (int j = 0; j < 16; ++j)
        o << "        a[" << j << "] = (((li ^ " << loff[j] << "u ^ pj.px) & pj.pm) == pj.pv) ? mkc(a[" << j << "].x * ps, a["
          << j << "].y * ps) : mkc(decltype(ps)(0), decltype(ps)(0));\n";
      o << "      }\n";
    }
    for (uint32_t g = st.g0; g < uint32_t(st.g0) + st.ng; ++g) {
      const svp::DGate& gt = P.gates[d.g0 + g];
      const char* fn = op_template(gt.op);
      if (!fn) {  // a record kind without a template: the module fails to build (generic kernels run)
        o << "#error gate record kind " << int(gt.op) << " has no template\n";
        continue;
      }
      std::ostringstream call;
      call << fn;
      if (gt.op == svp::OP_D16) call << "<T, M, TC>(a, smat + " << gt.mat << ", tb, tc)";
      else if (two_qubit(gt.op)) call << "<" << int(gt.p0) << ", " << int(gt.p1) << ">(a, smat + " << gt.mat << ")";
      else call << "<" << int(gt.p0) << ">(a, smat + " << gt.mat << ")";
      if (gt.flag >= 0) o << "      if (sgk[" << g << "] & SGK_ON) " << call.str() << ";\n";
      else o << "      " << call.str() << ";\n";
    }
    const bool last = si + 1 == d.ns;
    if (direct_ok && d.direct && last) {
      // direct store: register j of group grp is state index base ^ G(grp) ^ goff[j],
      // G and goff XORs of the qubits behind the group and register bits
      uint64_t goff[16];
      goff[0] = 0;
      for (int j = 1; j < 16; ++j)
        goff[j] = goff[j & (j - 1)] ^ (1ull << d.tq[st.Rb[__builtin_ctz(unsigned(j))]]);
      o << "      uint64_t g = base;\n";
      for (int k = 0; k < GB; ++k) o << "      if (grp & " << (1 << k) << ") g |= " << (1ull << d.tq[st.Eb[k]]) << "ull;\n";
      o << "      if (fscale) {\n#pragma unroll\n        for (int j = 0; j < 16; ++j) a[j] = cmul(fT, a[j]);\n      }\n";
      // the group's and the registers' qubits are distinct, so g ^ goff[j] = g + goff[j]:
      // one base pointer and constant offsets
      o << "      V* const gp = reinterpret_cast<V*>(A.state) + g;\n";
      if (pairs) {
        for (int j = 0; j < 16; j += 2)
          o << "      __stcg(reinterpret_cast<float4*>(gp + " << goff[j] << "ll), make_float4(a[" << j << "].x, a[" << j
            << "].y, a[" << j + 1 << "].x, a[" << j + 1 << "].y));\n";
      } else {
        for (int j = 0; j < 16; ++j) o << "      __stcg(gp + " << goff[j] << "ll, a[" << j << "]);\n";
      }
    } else if (pairs) {
      for (int j = 0; j < 16; j += 2)
        o << "      *reinterpret_cast<float4*>(tb + (b ^ " << off[j] << "u)) = make_float4(a[" << j << "].x, a[" << j
          << "].y, a[" << j + 1 << "].x, a[" << j + 1 << "].y);\n";
    } else {
      for (int j = 0; j < 16; ++j) o << "      tb[b ^ " << off[j] << "u] = a[" << j << "];\n";
    }
    const bool bar = st.bar || (!direct_ok && d.direct && last);
    o << "    }\n    " << (bar ? "__syncthreads();" : "__syncwarp();") << "\n";
  }
  o << "  }\n};\n\n";
}

// Backward stage program of one adjoint pass (struct JSB<pass>): groups of 8
// phi + 8 lambda amplitudes (register bit 3 selects phi / lambda), the gates'
// templates and register positions, the derivative accumulations and every
// shared-memory address as constants.
void emit_bwd_stages(std::ostringstream& o, const svp::Plan& B, size_t bp) {
  const svp::DPass& d = B.passes[bp];
  const int GB = B.m - svp::ADJ_REG_BITS;
  o << "struct JSB" << bp << " {\n"
    << "  template <typename T, int M>\n"
    << "  static __device__ __forceinline__ void run(const DPass& sp, const PassShared<T>& sh,\n"
    << "                                             const uint16_t (&sdslot)[MAX_PASS_GATES],\n"
    << "                                             typename CxT<T>::V* tphi, typename CxT<T>::V* tlam,\n"
    << "                                             DotRows<T>& wdot) {\n"
    << "    using V = typename CxT<T>::V;\n"
    << "    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;\n"
    << "    const V* smat = sh.smat;\n";
  for (uint32_t si = 0; si < d.ns; ++si) {
    const svp::DStage& st = B.stages[d.s0 + si];
    uint32_t off[8];
    off[0] = 0;
    for (int j = 1; j < 8; ++j) off[j] = off[j & (j - 1)] ^ st.R[__builtin_ctz(unsigned(j))];
    // the group loop stays rolled and each accumulation is fenced off from the
    // gates around it: unrolled or interleaved, their registers spill at the
    // 128 per thread of two CTAs per SM
    o << "#pragma unroll 1\n    for (int grp = tid; grp < " << (1 << GB) << "; grp += " << svp::PASS_THREADS << ") {\n"
      << "      uint32_t b = 0;\n";
    for (int k = 0; k < GB; ++k) o << "      if (grp & " << (1 << k) << ") b ^= " << st.E[k] << "u;\n";
    o << "      V a[16];\n";
    for (int j = 0; j < 8; ++j)
      o << "      a[" << j << "] = tphi[b ^ " << off[j] << "u]; a[" << j + 8 << "] = tlam[b ^ " << off[j] << "u];\n";
    for (uint32_t g = st.g0; g < uint32_t(st.g0) + st.ng; ++g) {
      const svp::DGate& gt = B.gates[d.g0 + g];
      if (gt.op == svp::OP_DOT || gt.op == svp::OP_CDOT) {
        o << "      asm volatile(\"\" ::: \"memory\");\n      { auto r = ";
        if (gt.op == svp::OP_DOT) o << "g_dot<" << int(gt.p0) << ">(a, smat + " << gt.mat << ");";
        else o << "g_cdot<" << int(gt.p0) << ", " << int(gt.p1) << ">(a, smat + " << gt.mat << ");";
        o << "\n#pragma unroll\n        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);\n"
          << "        if (lane == 0) DotAcc<T>::add(wdot[warp][" << gt.dslot << "], r); }\n"
          << "      asm volatile(\"\" ::: \"memory\");\n";
        continue;
      }
      if (gt.op == svp::OP_D16) {  // a 16 x 16 on all four register bits (three-qubit dense gates: block diagonal)
        o << "      asm volatile(\"\" ::: \"memory\");\n      g_d16(a, smat + " << gt.mat
          << ");\n      asm volatile(\"\" ::: \"memory\");\n";
        continue;
      }
      const char* fn = op_template(gt.op);
      if (!fn) {  // a record kind without a template: the module fails to build (the generic kernel runs)
        o << "#error backward gate record kind " << int(gt.op) << " has no template\n";
        continue;
      }
      if (two_qubit(gt.op)) o << "      " << fn << "<" << int(gt.p0) << ", " << int(gt.p1) << ">(a, smat + " << gt.mat << ");\n";
      else o << "      " << fn << "<" << int(gt.p0) << ">(a, smat + " << gt.mat << ");\n";
    }
    for (int j = 0; j < 8; ++j)
      o << "      tphi[b ^ " << off[j] << "u] = a[" << j << "]; tlam[b ^ " << off[j] << "u] = a[" << j + 8 << "];\n";
    o << "    }\n    __syncthreads();\n";
  }
  o << "  }\n};\n\n";
}

// Driver entry points, resolved through the runtime at first use so that the
// library does not link libcuda (it loads where there is no driver, e.g. for
// host-only checks).
struct Driver {
  CUresult (*moduleLoadData)(CUmodule*, const void*) = nullptr;
  CUresult (*moduleUnload)(CUmodule) = nullptr;
  CUresult (*moduleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, CUstream,
                           void**, void**) = nullptr;
  CUresult (*getErrorString)(CUresult, const char**) = nullptr;
  CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
  bool ok = false;
};

template <typename F>
bool resolve(const char* name, F& fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !p)
    return false;
  fn = reinterpret_cast<F>(p);
  return true;
}

const Driver& driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    d.ok = resolve("cuModuleLoadData", d.moduleLoadData) && resolve("cuModuleUnload", d.moduleUnload) &&
           resolve("cuModuleGetFunction", d.moduleGetFunction) && resolve("cuFuncSetAttribute", d.funcSetAttribute) &&
           resolve("cuLaunchKernel", d.launchKernel) && resolve("cuGetErrorString", d.getErrorString) &&
           resolve("cuOccupancyMaxActiveBlocksPerMultiprocessor", d.occupancy);
  });
  return d;
}

std::string cu_err(CUresult r) {
  const char* s = nullptr;
  if (driver().getErrorString) driver().getErrorString(r, &s);
  return s ? s : ("driver error " + std::to_string(int(r)));
}

}  // namespace

// Source of one module: the stage programs of passes [p0, p1) and one kernel
// that selects among them by pass index (a uniform branch per CTA).
// the pass may run on the tensor cores (dense gate, complex64, 2^12-amplitude tiles)
bool pass_tc(const svp::Plan& P, size_t pi) { return P.dtype == SV_C64 && P.m == 12 && P.passes[pi].dense; }

const char* variant_name(bool tc, bool proj) {
  return tc ? (proj ? "sv_jit_passes_tc_p" : "sv_jit_passes_tc") : (proj ? "sv_jit_passes_p" : "sv_jit_passes");
}

// some pass of [p0, p1) launches variant (tc, proj): the plain-arithmetic
// variant of every pass exists (sv_set_dense_tc(0) runs it), the tensor-core
// one for passes with a dense gate
bool chunk_has_variant(const svp::Plan& P, size_t p0, size_t p1, bool tc, bool proj) {
  for (size_t pi = p0; pi < p1; ++pi)
    if ((P.passes[pi].proj != 0) == proj && (!tc || pass_tc(P, pi))) return true;
  return false;
}

std::string generate_chunk(const svp::Plan& P, size_t p0, size_t p1) {
  std::ostringstream o;
  const bool c64 = P.dtype == SV_C64;
  o << "// specialised passes " << p0 << ".." << p1 << ": n = " << P.n_int << ", tile bits " << P.m << ", "
    << (c64 ? "complex64" : "complex128") << "\n"
    << "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\ntypedef unsigned int uint32_t;\n"
    << "typedef unsigned long long uint64_t;\ntypedef signed char int8_t;\ntypedef short int16_t;\n"
    << "typedef int int32_t;\ntypedef long long int64_t;\n"
    << "#include \"pass_body.cuh\"\n\nnamespace svk {\n\n";
  for (size_t pi = p0; pi < p1; ++pi)
    if (P.passes[pi].ns) emit_stages(o, P, pi);
  o << "struct JitStages {\n"
    << "  static constexpr bool kDirect = true;    // direct passes store from the last stage\n"
    << "  static constexpr bool kFoldProj = true;  // the first stage applies a pending projector\n"
    << "  template <typename T, int M, bool TC>\n"
    << "  static __device__ __forceinline__ void run(const PassArgs& A, const DPass& sp, const uint32_t* sgk,\n"
    << "                                             const typename CxT<T>::V* smat, typename CxT<T>::V* tb,\n"
    << "                                             TcCtx& tc, const uint64_t base, const typename CxT<T>::V fT,\n"
    << "                                             const bool fscale, const ProjFold& pj) {\n"
    << "    switch (A.pass) {\n";
  for (size_t pi = p0; pi < p1; ++pi)
    if (P.passes[pi].ns) o << "      case " << pi << ": JS" << pi << "::run<T, M, TC>(A, sp, sgk, smat, tb, tc, base, fT, fscale, pj); break;\n";
  o << "      default: break;\n    }\n  }\n};\n\n}  // namespace svk\n\n";
  const char* T = c64 ? "float" : "double";
  // kernel variants: tensor cores only where a pass of the chunk holds a dense
  // gate (kernels without tcgen05 instructions sweep faster), the projector
  // pipeline only where a pass may start with a measurement projector pending
  for (int v = 0; v < 4; ++v) {
    const bool vt = v & 1, vp = v & 2;
    if (!chunk_has_variant(P, p0, p1, vt, vp)) continue;
    const int minb = P.jit_min_blocks > 0 ? P.jit_min_blocks : (c64 ? 2 : 1);
    o << "extern \"C\" __global__ void __launch_bounds__(" << svp::PASS_THREADS << ", " << minb << ") "
      << variant_name(vt, vp) << "(const svk::PassArgs A) {\n"
      << "  extern __shared__ __align__(16) unsigned char smem_raw[];\n"
      << "  __shared__ svk::PassShared<" << T << ", " << (vt ? "true" : "false") << "> sh;\n"
      << "  svk::pass_body<" << T << ", " << P.m << ", false, svk::JitStages, " << (vt ? "true" : "false") << ", "
      << (vp ? "true" : "false") << ">(A, A.pass, sh, smem_raw);\n}\n";
  }
  return o.str();
}

size_t chunk_count(const svp::Plan& P) {
  const size_t passes = P.passes.size();
  return passes ? std::min<size_t>(passes, 12) : 1;
}

std::string generate_source(const svp::Plan& P) { return generate_chunk(P, 0, P.passes.size()); }

std::string generate_batch_source(const std::vector<const svp::Plan*>& plans) {
  std::ostringstream o;
  const bool c64 = plans.front()->dtype == SV_C64;
  const int m = plans.front()->m;
  o << "// specialised batch kernel: " << plans.size() << " programs, tile bits " << m << ", "
    << (c64 ? "complex64" : "complex128") << "\n"
    << "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\ntypedef unsigned int uint32_t;\n"
    << "typedef unsigned long long uint64_t;\ntypedef signed char int8_t;\ntypedef short int16_t;\n"
    << "typedef int int32_t;\ntypedef long long int64_t;\n"
    << "#include \"batch_body.cuh\"\n\nnamespace svk {\n\n";
  std::vector<std::string> cases;
  size_t base = 0;
  for (size_t k = 0; k < plans.size(); ++k) {
    const svp::Plan& P = *plans[k];
    const std::string prefix = "JSP" + std::to_string(k) + "_";
    for (size_t pi = 0; pi < P.passes.size(); ++pi)
      if (P.passes[pi].ns) {
        // one function per pass: a module of hundreds of inlined passes takes ptxas minutes
        emit_stages(o, P, pi, prefix.c_str(), false, false);
        cases.push_back("      case " + std::to_string(base + pi) + ": " + prefix + std::to_string(pi) +
                        "::run<T, M, TC>(A, sp, sgk, smat, tb, tc, base, fT, fscale, pj); break;\n");
      }
    base += P.passes.size();
  }
  o << "struct JitBatch {\n"
    << "  static constexpr bool kDirect = false;    // the CTA-mode tile loop stores from shared memory\n"
    << "  static constexpr bool kFoldProj = false;  // the CTA-mode tile loop applies a pending projector\n"
    << "  template <typename T, int M, bool TC>\n"
    << "  static __device__ __forceinline__ void run(const PassArgs& A, const DPass& sp, const uint32_t* sgk,\n"
    << "                                             const typename CxT<T>::V* smat, typename CxT<T>::V* tb,\n"
    << "                                             TcCtx& tc, const uint64_t base, const typename CxT<T>::V fT,\n"
    << "                                             const bool fscale, const ProjFold& pj) {\n"
    << "    switch (A.pass) {\n";
  for (const std::string& c : cases) o << c;
  o << "      default: break;\n    }\n  }\n};\n\n}  // namespace svk\n\n";
  o << "extern \"C\" __global__ void __launch_bounds__(" << svp::PASS_THREADS << ", " << (c64 ? 2 : 1)
    << ") sv_jit_batch(const svk::BatchArgs B) {\n"
    << "  svk::batch_body<" << (c64 ? "float" : "double") << ", " << m << ", svk::JitBatch>(B);\n}\n";
  return o.str();
}

std::string generate_adjoint_source(const svp::Plan& F, const svp::Plan& B) {
  std::ostringstream o;
  const bool c64 = F.dtype == SV_C64;
  o << "// specialised adjoint kernel: n = " << F.n_int << ", tile bits " << F.m << ", "
    << (c64 ? "complex64" : "complex128") << ", " << F.passes.size() << " forward and " << B.passes.size()
    << " backward passes\n"
    << "typedef unsigned char uint8_t;\ntypedef unsigned short uint16_t;\ntypedef unsigned int uint32_t;\n"
    << "typedef unsigned long long uint64_t;\ntypedef signed char int8_t;\ntypedef short int16_t;\n"
    << "typedef int int32_t;\ntypedef long long int64_t;\n"
    << "#include \"adjoint_body.cuh\"\n\nnamespace svk {\n\n";
  for (size_t pi = 0; pi < F.passes.size(); ++pi)
    if (F.passes[pi].ns) emit_stages(o, F, pi, "JSF", false);
  o << "struct JitFwd {\n"
    << "  static constexpr bool kDirect = false;    // the CTA-mode tile loop stores from shared memory\n"
    << "  static constexpr bool kFoldProj = false;  // adjoint programs measure nothing\n"
    << "  template <typename T, int M, bool TC>\n"
    << "  static __device__ __forceinline__ void run(const PassArgs& A, const DPass& sp, const uint32_t* sgk,\n"
    << "                                             const typename CxT<T>::V* smat, typename CxT<T>::V* tb,\n"
    << "                                             TcCtx& tc, const uint64_t base, const typename CxT<T>::V fT,\n"
    << "                                             const bool fscale, const ProjFold& pj) {\n"
    << "    switch (A.pass) {\n";
  for (size_t pi = 0; pi < F.passes.size(); ++pi)
    if (F.passes[pi].ns)
      o << "      case " << pi << ": JSF" << pi << "::run<T, M, TC>(A, sp, sgk, smat, tb, tc, base, fT, fscale, pj); break;\n";
  o << "      default: break;\n    }\n  }\n};\n\n";
  for (size_t bp = 0; bp < B.passes.size(); ++bp)
    if (B.passes[bp].ns) emit_bwd_stages(o, B, bp);
  o << "struct JitBwd {\n"
    << "  template <typename T, int M>\n"
    << "  static __device__ __forceinline__ void run(const DStage*, uint32_t bp, const DPass& sp, const PassShared<T>& sh,\n"
    << "                                             const uint16_t (&sdslot)[MAX_PASS_GATES],\n"
    << "                                             typename CxT<T>::V* tphi, typename CxT<T>::V* tlam,\n"
    << "                                             DotRows<T>& wdot) {\n"
    << "    switch (bp) {\n";
  for (size_t bp = 0; bp < B.passes.size(); ++bp)
    if (B.passes[bp].ns) o << "      case " << bp << ": JSB" << bp << "::run<T, M>(sp, sh, sdslot, tphi, tlam, wdot); break;\n";
  o << "      default: break;\n    }\n  }\n};\n\n}  // namespace svk\n\n";
  const char* T = c64 ? "float" : "double";
  o << "extern \"C\" __global__ void __launch_bounds__(" << svp::PASS_THREADS << ", " << (c64 ? 2 : 1)
    << ") sv_jit_adjoint(const svk::AdjArgs J) {\n"
    << "  svk::adjoint_body<" << T << ", " << F.m << ", svk::JitFwd, svk::JitBwd>(J);\n}\n";
  return o.str();
}

namespace {

// verbose: ptxas resource usage (registers, spills, stack) into *info
sv_status compile_source(const std::string& src, std::vector<char>& cubin, std::string& err,
                         std::string* info = nullptr) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "sv_jit_passes.cu", kJitHeaderCount, kJitHeaderSources,
                         kJitHeaderNames) != NVRTC_SUCCESS) {
    err = "nvrtcCreateProgram failed";
    return SV_ERR_CUDA;
  }
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "--ptxas-options=-v"};
  const nvrtcResult rc = nvrtcCompileProgram(prog, info ? 3 : 2, opts);
  if (rc == NVRTC_SUCCESS && info) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &log[0]);
    *info += log.c_str();
  }
  if (rc != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string log(n, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    err = std::string("NVRTC compile failed: ") + nvrtcGetErrorString(rc) + "\n" + log.substr(0, 4000);
    return SV_ERR_CUDA;
  }
  size_t nbin = 0;
  nvrtcGetCUBINSize(prog, &nbin);
  cubin.assign(nbin, 0);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  return SV_OK;
}

// Compiles the module chunks in parallel (NVRTC programs are independent).
sv_status compile_chunks(const svp::Plan& P, std::vector<std::vector<char>>& cubins, std::vector<size_t>& first,
                         std::string& err, std::vector<std::string>* infos = nullptr) {
  const size_t passes = P.passes.size(), k = chunk_count(P);
  first.assign(k + 1, 0);
  for (size_t c = 0; c <= k; ++c) first[c] = passes * c / k;
  cubins.assign(k, {});
  std::vector<sv_status> st(k, SV_OK);
  std::vector<std::string> errs(k);
  std::vector<std::thread> th;
  for (size_t c = 0; c < k; ++c)
    th.emplace_back([&, c] {
      st[c] = compile_source(generate_chunk(P, first[c], first[c + 1]), cubins[c], errs[c],
                             infos ? &(*infos)[c] : nullptr);
    });
  for (auto& t : th) t.join();
  for (size_t c = 0; c < k; ++c)
    if (st[c] != SV_OK) {
      err = errs[c];
      return st[c];
    }
  return SV_OK;
}

}  // namespace

sv_status compile_cubin(const svp::Plan& P, std::vector<char>& cubin, std::string& err, std::string* info) {
  std::vector<std::vector<char>> cubins;
  std::vector<size_t> first;
  std::vector<std::string> infos(chunk_count(P));
  sv_status st = compile_chunks(P, cubins, first, err, info ? &infos : nullptr);
  if (st == SV_OK && !cubins.empty()) cubin = cubins[0];
  if (info)
    for (const std::string& s : infos) *info += s;
  return st;
}

JitModule::~JitModule() {
  for (void* m : modules)
    if (m && driver().moduleUnload) driver().moduleUnload(static_cast<CUmodule>(m));
}

sv_status compile(const svp::Plan& P, std::shared_ptr<JitModule>& out, std::string& err) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, std::shared_ptr<JitModule>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  // the generated source is a function of these plan fields (whole records
  // hashed, so plans that differ anywhere in them get their own module);
  // hashing them costs far less than generating the text of every chunk
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  };
  const int head[4] = {P.dtype, P.m, P.n_int, P.jit_min_blocks};
  mix(head, sizeof(head));
  mix(P.passes.data(), P.passes.size() * sizeof(svp::DPass));
  mix(P.stages.data(), P.stages.size() * sizeof(svp::DStage));
  mix(P.gates.data(), P.gates.size() * sizeof(svp::DGate));
  const auto key = std::make_pair(dev, size_t(h));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      out = it->second;
      return SV_OK;
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<std::vector<char>> cubins;
  std::vector<size_t> first;
  sv_status st = compile_chunks(P, cubins, first, err);
  if (st != SV_OK) return st;
  const Driver& D = driver();
  if (!D.ok) {
    err = "CUDA driver entry points unavailable";
    return SV_ERR_CUDA;
  }
  std::unique_ptr<JitModule> J(new JitModule());
  const size_t amp = P.dtype == SV_C64 ? 8 : 16;
  const size_t one = (size_t(1) << P.m) * amp;
  J->smem = 2 * one <= size_t(128) * 1024 ? 2 * one : one;
  J->functions.assign(P.passes.size(), nullptr);
  J->functions_tc.assign(P.passes.size(), nullptr);
  for (size_t c = 0; c < cubins.size(); ++c) {
    CUmodule mod;
    CUresult r = D.moduleLoadData(&mod, cubins[c].data());
    if (r != CUDA_SUCCESS) {
      err = "cuModuleLoadData: " + cu_err(r);
      return SV_ERR_CUDA;
    }
    J->modules.push_back(mod);
    CUfunction fv[4] = {nullptr, nullptr, nullptr, nullptr};  // index: tc | proj << 1
    for (int v = 0; v < 4 && r == CUDA_SUCCESS; ++v) {
      if (!chunk_has_variant(P, first[c], first[c + 1], v & 1, v & 2)) continue;
      r = D.moduleGetFunction(&fv[v], mod, variant_name(v & 1, v & 2));
      if (r == CUDA_SUCCESS)
        r = D.funcSetAttribute(fv[v], CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, int(J->smem));
    }
    if (r != CUDA_SUCCESS) {
      err = "loading a specialised module: " + cu_err(r);
      return SV_ERR_CUDA;
    }
    for (size_t pi = first[c]; pi < first[c + 1]; ++pi) {
      const int pj = P.passes[pi].proj ? 2 : 0;
      J->functions[pi] = fv[pj];
      J->functions_tc[pi] = pass_tc(P, pi) ? fv[pj | 1] : nullptr;
    }
  }
  J->compile_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out = std::shared_ptr<JitModule>(std::move(J));
  std::lock_guard<std::mutex> lk(mu);
  if (cache.size() > 64) cache.clear();
  cache[key] = out;
  return SV_OK;
}

sv_status compile_batch_cubin(const std::vector<const svp::Plan*>& plans, std::vector<char>& cubin, std::string& err,
                              std::string* info) {
  if (plans.empty()) {
    err = "no programs";
    return SV_ERR_ARG;
  }
  return compile_source(generate_batch_source(plans), cubin, err, info);
}

sv_status compile_adjoint_cubin(const svp::Plan& F, const svp::Plan& B, std::vector<char>& cubin, std::string& err,
                                std::string* info) {
  return compile_source(generate_adjoint_source(F, B), cubin, err, info);
}

JitAdjoint::~JitAdjoint() {
  if (module && driver().moduleUnload) driver().moduleUnload(static_cast<CUmodule>(module));
}

sv_status compile_adjoint(const svp::Plan& F, const svp::Plan& B, size_t smem, std::shared_ptr<JitAdjoint>& out,
                          std::string& err) {
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, std::shared_ptr<JitAdjoint>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string src = generate_adjoint_source(F, B);
  const auto key = std::make_pair(dev, std::hash<std::string>{}(src + "/" + std::to_string(smem)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      out = it->second;
      return SV_OK;
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<char> cubin;
  sv_status st = compile_source(src, cubin, err);
  if (st != SV_OK) return st;
  const Driver& D = driver();
  if (!D.ok) {
    err = "CUDA driver entry points unavailable";
    return SV_ERR_CUDA;
  }
  std::unique_ptr<JitAdjoint> J(new JitAdjoint());
  CUmodule mod;
  CUresult r = D.moduleLoadData(&mod, cubin.data());
  if (r != CUDA_SUCCESS) {
    err = "cuModuleLoadData: " + cu_err(r);
    return SV_ERR_CUDA;
  }
  J->module = mod;
  CUfunction fn;
  r = D.moduleGetFunction(&fn, mod, "sv_jit_adjoint");
  if (r == CUDA_SUCCESS) r = D.funcSetAttribute(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, int(smem));
  int per_sm = 0;
  if (r == CUDA_SUCCESS) r = D.occupancy(&per_sm, fn, svp::PASS_THREADS, smem);
  if (r != CUDA_SUCCESS) {
    err = "loading the specialised adjoint kernel: " + cu_err(r);
    return SV_ERR_CUDA;
  }
  J->fn = fn;
  J->smem = smem;
  J->per_sm = per_sm > 0 ? per_sm : 1;
  J->compile_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  out = std::shared_ptr<JitAdjoint>(std::move(J));
  std::lock_guard<std::mutex> lk(mu);
  if (cache.size() > 64) cache.clear();
  cache[key] = out;
  return SV_OK;
}

// one module holding one kernel: compiled, loaded, its dynamic shared memory
// set and its occupancy read
sv_status load_single(const std::string& src, const char* name, size_t smem, JitKernel& K, std::string& err) {
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<char> cubin;
  sv_status st = compile_source(src, cubin, err);
  if (st != SV_OK) return st;
  const Driver& D = driver();
  if (!D.ok) {
    err = "CUDA driver entry points unavailable";
    return SV_ERR_CUDA;
  }
  CUmodule mod;
  CUresult r = D.moduleLoadData(&mod, cubin.data());
  if (r != CUDA_SUCCESS) {
    err = "cuModuleLoadData: " + cu_err(r);
    return SV_ERR_CUDA;
  }
  K.module = mod;
  CUfunction fn;
  r = D.moduleGetFunction(&fn, mod, name);
  if (r == CUDA_SUCCESS) r = D.funcSetAttribute(fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, int(smem));
  int per_sm = 0;
  if (r == CUDA_SUCCESS) r = D.occupancy(&per_sm, fn, svp::PASS_THREADS, smem);
  if (r != CUDA_SUCCESS) {
    err = std::string("loading ") + name + ": " + cu_err(r);
    return SV_ERR_CUDA;
  }
  K.fn = fn;
  K.smem = smem;
  K.per_sm = per_sm > 0 ? per_sm : 1;
  K.compile_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return SV_OK;
}

sv_status compile_batch(const std::vector<const svp::Plan*>& plans, size_t smem, std::shared_ptr<JitKernel>& out,
                        std::string& err) {
  if (plans.empty()) {
    err = "no programs";
    return SV_ERR_ARG;
  }
  static std::mutex mu;
  static std::map<std::pair<int, size_t>, std::shared_ptr<JitKernel>> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const std::string src = generate_batch_source(plans);
  const auto key = std::make_pair(dev, std::hash<std::string>{}(src + "/" + std::to_string(smem)));
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      out = it->second;
      return SV_OK;
    }
  }
  std::shared_ptr<JitKernel> K(new JitKernel());
  const sv_status st = load_single(src, "sv_jit_batch", smem, *K, err);
  if (st != SV_OK) return st;
  out = K;
  std::lock_guard<std::mutex> lk(mu);
  if (cache.size() > 16) cache.clear();
  cache[key] = out;
  return SV_OK;
}

sv_status launch_single(const JitKernel& K, void* args, int grid, cudaStream_t s, std::string& err) {
  void* params[] = {args};
  const CUresult r = driver().launchKernel(static_cast<CUfunction>(K.fn), unsigned(grid), 1, 1, svp::PASS_THREADS, 1,
                                           1, unsigned(K.smem), reinterpret_cast<CUstream>(s), params, nullptr);
  if (r != CUDA_SUCCESS) {
    err = "specialised kernel launch: " + cu_err(r);
    return SV_ERR_CUDA;
  }
  return SV_OK;
}

JitKernel::~JitKernel() {
  if (module && driver().moduleUnload) driver().moduleUnload(static_cast<CUmodule>(module));
}

sv_status launch_adjoint(const JitAdjoint& J, const svk::AdjArgs& a, int grid, cudaStream_t s, std::string& err) {
  svk::AdjArgs b = a;
  void* args[] = {&b};
  const CUresult r = driver().launchKernel(static_cast<CUfunction>(J.fn), unsigned(grid), 1, 1, svp::PASS_THREADS, 1,
                                           1, unsigned(J.smem), reinterpret_cast<CUstream>(s), args, nullptr);
  if (r != CUDA_SUCCESS) {
    err = "specialised adjoint launch: " + cu_err(r);
    return SV_ERR_CUDA;
  }
  return SV_OK;
}

sv_status launch(const JitModule& J, int pass, const svk::PassArgs& a, int grid, cudaStream_t s, std::string& err) {
  svk::PassArgs b = a;
  b.pass = pass;
  void* args[] = {&b};
  void* fn = (a.dense_tc && J.functions_tc[size_t(pass)]) ? J.functions_tc[size_t(pass)] : J.functions[size_t(pass)];
  const CUresult r = driver().launchKernel(static_cast<CUfunction>(fn), unsigned(grid), 1, 1,
                                    svp::PASS_THREADS, 1, 1, unsigned(J.smem), reinterpret_cast<CUstream>(s), args,
                                    nullptr);
  if (r != CUDA_SUCCESS) {
    err = "specialised pass launch: " + cu_err(r);
    return SV_ERR_CUDA;
  }
  return SV_OK;
}

}  // namespace svj
