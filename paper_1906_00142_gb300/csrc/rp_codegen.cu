// The rational program as generated code (Sec. 3.3 Step 3; Sec. 4.3.1): for
// one kernel, CUDA source whose coefficient table, data-parameter maps and
// architecture constants are written in as constants, around the same
// per-configuration evaluation the table-driven search uses
// (rp_eval_cfg.cuh, embedded here as text at build time); compiled at run
// time with NVRTC for the current device and launched on that kernel's
// queries.  NVRTC is opened with dlopen, so the library loads (and every
// other entry point works) where it is absent; the codegen calls then
// return RP_ERR_UNSUPPORTED.
#include <dlfcn.h>
#include <nvrtc.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "rp_internal.cuh"

namespace rpk {
namespace {

// rp_eval_cfg.cuh as a string literal (written by the build before compiling)
const char kEvalSrc[] =
#include "rp_eval_cfg_src.inc"
    ;

// Exact decimal-free spelling of a float: hexadecimal significand and
// binary exponent ("%a"), or a bit pattern for non-finite values.
void put_float(std::string &s, float v) {
  char b[64];
  if (v != v || v == __builtin_inff() || v == -__builtin_inff()) {
    uint32_t u;
    memcpy(&u, &v, 4);
    snprintf(b, sizeof b, "__int_as_float(0x%08x)", u);
  } else {
    snprintf(b, sizeof b, "%af", (double)v);
  }
  s += b;
}

struct Nvrtc {
  void *h = nullptr;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  bool ok() const { return h && create && compile && log_size && log && cubin_size && cubin && destroy; }
};

const Nvrtc &nvrtc() {
  static Nvrtc n = [] {
    Nvrtc r;
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"};
    for (const char *nm : names)
      if ((r.h = dlopen(nm, RTLD_NOW | RTLD_LOCAL)) != nullptr) break;
    if (!r.h) return r;
    r.create = (decltype(r.create))dlsym(r.h, "nvrtcCreateProgram");
    r.compile = (decltype(r.compile))dlsym(r.h, "nvrtcCompileProgram");
    r.log_size = (decltype(r.log_size))dlsym(r.h, "nvrtcGetProgramLogSize");
    r.log = (decltype(r.log))dlsym(r.h, "nvrtcGetProgramLog");
    r.cubin_size = (decltype(r.cubin_size))dlsym(r.h, "nvrtcGetCUBINSize");
    r.cubin = (decltype(r.cubin))dlsym(r.h, "nvrtcGetCUBIN");
    r.destroy = (decltype(r.destroy))dlsym(r.h, "nvrtcDestroyProgram");
    return r;
  }();
  return n;
}

}  // namespace

struct CodegenHandle {
  cudaLibrary_t lib;
  cudaKernel_t kern;
  int device;
};

std::string codegen_source(const void *program_host, int64_t K, int d, int64_t kid,
                           const rp_hw_fixed &hw) {
  const int D1 = d + 1;
  auto pv = program_sections<ProgramView>(program_host, K);
  const float *tab = pv.table + kid * kNcfg * kNmet * 2 * D1;
  int8_t la[kNcfg], lb[kNcfg];
  int32_t wpb[kNcfg], bact_w[kNcfg], rsm_w[kNcfg], rsm_t[kNcfg];
  search_cfg_table(hw, la, lb, wpb, bact_w, rsm_w, rsm_t);
  std::string s;
  char b[4096];
  snprintf(b, sizeof b,
           "// Rational program of kernel %lld (degree %d) generated by the rational-program\n"
           "// library: the coefficient table of its 66 configurations x 8 metrics and the\n"
           "// architecture constants are written in below.\n",
           (long long)kid, d);
  s += b;
  s += "typedef unsigned int uint32_t;\ntypedef int int32_t;\ntypedef signed char int8_t;\n";
  s += "#define INFINITY __int_as_float(0x7f800000)\n";
  s += "namespace rpk {\nconstexpr int kNcfg = 66, kNmet = 8;\n";
  s += kEvalSrc;
  snprintf(b, sizeof b, "\n__constant__ __align__(16) float g_tab[%d] = {", kNcfg * kNmet * 2 * D1);
  s += b;
  for (int i = 0; i < kNcfg * kNmet * 2 * D1; ++i) {
    if (i % 6 == 0) s += "\n  ";
    put_float(s, tab[i]);
    s += ",";
  }
  s += "};\n__constant__ float g_ab[16] = {";
  for (int m = 0; m < kNmet; ++m) { put_float(s, pv.aN[kid * kNmet + m]); s += ", "; }
  for (int m = 0; m < kNmet; ++m) { put_float(s, pv.bN[kid * kNmet + m]); s += m + 1 < kNmet ? ", " : ""; }
  s += "};\n";
  auto arr = [&](const char *name, const char *type, auto *v) {
    s += "constexpr ";
    s += type;
    s += " ";
    s += name;
    s += "[66] = {";
    for (int i = 0; i < kNcfg; ++i) {
      snprintf(b, sizeof b, "%d%s", (int)v[i], i + 1 < kNcfg ? "," : "");
      s += b;
    }
    s += "};\n";
  };
  arr("kLa", "int8_t", la);
  arr("kLb", "int8_t", lb);
  arr("kWpb", "int32_t", wpb);
  arr("kBactW", "int32_t", bact_w);
  arr("kRsmW", "int32_t", rsm_w);
  arr("kRsmT", "int32_t", rsm_t);
  s += "}  // namespace rpk\n\n";
  snprintf(b, sizeof b,
           "extern \"C\" __global__ void __launch_bounds__(256) rp_generated_search(\n"
           "    const float4 *__restrict__ q, long long Q, int *argmin, float *best, float *second,\n"
           "    int *status) {\n"
           "  using namespace rpk;\n"
           "  // the coefficient table in shared memory: every lane of a warp reads\n"
           "  // the same row (broadcast 16-byte loads)\n"
           "  __shared__ float4 s_tab[sizeof(g_tab) / 16];\n"
           "  for (int j = threadIdx.x; j < (int)(sizeof(g_tab) / 16); j += blockDim.x)\n"
           "    s_tab[j] = reinterpret_cast<const float4 *>(g_tab)[j];\n"
           "  __syncthreads();\n"
           "  const float *tab = reinterpret_cast<const float *>(s_tab);\n"
           "  CfgTab cfg;\n"
           "  for (int c = 0; c < kNcfg; ++c) {\n"
           "    cfg.la[c] = kLa[c]; cfg.lb[c] = kLb[c]; cfg.wpb[c] = kWpb[c];\n"
           "    cfg.bact_w[c] = kBactW[c]; cfg.rsm_w[c] = kRsmW[c]; cfg.rsm_t[c] = kRsmT[c];\n"
           "  }\n"
           "  const HwC hw = {%d, %d, %d, %d, ",
           hw.warp_size, hw.w_max, hw.r_sm, hw.z_sm);
  s += b;
  put_float(s, hw.issue_cycles);
  snprintf(b, sizeof b,
           "};\n"
           "  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < Q;\n"
           "       i += (long long)gridDim.x * blockDim.x) {\n"
           "    const float4 q0 = q[2 * i], q1 = q[2 * i + 1];\n"
           "    const bool kid_ok = __float_as_int(q1.w) == %lld;\n"
           "    float b1 = INFINITY, b2 = INFINITY;\n"
           "    int arg = -1, st = 0;\n"
           "    QState s;\n"
           "    if (!query_state<true>(q0, q1, kid_ok, g_ab, g_ab + kNmet, %d, s)) {\n"
           "      st = %d;\n"
           "    } else {\n"
           "      bool any_pole = false;\n"
           "      for (int c = 0; c < kNcfg; ++c) {\n"
           "        const CfgOut o = eval_cfg<%d, true>(c, s, tab, cfg, hw);\n"
           "        any_pole |= o.pole;\n"
           "        const bool better = o.ex < b1;\n"
           "        const bool second_better = !better && o.ex < b2;\n"
           "        b2 = better ? b1 : (second_better ? o.ex : b2);\n"
           "        arg = better ? c : arg;\n"
           "        b1 = better ? o.ex : b1;\n"
           "      }\n"
           "      st |= any_pole ? %d : 0;\n"
           "      if (arg < 0) st |= %d;\n"
           "    }\n"
           "    argmin[i] = arg; best[i] = b1; second[i] = b2; status[i] = st;\n"
           "  }\n"
           "}\n",
           (long long)kid, (int)pv.grid[kid], RP_Q_BAD, D1, RP_Q_POLE, RP_Q_NO_VALID);
  s += b;
  return s;
}

int codegen_compile(const char *src, void **handle, char *log, size_t log_len) {
  const Nvrtc &n = nvrtc();
  if (log && log_len) log[0] = 0;
  if (!n.ok()) return RP_ERR_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RP_ERR_NO_DEVICE;
  int maj = 0, min = 0;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&min, cudaDevAttrComputeCapabilityMinor, dev);
  nvrtcProgram prog;
  if (n.create(&prog, src, "rp_generated.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) return RP_ERR_CUDA;
  char arch[64];
  snprintf(arch, sizeof arch, "--gpu-architecture=sm_%d%d%s", maj, min, maj >= 9 ? "a" : "");
  const char *opts[] = {arch, "-std=c++17"};
  const nvrtcResult rc = n.compile(prog, 2, opts);
  size_t ls = 0;
  n.log_size(prog, &ls);
  if (log && log_len && ls > 1) {
    std::vector<char> buf(ls);
    n.log(prog, buf.data());
    const size_t c = ls < log_len ? ls : log_len;
    memcpy(log, buf.data(), c);
    log[c - 1] = 0;
  }
  if (rc != NVRTC_SUCCESS) {
    n.destroy(&prog);
    return RP_ERR_INVALID_ARG;
  }
  size_t cs = 0;
  n.cubin_size(prog, &cs);
  std::vector<char> cubin(cs);
  n.cubin(prog, cubin.data());
  n.destroy(&prog);
  CodegenHandle *h = new CodegenHandle{};
  h->device = dev;
  if (cudaLibraryLoadData(&h->lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess ||
      cudaLibraryGetKernel(&h->kern, h->lib, "rp_generated_search") != cudaSuccess) {
    delete h;
    return RP_ERR_CUDA;
  }
  *handle = h;
  return RP_OK;
}

cudaError_t codegen_search(void *handle, const float *queries, int64_t Q, int32_t *argmin,
                           float *best, float *second, int32_t *status, cudaStream_t s) {
  CodegenHandle *h = static_cast<CodegenHandle *>(handle);
  if (Q == 0) return cudaSuccess;
  const int threads = 128;
  int64_t blocks = (Q + threads - 1) / threads;
  if (blocks > (int64_t)num_sms() * 16) blocks = (int64_t)num_sms() * 16;
  const float4 *q4 = reinterpret_cast<const float4 *>(queries);
  long long QQ = (long long)Q;
  void *args[] = {(void *)&q4, (void *)&QQ, (void *)&argmin, (void *)&best, (void *)&second,
                  (void *)&status};
  return cudaLaunchKernel((const void *)h->kern, dim3((unsigned)blocks), dim3(threads), args, 0, s);
}

void codegen_free(void *handle) {
  CodegenHandle *h = static_cast<CodegenHandle *>(handle);
  if (!h) return;
  cudaLibraryUnload(h->lib);
  delete h;
}

}  // namespace rpk
