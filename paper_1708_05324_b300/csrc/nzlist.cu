// K3 for N <= 8 as a nonzero list compiled for the context: the coupling
// contraction R_pl = sum_k G[(p,l)][k] V_k, NL_p = sum_l A_l R_pl (Eq. 1
// bracket after the symmetry rewrite) with the nonzero entries of the reduced
// coupling G written into the kernel as constants, one fused multiply-add
// each; the zero entries cost nothing.  The coupling tensors of the paper's
// fibers are mostly zeros (graded-index Hermite-Gaussian modes: 29% of the
// 441 entries at N = 6, 27% of 1296 at N = 8, from the parity of the modes).
//
// At context creation the host writes the kernel's source (the modes, the
// Raman form and the nonzeros of G) and compiles it with NVRTC for the
// device's architecture; the launch replaces k_contract_reg.  The generated
// kernel performs k_contract_reg's operations in its order (the same
// expressions for U and V, the row sums in increasing k, the same l-sum), so
// the two give the same bits; it only leaves out the products with the zeros
// of G.  A context whose kernel cannot be built keeps k_contract_reg (a GPU
// kernel as well); GMMNLSE_NZ=0 keeps it always, GMMNLSE_NZ=require makes a
// failed build an error of gmmnlse_create.  NVRTC is opened at run time
// (dlopen of libnvrtc) and the module calls come from the driver's entry
// points, so the library itself links neither.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gmmnlse.h"
#include "ctx.h"
#include "engine.h"

namespace {

// exact decimal-free text of a coefficient in the working precision
std::string literal(double x, bool fp64) {
  char buf[64];
  if (fp64) std::snprintf(buf, sizeof buf, "%a", x);
  else std::snprintf(buf, sizeof buf, "%af", (double)(float)x);
  return buf;
}

std::string kernel_source(const gmmnlse_ctx* c, const std::vector<double>& Gd) {
  const bool fp64 = c->fp64;
  const int N = c->N, K = c->K, KK = c->KK, mode = c->raman_mode;
  const char* R = fp64 ? "double" : "float";
  const char* R2 = fp64 ? "double2" : "float2";
  std::string s;
  s += "typedef " + std::string(R) + " R;\ntypedef " + R2 + " R2;\n";
  s += "extern \"C\" __global__ void __launch_bounds__(128) k_nz(const R2* __restrict__ A, "
       "const R* __restrict__ Y, R2* __restrict__ NL, const char* __restrict__ ls, int n, int M, int B, "
       "R fR, R fK) {\n";
  // programmatic dependent launch, as pdl_enter(): let the next kernel start
  // launching, then wait for the ones this one depends on
  s += "  asm volatile(\"griddepcontrol.launch_dependents;\");\n";
  s += "  asm volatile(\"griddepcontrol.wait;\" ::: \"memory\");\n";
  s += "  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;\n";
  s += "  if (pt >= (long long)B * (M + 1) * n) return;\n";
  s += "  const int slice = (int)(pt / n), b = slice / (M + 1), j = slice - b * (M + 1);\n";
  s += "  const int t = (int)(pt - (long long)slice * n);\n";
  // the slice is skipped as by slice_skipped(): an idle or finished slot,
  // and z0 after the first iteration
  char buf[256];
  std::snprintf(buf, sizeof buf,
                "  const char* lb = ls + (size_t)b * %zu;\n"
                "  if (*(const int*)(lb + %zu) || *(const int*)(lb + %zu) || (*(const int*)(lb + %zu) > 0 && j == 0)) "
                "return;\n",
                sizeof(gm::LoopState), offsetof(gm::LoopState, idle), offsetof(gm::LoopState, done),
                offsetof(gm::LoopState, iter));
  s += buf;
  s += "  const R2* a = A + (size_t)slice * " + std::to_string(N) + " * n + t;\n";
  for (int l = 0; l < N; ++l) s += "  const R2 a" + std::to_string(l) + " = __ldcg(a + (size_t)" + std::to_string(l) + " * n);\n";
  if (mode != 0) s += "  const R* yp = Y + (size_t)slice * " + std::to_string(K) + " * n + t;\n";
  int k = 0;
  for (int m = 0; m < N; ++m)
    for (int q = m; q < N; ++q, ++k) {
      const std::string am = "a" + std::to_string(m), aq = "a" + std::to_string(q), ks = std::to_string(k);
      const std::string u = (m == q) ? am + ".x * " + am + ".x + " + am + ".y * " + am + ".y"
                                     : "(R)2 * (" + am + ".x * " + aq + ".x + " + am + ".y * " + aq + ".y)";
      s += "  const R u" + ks + " = " + u + ";\n";
      if (mode == 0) s += "  const R v" + ks + " = u" + ks + ";\n";
      else if (mode == 1) s += "  const R v" + ks + " = fK * u" + ks + " + fR * __ldcg(yp + (size_t)" + ks + " * n);\n";
      else {
        s += "  const R v" + ks + " = u" + ks + ";\n";
        s += "  const R v" + std::to_string(K + k) + " = __ldcg(yp + (size_t)" + ks + " * n);\n";
      }
    }
  for (int p = 0; p < N; ++p) s += "  R2 nl" + std::to_string(p) + " = make_" + R2 + "(0, 0);\n";
  int r = 0;
  for (int p = 0; p < N; ++p)
    for (int l = p; l < N; ++l, ++r) {
      s += "  {\n    R acc = (R)0;\n";
      for (int kk = 0; kk < KK; ++kk) {
        const double g = Gd[(size_t)r * KK + kk];
        const double gr = fp64 ? g : (double)(float)g;  // the value k_contract_reg reads
        if (gr == 0.0) continue;
        s += "    acc += " + literal(g, fp64) + " * v" + std::to_string(kk) + ";\n";
      }
      const std::string P = std::to_string(p), L = std::to_string(l);
      s += "    nl" + P + ".x += a" + L + ".x * acc;\n    nl" + P + ".y += a" + L + ".y * acc;\n";
      if (l != p) s += "    nl" + L + ".x += a" + P + ".x * acc;\n    nl" + L + ".y += a" + P + ".y * acc;\n";
      s += "  }\n";
    }
  s += "  R2* out = NL + (size_t)slice * " + std::to_string(N) + " * n + t;\n";
  for (int p = 0; p < N; ++p) s += "  out[(size_t)" + std::to_string(p) + " * n] = nl" + std::to_string(p) + ";\n";
  s += "}\n";
  return s;
}

// NVRTC and driver calls, resolved once (null when unavailable).
struct NzApi {
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleGetFunction) get = nullptr;
  decltype(&cuModuleUnload) unload = nullptr;
  decltype(&cuLaunchKernelEx) launch = nullptr;
  bool ok = false;
};

template <class F>
void driver_fn(const char* name, F& out) {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    out = (F)fn;
}

const NzApi& nz_api() {
  static NzApi api = [] {
    NzApi a;
    void* h = nullptr;
    for (const char* name : {"libnvrtc.so.13", "libnvrtc.so"})
      if (!h) h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (h) {
      a.create = (decltype(a.create))dlsym(h, "nvrtcCreateProgram");
      a.compile = (decltype(a.compile))dlsym(h, "nvrtcCompileProgram");
      a.cubin_size = (decltype(a.cubin_size))dlsym(h, "nvrtcGetCUBINSize");
      a.cubin = (decltype(a.cubin))dlsym(h, "nvrtcGetCUBIN");
      a.destroy = (decltype(a.destroy))dlsym(h, "nvrtcDestroyProgram");
    }
    driver_fn("cuModuleLoadData", a.load);
    driver_fn("cuModuleGetFunction", a.get);
    driver_fn("cuModuleUnload", a.unload);
    driver_fn("cuLaunchKernelEx", a.launch);
    a.ok = a.create && a.compile && a.cubin_size && a.cubin && a.destroy && a.load && a.get && a.unload && a.launch;
    return a;
  }();
  return api;
}

}  // namespace

int gm_nz_build(gmmnlse_ctx* c, const std::vector<double>& Gd) {
  const char* env = std::getenv("GMMNLSE_NZ");
  const bool off = env && env[0] == '0';
  const bool require = env && std::strcmp(env, "require") == 0;
  if (off || c->N > 8 || c->general || c->tc) return GMMNLSE_OK;
  const NzApi& api = nz_api();
  if (!api.ok) {
    if (require) {
      gm_set_last_error_text("NVRTC or the driver's module calls are not available");
      return GMMNLSE_E_CUDA;
    }
    return GMMNLSE_OK;
  }
  const std::string src = kernel_source(c, Gd);
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  // the architecture-specific target of this device (sm_103a on a B300)
  const std::string arch = "--gpu-architecture=sm_" + std::to_string(10 * major + minor) + "a";
  nvrtcProgram prog;
  if (api.create(&prog, src.c_str(), "gmmnlse_nz.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return require ? GMMNLSE_E_CUDA : GMMNLSE_OK;
  const char* opts[] = {arch.c_str(), "--std=c++17", "--fmad=true"};
  const nvrtcResult cr = api.compile(prog, 3, opts);
  std::vector<char> cubin;
  size_t sz = 0;
  if (cr == NVRTC_SUCCESS && api.cubin_size(prog, &sz) == NVRTC_SUCCESS && sz > 0) {
    cubin.resize(sz);
    if (api.cubin(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
  }
  api.destroy(&prog);
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
  if (cubin.empty() || api.load(&mod, cubin.data()) != CUDA_SUCCESS || api.get(&fn, mod, "k_nz") != CUDA_SUCCESS) {
    if (mod) api.unload(mod);
    if (require) {
      gm_set_last_error_text("the nonzero-list contraction kernel could not be built");
      return GMMNLSE_E_CUDA;
    }
    return GMMNLSE_OK;
  }
  c->nz_mod = mod;
  c->nz_fn = fn;
  return GMMNLSE_OK;
}

void gm_nz_free(gmmnlse_ctx* c) {
  if (c->nz_mod) nz_api().unload((CUmodule)c->nz_mod);
  c->nz_mod = nullptr;
  c->nz_fn = nullptr;
}

bool gm_nz_launch(const gmmnlse_ctx* c, const gm::Geo& g, const void* A, const void* V, void* NL,
                  const gm::LoopState* ls, cudaStream_t s) {
  const size_t pts = (size_t)g.B * (g.M + 1) * g.n;
  const unsigned grid = (unsigned)((pts + 127) / 128);
  const void* a = A;
  const void* y = V;
  void* nl = NL;
  const void* l = ls;
  int n = g.n, M = g.M, B = g.B;
  double fR64 = g.fR, fK64 = 1.0 - g.fR;
  float fR32 = (float)g.fR, fK32 = (float)(1.0 - g.fR);
  void* args[] = {(void*)&a, (void*)&y, (void*)&nl, (void*)&l, &n, &M, &B,
                  c->fp64 ? (void*)&fR64 : (void*)&fR32, c->fp64 ? (void*)&fK64 : (void*)&fK32};
  CUlaunchConfig cfg = {};
  cfg.gridDimX = grid;
  cfg.gridDimY = cfg.gridDimZ = 1;
  cfg.blockDimX = 128;
  cfg.blockDimY = cfg.blockDimZ = 1;
  cfg.hStream = (CUstream)s;
  CUlaunchAttribute at;
  at.id = CU_LAUNCH_ATTRIBUTE_PROGRAMMATIC_STREAM_SERIALIZATION;
  at.value.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = &at;
  cfg.numAttrs = pdl_disabled() ? 0 : 1;  // as pdl_launch
  return nz_api().launch(&cfg, (CUfunction)c->nz_fn, args, nullptr) == CUDA_SUCCESS;
}
