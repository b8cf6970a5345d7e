// gmmnlse_propagate_noalloc: a propagation that allocates no memory.
//
// gmmnlse_propagate keeps its iteration workspace (the substep fields, pair
// products, integrands, phase tables and loop state) in device memory that it
// obtains with cudaMalloc on first use.  Some callers cannot let a library do
// that: latency-critical loops that cannot afford the implicit device-wide
// synchronisation of cudaMalloc/cudaFree, and host applications whose device
// memory is all handed out by their own pool allocator (a framework's caching
// allocator that must account for every byte, or a service with a fixed
// memory budget per GPU).  This entry point runs the same transforms and
// trapezoid kernels with the workspace placed in one fixed array in device
// global memory, declared below; the array is part of the library image, so
// every GPU that loads the library holds it until the process exits.  The
// caller still provides the input and output fields (device memory) and a
// context made beforehand with gmmnlse_create.  The call is synchronous: it
// reads the iteration state back after every iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/gmmnlse.h"
#include "ctx.h"
#include "engine.h"
#include "kernels.cuh"

using namespace gm;

namespace {
constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
}  // namespace

// The workspace.  In host code this name is only a stand-in for the device
// array: its device address comes from cudaGetSymbolAddress (per device).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

static std::mutex g_setup_mu;
static bool g_attrs_set[kMaxDevices];  // kernel attributes set on this device

#define CKN(call)                                             \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) {                                  \
      gm_set_last_cuda_error(e_, #call, __FILE__, __LINE__);  \
      return GMMNLSE_E_CUDA;                                  \
    }                                                         \
  } while (0)

template <typename R> static size_t fft_bytes(int n) { return (size_t)fft_smem_elems(n) * sizeof(cplx<R>); }

template <typename R, int EPT> static int set_attrs(int maxsm) {
  CKN(cudaFuncSetAttribute(k_ip_to_time<R, EPT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  CKN(cudaFuncSetAttribute(k_pairs_raman<R, EPT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  CKN(cudaFuncSetAttribute(k_integrand<R, EPT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
  return GMMNLSE_OK;
}

// With the device current: the device address of the scratch array (looked
// up on every call, so that it is right for the module loaded now), and,
// once per device, the shared-memory attributes of the kernels of this file.
static int setup_device(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (dev < 0 || dev >= kMaxDevices) return GMMNLSE_E_INVALID;
  void* p = nullptr;
  CKN(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  if (!g_attrs_set[dev]) {
    int maxsm = 0;
    CKN(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    int rc = set_attrs<float, 16>(maxsm);
    if (!rc) rc = set_attrs<float, 32>(maxsm);
    if (!rc) rc = set_attrs<double, 16>(maxsm);
    if (rc) return rc;
    for (auto kern : {k_contract_tile<float, 0, 0, 0>, k_contract_tile<float, 1, 0, 0>, k_contract_tile<float, 2, 0, 0>})
      CKN(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    for (auto kern : {k_contract_tile<double, 0, 0, 0>, k_contract_tile<double, 1, 0, 0>,
                      k_contract_tile<double, 2, 0, 0>})
      CKN(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CKN(cudaFuncSetAttribute(k_fft64_rows<+1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CKN(cudaFuncSetAttribute(k_fft64_rows<-1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CKN(cudaFuncSetAttribute(k_fft64_halves<+1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    CKN(cudaFuncSetAttribute(k_fft64_halves<-1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    g_attrs_set[dev] = true;
  }
  *out = static_cast<unsigned char*>(p);
  return GMMNLSE_OK;
}

// True if p is device (or managed) memory the device `dev` can address.
static bool device_pointer(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Carves the workspace out of the scratch array, 256-byte aligned pieces.
struct Carve {
  size_t off = 0;
  unsigned char* base = nullptr;
  template <typename T> T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += (count * sizeof(T) + 255) & ~(size_t)255;
    return p;
  }
};

struct Work {
  double2* psi0;
  void* psiR;
  void *dpsi, *A, *NL, *I, *E, *V;
  double2 *EM64, *io;
  int* flag;
  LoopState* ls;
  double2* part;  // per-block sums of K5
};

template <typename R> static size_t layout(const gmmnlse_ctx* c, int M, unsigned char* base, Work* w) {
  const size_t Nn = (size_t)c->N * c->n;
  Carve cv;
  cv.base = base;
  w->psi0 = cv.take<double2>(Nn);
  w->psiR = c->fp64 ? (void*)w->psi0 : (void*)cv.take<cplx<R>>(Nn);
  w->dpsi = cv.take<cplx<R>>((size_t)M * Nn);
  w->A = cv.take<cplx<R>>((size_t)(M + 1) * Nn);
  w->NL = cv.take<cplx<R>>((size_t)(M + 1) * Nn);
  w->I = cv.take<cplx<R>>((size_t)(M + 1) * Nn);
  w->E = cv.take<cplx<R>>((size_t)(M + 1) * Nn);
  w->V = c->raman_mode ? cv.take<R>((size_t)(M + 1) * c->K * c->n) : nullptr;
  w->EM64 = cv.take<double2>(2 * Nn);
  w->io = cv.take<double2>(2 * Nn);
  w->flag = cv.take<int>(1);
  w->ls = cv.take<LoopState>(1);
  w->part = cv.take<double2>(TRAPZ_MAX_BLOCKS);
  return cv.off;
}

static int blocks_for(size_t count) {
  return (int)std::max<size_t>(1, std::min<size_t>((count + 255) / 256, 148 * 8));
}

static void fft64_noalloc(const gmmnlse_ctx* c, double2* scratch, const double2* in, double2* out, int dir,
                          double scale, cudaStream_t s) {
  const int n = c->n, rows = c->N;
  if (n <= 8192) {
    const size_t sm = fft_bytes<double>(n);
    if (dir > 0) k_fft64_rows<+1, 16><<<rows, n / 16, sm, s>>>(in, out, n, scale, c->tw64);
    else k_fft64_rows<-1, 16><<<rows, n / 16, sm, s>>>(in, out, n, scale, c->tw64);
  } else {
    const int h = n / 2;
    const size_t sm = fft_bytes<double>(h);
    const dim3 grid(rows, 2);
    const unsigned cb = (unsigned)(((size_t)rows * n + 255) / 256);
    if (dir > 0) {
      k_fft64_halves<+1, 16><<<grid, h / 16, sm, s>>>(in, scratch, n, c->tw64h);
      k_fft64_combine<+1><<<cb, 256, 0, s>>>(scratch, out, rows, n, scale, c->tw64);
    } else {
      k_fft64_halves<-1, 16><<<grid, h / 16, sm, s>>>(in, scratch, n, c->tw64h);
      k_fft64_combine<-1><<<cb, 256, 0, s>>>(scratch, out, rows, n, scale, c->tw64);
    }
  }
}

template <typename R> static const cplx<R>* twiddles(const gmmnlse_ctx* c);
template <> const cplx<float>* twiddles<float>(const gmmnlse_ctx* c) { return c->tw32; }
template <> const cplx<double>* twiddles<double>(const gmmnlse_ctx* c) { return c->tw64; }

template <typename R, int EPT>
static int run(gmmnlse_ctx* c, unsigned char* base, const double* A0, double L, double dz, int M, double tol,
               double* Aout, gmmnlse_stats* st) {
  long nfull = 0;
  int Mrem = 0;
  int rc = gm_schedule(L, dz, M, &nfull, &Mrem);
  if (rc) return rc;
  if (!(tol >= 0) || !std::isfinite(tol)) return GMMNLSE_E_INVALID;
  Work w;
  const size_t need = layout<R>(c, M, nullptr, &w);
  if (need > kScratchBytes) {
    gm_set_last_error_text("gmmnlse_propagate_noalloc: workspace exceeds the 32 MiB static scratch "
                           "(reduce N, Nt or M, or use gmmnlse_propagate)");
    return GMMNLSE_E_NOMEM;
  }
  layout<R>(c, M, base, &w);
  cudaStream_t s = c->stream;
  const size_t Nn = (size_t)c->N * c->n;
  const int n = c->n, N = c->N, T = n / EPT;
  const size_t sm = fft_bytes<R>(n);
  const cplx<R>* tw = twiddles<R>(c);

  CKN(cudaMemcpyAsync(w.io, A0, Nn * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  CKN(cudaMemsetAsync(w.flag, 0, sizeof(int), s));
  k_nonfinite<<<blocks_for(Nn), 256, 0, s>>>(w.io, Nn, w.flag);
  int hflag = 0;
  CKN(cudaMemcpyAsync(&hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CKN(cudaStreamSynchronize(s));
  if (hflag) return GMMNLSE_E_INVALID;
  fft64_noalloc(c, w.io + Nn, w.io, w.psi0, +1, 1.0, s);
  if (!c->fp64) k_round_psi<R><<<blocks_for(Nn), 256, 0, s>>>(w.psi0, (cplx<R>*)w.psiR, Nn);
  k_phase_tables<R><<<blocks_for((size_t)(M + 1) * Nn), 256, 0, s>>>(c->beta, (int)Nn, M, dz, Mrem,
                                                                       (cplx<R>*)w.E, w.EM64);
  // every field of the loop state starts from these values (the scratch
  // keeps whatever the previous call left there)
  LoopState h = {};
  h.hdz = 0.5 * dz;
  h.tol = tol;
  h.floor_eps = c->fp64 ? 1e-14 : (c->prm.precision == GMMNLSE_FP32 ? 1e-6 : 1e-5);
  h.max_iter = c->prm.max_iter > 0 ? c->prm.max_iter : 50;
  h.fixed_iters = c->prm.fixed_iters;
  h.prev_eps = INFINITY;
  h.iters_min = 1 << 30;
  h.status = ST_OK;
  CKN(cudaMemcpyAsync(w.ls, &h, sizeof(LoopState), cudaMemcpyHostToDevice, s));
  k_spec_sums<<<blocks_for(Nn), 256, 0, s>>>(w.psi0, N, n, c->prm.dt, c->omega0, w.ls->spec);
  CKN(cudaGetLastError());
  CKN(cudaStreamSynchronize(s));

  LoopState hs = h;
  const long steps = nfull + (Mrem > 0 ? 1 : 0);
  for (long step = 0; step < steps; ++step) {
    const int Mj = step < nfull ? M : Mrem;
    const int which = step < nfull ? 0 : 1;
    Geo g;
    g.N = N; g.n = n; g.K = c->K; g.P = c->P; g.KK = c->KK; g.M = Mj;
    g.raman_mode = c->raman_mode;
    g.ss = c->prm.self_steepening ? 1 : 0;
    g.fR = c->fR; g.gamma0 = c->gamma0; g.omega0 = c->omega0; g.dt = c->prm.dt; g.hdz = 0.5 * dz;
    g.B = 1;
    const dim3 gridNM(N, Mj + 1);
    for (;;) {
      k_ip_to_time<R, EPT, 1><<<gridNM, T, sm, s>>>(g, (const cplx<R>*)w.psiR, (const cplx<R>*)w.dpsi,
                                                  (const cplx<R>*)w.E, (cplx<R>*)w.A, tw, w.ls);
      if (c->raman_mode)
        k_pairs_raman<R, EPT, 0><<<dim3((c->K + 1) / 2, Mj + 1), T, sm, s>>>(
            g, (const cplx<R>*)w.A, (R*)w.V, (const cplx<R>*)c->H, tw, c->pairs, (const R*)nullptr, c->K, w.ls);
      launch_contract<R>(g, c, w.A, w.V, w.NL, w.ls, s);
      k_integrand<R, EPT, 1><<<gridNM, T, sm, s>>>(g, (const cplx<R>*)w.NL, (const cplx<R>*)w.E, (const R*)c->fac,
                                                (cplx<R>*)w.I, tw, w.ls);
      k_trapz<R, false><<<trapz_blocks(Nn), TRAPZ_T, 0, s>>>(g, (const cplx<R>*)w.psiR, (cplx<R>*)w.dpsi,
                                                             (const cplx<R>*)w.I, w.ls, w.part, 0, 0);
      k_decide<<<1, 32, 0, s>>>(w.ls, 0, 0);
      CKN(cudaGetLastError());
      CKN(cudaMemcpyAsync(&hs, w.ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
      CKN(cudaStreamSynchronize(s));
      if (hs.done) break;
    }
    k_advance<R><<<blocks_for(Nn), 256, 0, s>>>(g, w.psi0, (cplx<R>*)w.psiR, (const cplx<R>*)w.dpsi,
                                               w.EM64 + (size_t)which * Nn, w.ls, 0, 0, 0, w.part, 0);
    CKN(cudaGetLastError());
    CKN(cudaMemcpyAsync(&hs, w.ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
    CKN(cudaStreamSynchronize(s));
    if (hs.status != ST_OK) break;
  }
  k_spec_sums<<<blocks_for(Nn), 256, 0, s>>>(w.psi0, N, n, c->prm.dt, c->omega0, w.ls->spec + 2);
  fft64_noalloc(c, w.io + Nn, w.psi0, w.io, -1, 1.0 / n, s);
  CKN(cudaMemcpyAsync(Aout, w.io, Nn * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  CKN(cudaMemcpyAsync(&hs, w.ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
  CKN(cudaStreamSynchronize(s));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->long_steps = hs.step;
    const long done = (hs.step <= nfull) ? (long)hs.step * M : nfull * M + Mrem;
    st->z = (double)done * dz;
    st->iters_total = hs.iters_total;
    st->iters_min = hs.step > 0 ? hs.iters_min : 0;
    st->iters_max = hs.iters_max;
    std::memcpy(st->iter_hist, hs.hist, sizeof(st->iter_hist));
    st->eps_max = hs.eps_max;
    st->eps_last = hs.eps;
    st->energy_in = hs.spec[0] * c->prm.dt / n;
    st->photons_in = hs.spec[1];
    st->energy_out = hs.spec[2] * c->prm.dt / n;
    st->photons_out = hs.spec[3];
    st->ms = 0.0;
    st->coupling_rank = c->K;  // this entry point runs the dense contraction
  }
  if (hs.status == ST_NOT_CONVERGED) return GMMNLSE_E_NOT_CONVERGED;
  if (hs.status == ST_NONFINITE) return GMMNLSE_E_NONFINITE;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_propagate_noalloc(gmmnlse_ctx* c, const double* A0, double L, double dz, int M, double tol,
                                         double* Aout, gmmnlse_stats* st) {
  if (!c || !A0 || !Aout) return GMMNLSE_E_INVALID;
  if (c->fp64 && c->n > 8192) return GMMNLSE_E_UNSUPPORTED;  // needs the cluster transforms
  if (c->Q || c->gain || c->sat != 0.0) return GMMNLSE_E_UNSUPPORTED;  // Sec. IV terms: not on this path
  if (c->general) return GMMNLSE_E_UNSUPPORTED;  // complex coupling: not on this path
  long nf;
  int mr;
  int rc = gm_schedule(L, dz, M, &nf, &mr);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  CKN(cudaSetDevice(c->prm.device));
  auto gate = gm_gate_device(c->prm.device);
  if (!device_pointer(A0, c->prm.device) || !device_pointer(Aout, c->prm.device)) {
    gm_set_last_error_text("gmmnlse_propagate_noalloc: A0 and Aout must be device memory of the context's device");
    return GMMNLSE_E_INVALID;
  }
  unsigned char* base = nullptr;
  rc = setup_device(c->prm.device, &base);
  if (rc) return rc;
  if (c->fp64) return run<double, 16>(c, base, A0, L, dz, M, tol, Aout, st);
  return c->ept == 16 ? run<float, 16>(c, base, A0, L, dz, M, tol, Aout, st)
                      : run<float, 32>(c, base, A0, L, dz, M, tol, Aout, st);
}
