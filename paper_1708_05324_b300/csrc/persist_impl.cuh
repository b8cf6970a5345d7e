// The opt-in cooperative long-step kernel's host side (persist.cuh), for one
// working precision R; included by persist_fp32.cu and persist_fp64.cu.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "ctx.h"
#include "persist.cuh"
#include "persist_api.h"

namespace gm_persist {

using namespace gm;

template <typename R> static size_t fft_smem(int n) { return (size_t)fft_smem_elems(n) * sizeof(cplx<R>); }
template <typename R> static const cplx<R>* twid(const gmmnlse_ctx* c);
template <> const cplx<float>* twid<float>(const gmmnlse_ctx* c) { return c->tw32; }
template <> const cplx<double>* twid<double>(const gmmnlse_ctx* c) { return c->tw64; }

// ---------------------------------------------------------------------------
// The long step as one cooperative kernel (persist.cuh): N <= 8 on the CUDA
// cores with one-block transforms of 16 elements per thread (2048 <= n <=
// 8192), opt-in with GMMNLSE_PERSIST=1.  On the 6-mode workload it measured
// 89 us per iteration against 62 us for the kernel-per-step chain (the
// combined kernel spills ~1 KB of registers in its transform phases, and
// every phase waits for its slowest block), so the chain is the default.
// ---------------------------------------------------------------------------
static bool persist_disabled() {
  const char* v = getenv("GMMNLSE_PERSIST");
  return !(v && v[0] == '1');
}

// Calls f with the long-step kernel of this context's N and raman_mode.
template <typename R, class F>
static void with_long_step(const gmmnlse_ctx* c, F&& f) {
  auto modes = [&](auto nc) {
    constexpr int NN = decltype(nc)::value;
    if (c->raman_mode == 0) f(k_long_step<R, NN, 0>);
    else if (c->raman_mode == 1) f(k_long_step<R, NN, 1>);
    else f(k_long_step<R, NN, 2>);
  };
  switch (c->N) {
    case 1: modes(std::integral_constant<int, 1>()); break;
    case 2: modes(std::integral_constant<int, 2>()); break;
    case 3: modes(std::integral_constant<int, 3>()); break;
    case 4: modes(std::integral_constant<int, 4>()); break;
    case 5: modes(std::integral_constant<int, 5>()); break;
    case 6: modes(std::integral_constant<int, 6>()); break;
    case 7: modes(std::integral_constant<int, 7>()); break;
    case 8: modes(std::integral_constant<int, 8>()); break;
    default: break;
  }
}

// Blocks of the long-step kernel for this job (every block resident), or 0
// where it does not apply.
template <typename R>
static int long_step_grid_impl(gm_job* jb) {
  const gmmnlse_ctx* c = jb->ctx;
  if (persist_disabled() || c->N > 8 || c->tc || c->lr || c->general || c->Q || c->gain || c->sat != 0.0 || c->n < 2048 || c->n > 8192) return 0;
  const int threads = c->n / 16;
  const size_t smem = fft_smem<R>(c->n);
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->prm.device) != cudaSuccess) return 0;
  int rc = -1;
  with_long_step<R>(c, [&](auto kern) {
    rc = (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
  });
  if (rc != (int)cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return std::min(sms * per_sm, TRAPZ_MAX_BLOCKS);
}

// Zero the barrier counter, then the cooperative long-step kernel.
template <typename R>
static void launch_long_step_impl(gm_job* jb, const Geo& g, int which, cudaStream_t s, cudaGraphConditionalHandle hStep,
                                  int use_cond) {
  gmmnlse_ctx* c = jb->ctx;
  const size_t Nn = (size_t)c->N * c->n;
  StepArgs a;
  a.psiR = jb->psiR;
  a.dpsi = jb->dpsi;
  a.E = jb->E;
  a.A = jb->A;
  a.Y = jb->V;
  a.NL = jb->NL;
  a.I = jb->I;
  a.H = c->H;
  a.fac = c->fac;
  a.tw = twid<R>(c);
  a.pairs = c->pairs;
  a.G = c->G;
  a.psi0 = jb->psi0;
  a.EM = jb->EM64 + (size_t)which * Nn;
  a.part = jb->part;
  a.bar = jb->bar;
  cudaMemsetAsync(jb->bar, 0, sizeof(unsigned), s);
  with_long_step<R>(c, [&](auto kern) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(jb->persist_grid);
    cfg.blockDim = dim3(c->n / 16);
    cfg.dynamicSmemBytes = fft_smem<R>(c->n);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, g, a, jb->ls, hStep, use_cond);
  });
}


template <typename R>
static int persist_setup_impl(int smax) {
  gmmnlse_ctx probe;
  for (int N = 1; N <= 8; ++N)
    for (int mode = 0; mode < 3; ++mode) {
      probe.N = N;
      probe.raman_mode = mode;
      int rc = 0;
      with_long_step<R>(&probe, [&](auto kern) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess ||
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smax - (int)fa.sharedSizeBytes) !=
                cudaSuccess)
          rc = -1;
      });
      if (rc) return rc;
    }
  return 0;
}

}  // namespace gm_persist

#define GM_PERSIST_INSTANTIATE(R)                                                                        \
  template <> int persist_setup<R>(int smax) { return gm_persist::persist_setup_impl<R>(smax); }          \
  template <> int long_step_grid<R>(gm_job* jb) { return gm_persist::long_step_grid_impl<R>(jb); }        \
  template <>                                                                                             \
  void launch_long_step<R>(gm_job* jb, const gm::Geo& g, int which, cudaStream_t s,                       \
                           cudaGraphConditionalHandle hStep, int use_cond) {                              \
    gm_persist::launch_long_step_impl<R>(jb, g, which, s, hStep, use_cond);                               \
  }
