// Templated host driver of the MPA long steps (Sec. III.D) for one working
// precision R; instantiated once per precision (prop_fp32.cu, prop_fp64.cu).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "../../include/gmmnlse.h"
#include "ctx.h"
#include "engine.h"
#include "persist_api.h"
#include "kernels.cuh"
#include "tc_contract.cuh"
#include "tc_gemm.h"

#include <type_traits>

namespace gm_prop {

using namespace gm;

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      gm_set_last_cuda_error(e_, #call, __FILE__, __LINE__);            \
      return GMMNLSE_E_CUDA;                                            \
    }                                                                   \
  } while (0)

template <typename R> static size_t fft_smem(int n) { return (size_t)fft_smem_elems(n) * sizeof(cplx<R>); }

// FP64 transforms of the N rows of a [N][n] field (input / output of a call).
static int fft64(gmmnlse_ctx* c, double2* scratch, const double2* in, double2* out, int rows, int dir,
                 double scale, cudaStream_t s) {
  const int n = c->n;
  if (n <= 8192) {
    const size_t sm = fft_smem<double>(n);
    if (dir > 0) k_fft64_rows<+1, 16><<<rows, n / 16, sm, s>>>(in, out, n, scale, c->tw64);
    else k_fft64_rows<-1, 16><<<rows, n / 16, sm, s>>>(in, out, n, scale, c->tw64);
  } else {
    const int h = n / 2;
    const size_t sm = fft_smem<double>(h);
    dim3 grid(rows, 2);
    if (dir > 0) {
      k_fft64_halves<+1, 16><<<grid, h / 16, sm, s>>>(in, scratch, n, c->tw64h);
      k_fft64_combine<+1><<<(rows * n + 255) / 256, 256, 0, s>>>(scratch, out, rows, n, scale, c->tw64);
    } else {
      k_fft64_halves<-1, 16><<<grid, h / 16, sm, s>>>(in, scratch, n, c->tw64h);
      k_fft64_combine<-1><<<(rows * n + 255) / 256, 256, 0, s>>>(scratch, out, rows, n, scale, c->tw64);
    }
  }
  CK(cudaGetLastError());
  return GMMNLSE_OK;
}

// Once per device: raise the shared-memory limit of this unit's kernels.
template <typename R>
static int setup_device(int dev) {
  static std::mutex mu;
  static bool done[64];
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return GMMNLSE_E_INVALID;
  if (done[dev]) return GMMNLSE_OK;
  int smax = 0;
  CK(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // the limit covers dynamic shared memory only: leave room for each kernel's
  // static shared variables
  auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  int sm = smax;
  CK(cudaFuncSetAttribute(k_ip_to_time<R, 16, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_ip_to_time<R, 16, 2>, A, sm));
  CK(cudaFuncSetAttribute(k_ip_to_time<R, 16, 4>, A, sm));
  CK(cudaFuncSetAttribute(k_ip_to_time<R, 32, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_integrand<R, 16, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_integrand<R, 16, 2>, A, sm));
  CK(cudaFuncSetAttribute(k_integrand<R, 16, 4>, A, sm));
  CK(cudaFuncSetAttribute(k_integrand<R, 32, 1>, A, sm));

  CK(cudaFuncSetAttribute(k_pairs_raman<R, 16, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman<R, 32, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman<R, 16, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman<R, 32, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman_cl<R, 16, 2, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman_cl<R, 16, 4, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman_cl<R, 16, 2, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_pairs_raman_cl<R, 16, 4, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 0, 0, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 1, 0, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 2, 0, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 0, 0, 1>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 0, 1, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 1, 1, 0>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 0, 1, 2>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 1, 1, 2>, A, sm));
  CK(cudaFuncSetAttribute(k_contract_tile<R, 2, 1, 2>, A, sm));
  if constexpr (std::is_same<R, float>::value) {
    CK(cudaFuncSetAttribute(k_raman_vpack<16, 0>, A, sm));
    CK(cudaFuncSetAttribute(k_raman_vpack<32, 0>, A, sm));
    CK(cudaFuncSetAttribute(k_raman_vpack<16, 1>, A, sm));
    CK(cudaFuncSetAttribute(k_raman_vpack<32, 1>, A, sm));
    if (gm_tc_setup(smax)) {
      gm_set_last_error_text("tensor-core GEMM: shared-memory attribute");
      return GMMNLSE_E_CUDA;
    }
  }
  // the long-step kernels (dynamic shared memory: one transform buffer)
  if (persist_setup<R>(smax)) {
    gm_set_last_error_text("long-step kernel: shared-memory attribute");
    return GMMNLSE_E_CUDA;
  }
  CK(cudaFuncSetAttribute(k_fft64_rows<+1, 16>, A, sm));
  CK(cudaFuncSetAttribute(k_fft64_rows<-1, 16>, A, sm));
  CK(cudaFuncSetAttribute(k_fft64_halves<+1, 16>, A, sm));
  CK(cudaFuncSetAttribute(k_fft64_halves<-1, 16>, A, sm));
  done[dev] = true;
  return GMMNLSE_OK;
}

// Blocks per transform for K1/K4 (output-residue split) so that a launch
// fills the 148 SMs: 1, 2 or 4.
// GMMNLSE_CLUSTER_FFT=1 spreads each transform of a launch that would leave
// SMs idle over a 2- or 4-block cluster (fft_cluster).  Measured slower than
// one block per transform at the benchmark sizes (every kernel has a fixed
// in-GPU cost of a few microseconds and the cluster synchronisations add to
// it), so it is off by default; the tests run both.
static inline bool cluster_fft() {
  const char* v = getenv("GMMNLSE_CLUSTER_FFT");
  return v && v[0] == '1';
}

// An FP64 transform above 8192 points does not fit one block's shared
// memory: it always takes a 4-block cluster (n/4 points per block).
template <typename R>
static inline int split_for(int transforms, int n) {
  if (sizeof(R) == 8 && n > 8192) return 4;
  if (!cluster_fft()) return 1;
  if (transforms <= 74 && n >= 128) return 4;
  if (transforms <= 148 && n >= 64) return 2;
  return 1;
}

// slices of a launch: B slots of M + 1 substeps
static inline int slices(const Geo& g) { return g.B * (g.M + 1); }

template <typename R>
static Geo make_geo(const gmmnlse_ctx* c, int Mj, double dz, int B = 1) {
  Geo g;
  g.B = B;
  g.N = c->N;
  g.n = c->n;
  g.K = c->K;
  g.P = c->P;
  g.KK = c->KK;
  g.M = Mj;
  g.raman_mode = c->raman_mode;
  g.ss = c->prm.self_steepening ? 1 : 0;
  g.fR = c->fR;
  g.gamma0 = c->gamma0;
  g.omega0 = c->omega0;
  g.dt = c->prm.dt;
  g.hdz = 0.5 * dz;
  return g;
}

template <typename R> static const cplx<R>* twid(const gmmnlse_ctx* c);
template <> const cplx<float>* twid<float>(const gmmnlse_ctx* c) { return c->tw32; }
template <> const cplx<double>* twid<double>(const gmmnlse_ctx* c) { return c->tw64; }

static int elementwise_blocks(size_t count) {
  const size_t b = (count + 255) / 256;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 148 * 8));
}

// Elements per thread of a one-block transform of np points in a launch of
// `blocks` transforms: above 8192 points always 32; at 8192 points in FP32,
// 32 (256 threads, two blocks per SM) when the launch has at least two
// blocks per SM, which measured faster for throughput (the 42-mode
// workload) and slower for a launch of fewer blocks than SMs (the 6-mode
// workload: 8 warps per SM), where 16 per thread is kept.
template <typename R> static int fft_ept(int np, int blocks) {
  return (np > 8192 || (sizeof(R) == 4 && np == 8192 && blocks >= 2 * 148)) ? 32 : 16;
}

// bytes of shared memory of a transform of n points over S blocks
template <typename R> static size_t fft_cluster_smem(int n, int S) {
  return S == 1 ? fft_smem<R>(n) : fft_smem<R>(n / S) + (size_t)(n / S) * sizeof(cplx<R>);
}

// K1: phase x inverse FFT; one transform per block or per S-block cluster
template <typename R>
static void launch_k1(gm_job* jb, const Geo& g, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const int n = c->n, N = c->N;
  const int S = split_for<R>(N * slices(g), n), np = n / S, ept = S > 1 ? 16 : fft_ept<R>(np, N * slices(g));
  const dim3 grid(N * S, slices(g));
  const size_t sm = fft_cluster_smem<R>(n, S);
  auto go = [&](auto kern) {
    pdl_launch_cl(kern, grid, dim3(np / ept), sm, s, S, g, (const cplx<R>*)jb->psiR, (const cplx<R>*)jb->dpsi,
                  (const cplx<R>*)jb->E, (cplx<R>*)jb->A, twid<R>(c), (const LoopState*)jb->ls);
  };
  if (ept == 32) go(k_ip_to_time<R, 32, 1>);
  else if (S == 1) go(k_ip_to_time<R, 16, 1>);
  else if (S == 2) go(k_ip_to_time<R, 16, 2>);
  else go(k_ip_to_time<R, 16, 4>);
}

// K2: pair products + Raman convolution, a cluster per transform pair when
// one block per pair would leave SMs idle
template <typename R>
static void launch_k2(gm_job* jb, const Geo& g, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const int n = c->n;
  const int pp = (c->K + 1) / 2;
  const int S = split_for<R>(pp * slices(g), n);
  auto args = [&](auto kern, dim3 grid, int threads, size_t sm, int cl) {
    pdl_launch_cl(kern, grid, dim3(threads), sm, s, cl, g, (const cplx<R>*)jb->A, (R*)jb->V,
                  (const cplx<R>*)c->H, twid<R>(c), (const int2*)c->pairs, (const R*)nullptr, c->K,
                  (const LoopState*)jb->ls);
  };
  auto one = [&](auto kern, int ept) {
    pdl_launch(kern, dim3(pp, slices(g)), dim3(n / ept), fft_smem<R>(n), s, g, (const cplx<R>*)jb->A, (R*)jb->V,
               (const cplx<R>*)c->H, twid<R>(c), (const int2*)c->pairs, (const R*)nullptr, c->K,
               (const LoopState*)jb->ls);
  };
  if (S > 1) {
    const int np = n / S;
    if (S == 2) args(k_pairs_raman_cl<R, 16, 2, 0>, dim3(S * pp, slices(g)), np / 16, fft_cluster_smem<R>(n, S), S);
    else args(k_pairs_raman_cl<R, 16, 4, 0>, dim3(S * pp, slices(g)), np / 16, fft_cluster_smem<R>(n, S), S);
  } else if (fft_ept<R>(n, pp * slices(g)) == 32) {
    one(k_pairs_raman<R, 32, 0>, 32);
  } else {
    one(k_pairs_raman<R, 16, 0>, 16);
  }
}

// K4: forward FFT x integrand prefactor, split as K1
template <typename R>
static void launch_k4(gm_job* jb, const Geo& g, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const int n = c->n, N = c->N;
  // K4 takes 32 per thread at 8192 FP32 points whatever the launch size:
  // its 32 x 16 x 16 schedule measured faster than 16 per thread even for a
  // launch of fewer blocks than SMs (6-mode workload: 7.4 against 8.9 us),
  // unlike K1 and K2
  const int S = split_for<R>(N * slices(g), n), np = n / S;
  const int ept = S > 1 ? 16 : ((sizeof(R) == 4 && np == 8192) ? 32 : fft_ept<R>(np, N * slices(g)));
  const dim3 grid(N * S, slices(g));
  const size_t sm = fft_cluster_smem<R>(n, S);
  auto go = [&](auto kern) {
    pdl_launch_cl(kern, grid, dim3(np / ept), sm, s, S, g, (const cplx<R>*)jb->NL, (const cplx<R>*)jb->E,
                  (const R*)c->fac, (cplx<R>*)jb->I, twid<R>(c), (const LoopState*)jb->ls);
  };
  if (ept == 32) go(k_integrand<R, 32, 1>);
  else if (S == 1) go(k_integrand<R, 16, 1>);
  else if (S == 2) go(k_integrand<R, 16, 2>);
  else go(k_integrand<R, 16, 4>);
}

// The tcgen05 GEMM with the l-sum epilogue: V operand maps mV*, coupling
// operand maps mG*, over the mode count of the context.
static void launch_tc_lsum(gm_job* jb, const Geo& g, cudaStream_t s, const CUtensorMap& mVhi,
                           const CUtensorMap& mVlo, const CUtensorMap& mGhi, const CUtensorMap& mGlo,
                           const TcArgs& a) {
  gmmnlse_ctx* c = jb->ctx;
  TcLaunch L = {&mVhi, &mVlo, &mGhi, &mGlo, a, (const LoopState*)jb->ls, s, slices(g) * c->n / TC_PTS, c->tf32};
  gm_tc_lsum(c->N, L);
}

static TcArgs tc_args(gm_job* jb, const Geo& g) {
  gmmnlse_ctx* c = jb->ctx;
  TcArgs a = {};
  a.f16 = c->f16 ? 1 : 0;
  a.n = c->n;
  a.M = g.M;
  a.A = (const float2*)jb->A;
  a.NL = (float2*)jb->NL;
  a.err = &jb->ls->tc_err;
  a.B = g.B;
  a.wait_ns = c->tc_wait_ns;
  a.stall = c->tc_stall;
  return a;
}

// Pack of V = U / (1 - fR) U + fR Y / [U; Y] from A and Y (K columns).
static void launch_pack_pairs(gm_job* jb, const Geo& g, cudaStream_t s, int mode) {
  gmmnlse_ctx* c = jb->ctx;
  const int n = c->n;
  const int npts_total = (jb->Mcap + 1) * n * jb->slots;
  const int pts = slices(g) * n;
  const dim3 pgrid((pts + PACK_PTS - 1) / PACK_PTS);
  auto pack = [&](auto kern) {
    pdl_launch(kern, pgrid, dim3(PACK_PTS * PACK_WARPS), (size_t)c->N * PACK_PTS * sizeof(float2), s, g,
               (const float2*)jb->A, (const float*)jb->V, (const int2*)c->pairs, c->KKp, npts_total,
               (void*)jb->Vhi, (void*)jb->Vlo, (const LoopState*)jb->ls);
  };
  auto by_mode = [&](auto k0, auto k1, auto k2) {
    if (mode == 0) pack(k0);
    else if (mode == 1) pack(k1);
    else pack(k2);
  };
  if (c->tf32) by_mode(k_pack_hilo<0, 2>, k_pack_hilo<1, 2>, k_pack_hilo<2, 2>);
  else if (c->f16) by_mode(k_pack_hilo<0, 1>, k_pack_hilo<1, 1>, k_pack_hilo<2, 1>);
  else by_mode(k_pack_hilo<0, 0>, k_pack_hilo<1, 0>, k_pack_hilo<2, 0>);
}

// K3 on the tensor cores (mixed precision): form V and pack it to 16-bit
// hi/lo, then the tcgen05 GEMM with the l-sum in its epilogue
template <typename R>
static void launch_tc(gm_job* jb, const Geo& g, cudaStream_t s) {
  if constexpr (std::is_same<R, float>::value) {
    gmmnlse_ctx* c = jb->ctx;
    launch_pack_pairs(jb, g, s, c->raman_mode);
    TcArgs a = tc_args(jb, g);
    a.KKp = c->KKp;
    a.eG = c->eG;
    launch_tc_lsum(jb, g, s, jb->mapHi, jb->mapLo, c->mapGhi, c->mapGlo, a);
  }
}

// ---------------------------------------------------------------------------
// Low-rank coupling G = X W (N > 8, S^R = S^K).  Per point the bracket of
// Eq. 1 becomes R = X V' with V' = (1 - fR) Z + fR h_R * Z and Z = W U, which
// holds because the Raman convolution acts on time and W on the pair index:
//   GEMM 1: Z = W U (r rows);  K2 on the r rows of Z;  GEMM 2: R = X V' and
//   the l-sum.
// ---------------------------------------------------------------------------
template <typename R>
static void launch_lr_z(gm_job* jb, const Geo& g, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const size_t pts = (size_t)slices(g) * c->n;
  if (c->tc) {
    if constexpr (std::is_same<R, float>::value) {
      // 16-bit operands: U is formed inside the GEMM (TcShape::FU); TF32: packed first
      if (c->tf32) launch_pack_pairs(jb, g, s, 0);
      TcArgs a = tc_args(jb, g);
      a.KKp = c->tf32 ? c->KKp : c->KKpU;
      a.eG = c->eW16;
      a.nrb = c->r_rows / c->NB1;
      a.Zout = (float*)jb->Z;
      a.zrows = c->r;
      a.nmodes = c->N;
      // 16-bit: U formed in the kernel from the 4 x 4 blocks of (m, n)
      a.K = c->tf32 ? c->K : c->nublk;
      a.pairs = c->tf32 ? (const int2*)c->pairs : (const int2*)c->ublk;
      TcLaunch L = {&jb->mapHi, &jb->mapLo, &c->mapWhi, &c->mapWlo, a, (const LoopState*)jb->ls, s,
                    (int)(pts / TC_PTS), c->tf32};
      gm_tc_store(c->NB1, L);
    }
    return;
  }
  TileArgs<R> a = {};
  a.A = (const cplx<R>*)jb->A;
  a.Ys = (const R*)jb->V;
  a.Gt = (const R*)c->Wt;
  a.KK = c->K;
  a.KKp = c->KKt;
  a.Pp = c->rP1;
  a.rows = c->r;
  a.cnt = c->r;
  a.pairs = (const int2*)c->pairs;
  a.Zout = (R*)jb->Z;
  const dim3 grid((unsigned)((pts + TileCfg<R>::TP - 1) / TileCfg<R>::TP));
  pdl_launch(k_contract_tile<R, 0, 0, 1>, grid, dim3(256), contract_tile_smem<R>(c->N), s, g, a,
             (const LoopState*)jb->ls);
}

template <typename R>
static void launch_lr_raman(gm_job* jb, const Geo& g, cudaStream_t s, int cnt = 0) {
  gmmnlse_ctx* c = jb->ctx;
  // rows h_R * Z of Z [slices][rows][n] (cnt > 0: the general coupling's
  // pair-product rows) to V
  const int rows = cnt > 0 ? cnt : c->r;
  const int n = c->n, pp = (rows + 1) / 2;
  if constexpr (std::is_same<R, float>::value) {
    if (c->tc && !c->tf32 && cnt == 0) {
      // 16-bit operands: K2 writes GEMM 2's V' operand itself (no Y', no pack)
      const int ept = fft_ept<float>(n, pp * slices(g));
      const int npts_total = (jb->Mcap + 1) * n * jb->slots;
      // clusters of four blocks, one per 8-row group of Z (k_raman_vpack)
      auto vp = [&](auto kern) {
        pdl_launch_cl(kern, dim3(4 * ((c->r + 7) / 8), slices(g)), dim3(n / ept), fft_smem<float>(n), s, 4, g,
                      (const float*)jb->Z, c->r,
                   (const float2*)c->Hv, (const float2*)twid<float>(c), npts_total, (void*)jb->Vhi, (void*)jb->Vlo,
                   c->eW, (const LoopState*)jb->ls);
      };
      if (c->f16) {
        if (ept == 32) vp(k_raman_vpack<32, 1>);
        else vp(k_raman_vpack<16, 1>);
      } else {
        if (ept == 32) vp(k_raman_vpack<32, 0>);
        else vp(k_raman_vpack<16, 0>);
      }
      return;
    }
  }
  auto one = [&](auto kern, int ept) {
    pdl_launch(kern, dim3(pp, slices(g)), dim3(n / ept), fft_smem<R>(n), s, g, (const cplx<R>*)jb->A, (R*)jb->V,
               (const cplx<R>*)c->H, twid<R>(c), (const int2*)c->pairs, (const R*)jb->Z, rows,
               (const LoopState*)jb->ls);
  };
  const int S = split_for<R>(pp * slices(g), n);
  if (S > 1) {
    auto cl = [&](auto kern) {
      pdl_launch_cl(kern, dim3(S * pp, slices(g)), dim3(n / S / 16), fft_cluster_smem<R>(n, S), s, S, g,
                    (const cplx<R>*)jb->A, (R*)jb->V, (const cplx<R>*)c->H, twid<R>(c), (const int2*)c->pairs,
                    (const R*)jb->Z, rows, (const LoopState*)jb->ls);
    };
    if (S == 2) cl(k_pairs_raman_cl<R, 16, 2, 1>);
    else cl(k_pairs_raman_cl<R, 16, 4, 1>);
  } else if (fft_ept<R>(n, pp * slices(g)) == 32) {
    one(k_pairs_raman<R, 32, 1>, 32);
  } else {
    one(k_pairs_raman<R, 16, 1>, 16);
  }
}

template <typename R>
static void launch_lr_r(gm_job* jb, const Geo& g, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const size_t pts = (size_t)slices(g) * c->n;
  const int mode = c->raman_mode ? 1 : 0;
  if (c->tc) {
    if constexpr (std::is_same<R, float>::value) {
      const int npts_total = (jb->Mcap + 1) * c->n * jb->slots;
      // with Raman and 16-bit operands K2 has written V' already (k_raman_vpack)
      const bool packed = mode == 1 && !c->tf32;
      auto pack = [&](auto kern) {
        if (packed) return;
        pdl_launch(kern, dim3((unsigned)((pts + PACK_PTS - 1) / PACK_PTS)), dim3(PACK_PTS * PACK_WARPS), 0, s, g,
                   (const float*)jb->Z,
                   (const float*)jb->V, c->r, c->rKKp, npts_total, (void*)jb->Vhi, (void*)jb->Vlo, c->eW,
                   (const LoopState*)jb->ls);
      };
      if (c->tf32) {
        if (mode) pack(k_pack_rows<1, 2>);
        else pack(k_pack_rows<0, 2>);
      } else if (c->f16) {
        if (mode) pack(k_pack_rows<1, 1>);
        else pack(k_pack_rows<0, 1>);
      } else {
        if (mode) pack(k_pack_rows<1, 0>);
        else pack(k_pack_rows<0, 0>);
      }
      TcArgs a = tc_args(jb, g);
      a.KKp = c->rKKp;
      a.eG = c->eX16;
      a.eVoff = c->eW;
      launch_tc_lsum(jb, g, s, jb->mapHi2, jb->mapLo2, c->mapXhi, c->mapXlo, a);
    }
    return;
  }
  TileArgs<R> a = {};
  a.A = (const cplx<R>*)jb->A;
  a.Ys = (const R*)jb->V;
  a.Zs = (const R*)jb->Z;
  a.Gt = (const R*)c->Xt;
  a.KK = c->r;
  a.KKp = c->rK2;
  a.Pp = c->Pt;
  a.rows = c->P;
  a.cnt = c->r;
  a.rowpl = (const int2*)c->rows_t;
  a.NL = (cplx<R>*)jb->NL;
  const dim3 grid((unsigned)((pts + TileCfg<R>::TP - 1) / TileCfg<R>::TP));
  auto go = [&](auto kern) {
    pdl_launch(kern, grid, dim3(256), contract_tile_smem<R>(c->N), s, g, a, (const LoopState*)jb->ls);
  };
  if (mode) go(k_contract_tile<R, 1, 1, 0>);
  else go(k_contract_tile<R, 0, 1, 0>);
}

// The general coupling (complex S^K, S^R; Eq. 1 without Eq. 2's real S):
// the N^2 real pair-product rows U to Z, their Raman convolution to V, and
// the CUDA-core GEMM R = G [U; h_R * U] with the complex l-sum
// NL_p = sum_l A_l R_pl.
template <typename R>
static void launch_gen(gm_job* jb, const Geo& g, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const int n = c->n;
  pdl_launch(k_gen_pairs<R>, dim3((n + 255) / 256, slices(g)), dim3(256), 0, s, g, (const cplx<R>*)jb->A,
             (R*)jb->Z, (const int2*)c->gpairs, (const LoopState*)jb->ls);
  if (c->raman_mode) launch_lr_raman<R>(jb, g, s, c->gK);
  TileArgs<R> a = {};
  a.A = (const cplx<R>*)jb->A;
  a.Ys = (const R*)jb->V;
  a.Zs = (const R*)jb->Z;
  a.Gt = (const R*)c->Gt;
  a.KK = c->KK;
  a.KKp = c->KKt;
  a.Pp = c->Pt;
  a.rows = c->P;
  a.cnt = c->gK;
  a.NL = (cplx<R>*)jb->NL;
  const size_t pts = (size_t)slices(g) * n;
  const dim3 grid((unsigned)((pts + TileCfg<R>::TP - 1) / TileCfg<R>::TP));
  auto go = [&](auto kern) {
    pdl_launch(kern, grid, dim3(256), contract_tile_smem<R>(c->N), s, g, a, (const LoopState*)jb->ls);
  };
  if (c->raman_mode == 0) go(k_contract_tile<R, 0, 1, 2>);
  else if (c->raman_mode == 1) go(k_contract_tile<R, 1, 1, 2>);
  else go(k_contract_tile<R, 2, 1, 2>);
}

// The Sec. IV terms added to the integrand I (after K4): linear coupling
// (with its longitudinal profile), gain and its saturation.  z0 of the
// substeps: from the loop state's long-step count (use_step) or zoff.
template <typename R>
static void launch_linear_coupling(gm_job* jb, const Geo& g, cudaStream_t s, int use_step, double zoff) {
  const gmmnlse_ctx* c = jb->ctx;
  LinTerms lt = {};
  lt.Q = c->Q;
  lt.gain = c->gain;
  lt.fprof = c->fprof;
  lt.fcount = c->fcount;
  lt.fdz = c->fdz;
  lt.Rs = c->sat != 0.0 ? jb->Rs : nullptr;
  lt.sat = c->sat;
  lt.Mfull = jb->Mprop;
  lt.use_step = use_step;
  lt.zoff = zoff;
  k_linear_coupling<R><<<elementwise_blocks((size_t)slices(g) * c->n), 256, 0, s>>>(
      g, lt, (const cplx<R>*)jb->psiR, (const cplx<R>*)jb->dpsi, (const cplx<R>*)jb->E, (cplx<R>*)jb->I, jb->ls);
}

// The saturation's per-substep rows R_pl(j) from the time-domain field A
// (after K1): the time integrals of the pair products, then S^R times them.
template <typename R>
static void launch_saturation(gm_job* jb, const Geo& g, cudaStream_t s) {
  const gmmnlse_ctx* c = jb->ctx;
  k_sat_gram<R><<<dim3(c->N, slices(g)), 256, 0, s>>>(g, (const cplx<R>*)jb->A, jb->Ubar, jb->ls);
  k_sat_rows<<<dim3((c->P + 127) / 128, slices(g)), 128, 0, s>>>(c->P, c->K, c->GRt, jb->Ubar, jb->Rs, jb->ls);
}

static inline bool extra_terms(const gmmnlse_ctx* c) { return c->Q || c->gain || c->sat != 0.0; }

// K5 with the convergence decision in its last block
template <typename R>
static void launch_k5(gm_job* jb, const Geo& g, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  pdl_launch(k_trapz<R, true>, dim3(trapz_blocks((size_t)jb->ctx->N * jb->ctx->n), g.B), dim3(TRAPZ_T), 0, s, g,
             (const cplx<R>*)jb->psiR, (cplx<R>*)jb->dpsi,
             (const cplx<R>*)jb->I, jb->ls, jb->part, h, use_cond);
}

// One MPA iteration (Sec. III.D): transform to the time domain, pair
// products and Raman convolution, coupling contraction, integrand, and the
// trapezoid with the convergence decision.
template <typename R>
static void launch_iteration(gm_job* jb, const Geo& g, cudaStream_t s, cudaGraphConditionalHandle h, int use_cond) {
  gmmnlse_ctx* c = jb->ctx;
  launch_k1<R>(jb, g, s);
  if (c->sat != 0.0) launch_saturation<R>(jb, g, s);
  if (c->general) {
    launch_gen<R>(jb, g, s);
  } else if (c->lr) {
    launch_lr_z<R>(jb, g, s);
    if (c->raman_mode) launch_lr_raman<R>(jb, g, s);
    launch_lr_r<R>(jb, g, s);
  } else {
    if (c->raman_mode) launch_k2<R>(jb, g, s);
    if (c->tc) launch_tc<R>(jb, g, s);
    else launch_contract<R>(g, c, jb->A, jb->V, jb->NL, jb->ls, s);
  }
  launch_k4<R>(jb, g, s);
  if (extra_terms(c)) launch_linear_coupling<R>(jb, g, s, 1, 0.0);
  launch_k5<R>(jb, g, s, h, use_cond);
}

// K6 with the long-step bookkeeping in its last block; in a graph it also
// sets the outer loop's condition and re-arms the iteration loop.
template <typename R>
static void launch_advance(gm_job* jb, const Geo& g, int which, cudaStream_t s, cudaGraphConditionalHandle hStep,
                           cudaGraphConditionalHandle hIter, int use_cond) {
  gmmnlse_ctx* c = jb->ctx;
  const size_t Nn = (size_t)c->N * c->n;
  pdl_launch(k_advance<R>, dim3(elementwise_blocks(Nn), g.B), dim3(256), 0, s, g, jb->psi0, (cplx<R>*)jb->psiR,
             (const cplx<R>*)jb->dpsi, (const double2*)(jb->EM64 + (size_t)which * Nn), jb->ls, hStep, hIter,
             use_cond, jb->part, 2 * Nn);
}

template <typename R>
static int build_graph(gm_job* jb, const Geo& g, int which, gm_job::G& out) {
  cudaStream_t cs = jb->cap;
  cudaGraph_t root = nullptr;
  CK(cudaGraphCreate(&root, 0));
  cudaGraphConditionalHandle hStep, hIter;
  CK(cudaGraphConditionalHandleCreate(&hStep, root, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = hStep;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t nStep;
  CK(cudaGraphAddNode(&nStep, root, nullptr, nullptr, 0, &cp));
  cudaGraph_t gS = cp.conditional.phGraph_out[0];
  if (jb->persist_grid > 0 && !extra_terms(jb->ctx)) {
    // long-step body: the cooperative long-step kernel (iterations inside)
    CK(cudaStreamBeginCaptureToGraph(cs, gS, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_long_step<R>(jb, g, which, cs, hStep, 1);
    CK(cudaStreamEndCapture(cs, &gS));
  } else {
  // the iteration loop's condition starts at 1 when the graph is launched;
  // the advance kernel re-arms it at the end of every long step
  CK(cudaGraphConditionalHandleCreate(&hIter, gS, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams ci = {};
  ci.type = cudaGraphNodeTypeConditional;
  ci.conditional.handle = hIter;
  ci.conditional.type = cudaGraphCondTypeWhile;
  ci.conditional.size = 1;
  cudaGraphNode_t nIter;
  CK(cudaGraphAddNode(&nIter, gS, nullptr, nullptr, 0, &ci));
  cudaGraph_t gI = ci.conditional.phGraph_out[0];
  // iteration body: K1 .. K5
  CK(cudaStreamBeginCaptureToGraph(cs, gI, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  launch_iteration<R>(jb, g, cs, hIter, 1);
  CK(cudaStreamEndCapture(cs, &gI));
  // after the loop: K6
  CK(cudaStreamBeginCaptureToGraph(cs, gS, &nIter, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  launch_advance<R>(jb, g, which, cs, hStep, hIter, 1);
  CK(cudaStreamEndCapture(cs, &gS));
  }
  cudaGraphExec_t exec = nullptr;
  CK(cudaGraphInstantiate(&exec, root, 0));
  out.graph = root;
  out.exec = exec;
  out.Mj = g.M;
  out.which = which;
  out.dz = 2.0 * g.hdz;
  return GMMNLSE_OK;
}

static bool graphs_disabled() {
  const char* v = getenv("GMMNLSE_NO_GRAPH");
  return v && v[0] == '1';
}

// Run `count` long steps of Mj substeps starting from the current psi0.
template <typename R>
static int run_long_steps(gm_job* jb, int Mj, int which, double dz, int count, cudaStream_t s) {
  if (count <= 0) return GMMNLSE_OK;
  const Geo g = make_geo<R>(jb->ctx, Mj, dz);
  // the step target for this launch
  CK(cudaMemcpyAsync(jb->h_ls, jb->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (jb->h_ls->status != ST_OK) return GMMNLSE_OK;
  const int target = jb->h_ls->step + count;
  CK(cudaMemcpyAsync(&jb->ls->nsteps, &target, sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (!graphs_disabled()) {
    gm_job::G* gr = nullptr;
    for (auto& x : jb->graphs)
      if (x.exec && x.Mj == Mj && x.which == which && x.dz == dz && x.qv == jb->ctx->qv && x.Mfull == jb->Mprop)
        gr = &x;
    if (!gr) {
      gm_job::G& slot = jb->graphs[which];
      if (slot.exec) {
        cudaGraphExecDestroy(slot.exec);
        cudaGraphDestroy(slot.graph);
        slot = gm_job::G();
      }
      if (build_graph<R>(jb, g, which, slot) == GMMNLSE_OK) {
        slot.qv = jb->ctx->qv;
        slot.Mfull = jb->Mprop;
        gr = &slot;
      }
      else {
        cudaGetLastError();
        if (getenv("GMMNLSE_VERBOSE")) fprintf(stderr, "gmmnlse: graph build failed, host loop\n");
      }
    }
    if (gr) {
      CK(cudaGraphLaunch(gr->exec, s));
      return GMMNLSE_OK;
    }
  }
  // host-driven loop over the same kernels
  for (int st = 0; st < count; ++st) {
    if (jb->persist_grid > 0 && !extra_terms(jb->ctx)) {
      launch_long_step<R>(jb, g, which, s, 0, 0);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(jb->h_ls, jb->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (jb->h_ls->status != ST_OK || jb->h_ls->sync_err) break;
      continue;
    }
    for (;;) {
      launch_iteration<R>(jb, g, s, 0, 0);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(jb->h_ls, jb->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (jb->h_ls->done) break;
    }
    launch_advance<R>(jb, g, which, s, 0, 0, 0);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(jb->h_ls, jb->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (jb->h_ls->status != ST_OK) break;
  }
  return GMMNLSE_OK;
}

template <typename R>
static int propagate_impl(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                          double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  long nfull = 0;
  int Mrem = 0;
  int rc = gm_schedule(L, dz, M, &nfull, &Mrem);
  if (rc) return rc;
  if (!(tol >= 0) || !std::isfinite(tol)) return GMMNLSE_E_INVALID;
  const size_t Nn = (size_t)c->N * c->n;
  jb->Mprop = M;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  // input: time-domain FP64 field -> io[0]
  double2* tin = jb->io;
  if (dev_io) {
    CK(cudaMemcpyAsync(tin, A0, Nn * 16, cudaMemcpyDeviceToDevice, s));
  } else {
    std::memcpy(jb->h_io, A0, Nn * 16);
    CK(cudaMemcpyAsync(tin, jb->h_io, Nn * 16, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemsetAsync(jb->flag, 0, sizeof(int), s));
  k_nonfinite<<<elementwise_blocks(Nn), 256, 0, s>>>(tin, Nn, jb->flag);
  int hflag = 0;
  CK(cudaMemcpyAsync(&hflag, jb->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hflag) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return GMMNLSE_E_INVALID;
  }
  // the long-step kernel, where it applies (chosen once per workspace)
  if (jb->persist_grid < 0) jb->persist_grid = long_step_grid<R>(jb);
  // psi0 = F{A0} (FP64)
  rc = fft64(c, jb->io + Nn, tin, jb->psi0, c->N, +1, 1.0, s);
  if (rc) return rc;
  if (!c->fp64) k_round_psi<R><<<elementwise_blocks(Nn), 256, 0, s>>>(jb->psi0, (cplx<R>*)jb->psiR, Nn);
  // phase tables for (dz, M, Mrem)
  if (jb->tab_dz != dz || jb->tab_M != M || jb->tab_Mrem != Mrem) {
    k_phase_tables<R><<<elementwise_blocks((size_t)(M + 1) * Nn), 256, 0, s>>>(
        c->beta, (int)Nn, M, dz, Mrem, (cplx<R>*)jb->E, jb->EM64);
    CK(cudaGetLastError());
    jb->tab_dz = dz;
    jb->tab_M = M;
    jb->tab_Mrem = Mrem;
  }
  // loop state
  LoopState h = {};
  h.hdz = 0.5 * dz;
  h.tol = tol;
  h.floor_eps = c->fp64 ? 1e-14 : (c->prm.precision == GMMNLSE_FP32 ? 1e-6 : 1e-5);
  h.max_iter = c->prm.max_iter > 0 ? c->prm.max_iter : 50;
  h.fixed_iters = c->prm.fixed_iters;
  h.prev_eps = INFINITY;
  h.iters_min = 1 << 30;
  h.status = ST_OK;
  *jb->h_ls = h;
  CK(cudaMemcpyAsync(jb->ls, jb->h_ls, sizeof(LoopState), cudaMemcpyHostToDevice, s));
  k_spec_sums<<<elementwise_blocks(Nn), 256, 0, s>>>(jb->psi0, c->N, c->n, c->prm.dt, c->omega0, jb->ls->spec);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  rc = run_long_steps<R>(jb, M, 0, dz, (int)nfull, s);
  if (rc) return rc;
  if (Mrem > 0) {
    rc = run_long_steps<R>(jb, Mrem, 1, dz, 1, s);
    if (rc) return rc;
  }
  // output sums and Aout = F^-1{psi0}
  k_spec_sums<<<elementwise_blocks(Nn), 256, 0, s>>>(jb->psi0, c->N, c->n, c->prm.dt, c->omega0,
                                                     jb->ls->spec + 2);
  rc = fft64(c, jb->io + Nn, jb->psi0, jb->io, c->N, -1, 1.0 / c->n, s);
  if (rc) return rc;
  if (dev_io) {
    CK(cudaMemcpyAsync(Aout, jb->io, Nn * 16, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemcpyAsync(jb->h_io, jb->io, Nn * 16, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaMemcpyAsync(jb->h_ls, jb->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  if (!dev_io) std::memcpy(Aout, jb->h_io, Nn * 16);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const LoopState& hs = *jb->h_ls;
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
    st->energy_in = hs.spec[0] * c->prm.dt / c->n;
    st->photons_in = hs.spec[1];
    st->energy_out = hs.spec[2] * c->prm.dt / c->n;
    st->photons_out = hs.spec[3];
    st->ms = ms;
    st->coupling_rank = c->lr ? c->r : c->K;
  }
  if (hs.tc_err) {
    gm_set_last_error_text("tensor-core contraction: a wait for its operands timed out");
    return GMMNLSE_E_CUDA;
  }
  if (hs.sync_err) {
    gm_set_last_error_text("long-step kernel: a grid barrier timed out");
    return GMMNLSE_E_CUDA;
  }
  if (hs.status == ST_NOT_CONVERGED) return GMMNLSE_E_NOT_CONVERGED;
  if (hs.status == ST_NONFINITE) return GMMNLSE_E_NONFINITE;
  return GMMNLSE_OK;
}

// ---------------------------------------------------------------------------
// Packed propagations: the slots of one workspace (same context and M, each
// its own field, dz and tolerance) advance together, one long step per
// launch, every kernel of the iteration over all slots at once; a slot
// joins or leaves between launches.  Only whole long steps (L a multiple of
// M dz) and contexts without the Sec. IV terms are packed.
// ---------------------------------------------------------------------------
template <typename R>
static int pack_admit(gm_job* jb, int b, const double* A0, double L, double dz, double tol, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const int M = jb->Mcap;
  long nfull = 0;
  int Mrem = 0;
  int rc = gm_schedule(L, dz, M, &nfull, &Mrem);
  if (rc) return rc;
  if (Mrem != 0 || b < 0 || b >= jb->slots || !(tol >= 0) || !std::isfinite(tol)) return GMMNLSE_E_INVALID;
  const size_t Nn = (size_t)c->N * c->n;
  double2* tin = jb->io;
  std::memcpy(jb->h_io, A0, Nn * 16);
  CK(cudaMemcpyAsync(tin, jb->h_io, Nn * 16, cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(jb->flag, 0, sizeof(int), s));
  k_nonfinite<<<elementwise_blocks(Nn), 256, 0, s>>>(tin, Nn, jb->flag);
  int hflag = 0;
  CK(cudaMemcpyAsync(&hflag, jb->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hflag) return GMMNLSE_E_INVALID;
  double2* p0 = jb->psi0 + (size_t)b * Nn;
  rc = fft64(c, jb->io + Nn, tin, p0, c->N, +1, 1.0, s);
  if (rc) return rc;
  if (!c->fp64)
    k_round_psi<R><<<elementwise_blocks(Nn), 256, 0, s>>>(p0, (cplx<R>*)jb->psiR + (size_t)b * Nn, Nn);
  k_phase_tables<R><<<elementwise_blocks((size_t)(M + 1) * Nn), 256, 0, s>>>(
      c->beta, (int)Nn, M, dz, 0, (cplx<R>*)jb->E + (size_t)b * (M + 1) * Nn, jb->EM64 + (size_t)b * 2 * Nn);
  LoopState h = {};
  h.hdz = 0.5 * dz;
  h.tol = tol;
  h.floor_eps = c->fp64 ? 1e-14 : (c->prm.precision == GMMNLSE_FP32 ? 1e-6 : 1e-5);
  h.max_iter = c->prm.max_iter > 0 ? c->prm.max_iter : 50;
  h.fixed_iters = c->prm.fixed_iters;
  h.prev_eps = INFINITY;
  h.iters_min = 1 << 30;
  h.status = ST_OK;
  h.nsteps = (int)nfull;
  jb->h_ls[b] = h;
  CK(cudaMemcpyAsync(jb->ls + b, &jb->h_ls[b], sizeof(LoopState), cudaMemcpyHostToDevice, s));
  k_spec_sums<<<elementwise_blocks(Nn), 256, 0, s>>>(p0, c->N, c->n, c->prm.dt, c->omega0, (jb->ls + b)->spec);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return GMMNLSE_OK;
}

// The graph of one packed long step: the iteration loop over every slot (a
// while-node whose condition the trapezoid kernel's last deciding slot sets:
// continue while any slot iterates), then the advance of every slot.
template <typename R>
static int build_pack_graph(gm_job* jb, const Geo& g, gm_job::G& out) {
  cudaStream_t cs = jb->cap;
  cudaGraph_t root = nullptr;
  CK(cudaGraphCreate(&root, 0));
  cudaGraphConditionalHandle hIter;
  CK(cudaGraphConditionalHandleCreate(&hIter, root, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams ci = {};
  ci.type = cudaGraphNodeTypeConditional;
  ci.conditional.handle = hIter;
  ci.conditional.type = cudaGraphCondTypeWhile;
  ci.conditional.size = 1;
  cudaGraphNode_t nIter;
  CK(cudaGraphAddNode(&nIter, root, nullptr, nullptr, 0, &ci));
  cudaGraph_t gI = ci.conditional.phGraph_out[0];
  CK(cudaStreamBeginCaptureToGraph(cs, gI, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  launch_iteration<R>(jb, g, cs, hIter, 1);
  CK(cudaStreamEndCapture(cs, &gI));
  CK(cudaStreamBeginCaptureToGraph(cs, root, &nIter, nullptr, 1, cudaStreamCaptureModeThreadLocal));
  launch_advance<R>(jb, g, 0, cs, 0, 0, 0);
  CK(cudaStreamEndCapture(cs, &root));
  cudaGraphExec_t exec = nullptr;
  CK(cudaGraphInstantiate(&exec, root, 0));
  out.graph = root;
  out.exec = exec;
  out.Mj = g.M;
  out.which = 0;
  out.qv = jb->ctx->qv;
  return GMMNLSE_OK;
}

template <typename R>
static int pack_step(gm_job* jb, cudaStream_t s, int* finished) {
  gmmnlse_ctx* c = jb->ctx;
  const int B = jb->slots;
  // the launch covers the slots up to the last occupied one (the host mirror
  // of the loop states knows which: admission and retirement write it)
  int Bact = 0;
  for (int k = 0; k < B; ++k)
    if (!jb->h_ls[k].idle) Bact = k + 1;
  for (int k = 0; k < B; ++k) finished[k] = 0;
  if (Bact == 0) return GMMNLSE_OK;
  const Geo g = make_geo<R>(c, jb->Mcap, 0.0, Bact);
  if ((int)jb->pack_graphs.size() < B + 1) jb->pack_graphs.resize(B + 1);
  gm_job::G& slot = jb->pack_graphs[Bact];
  bool ran = false;
  if (!graphs_disabled()) {
    if (!slot.exec || slot.qv != c->qv) {
      if (slot.exec) {
        cudaGraphExecDestroy(slot.exec);
        cudaGraphDestroy(slot.graph);
        slot = gm_job::G();
      }
      if (build_pack_graph<R>(jb, g, slot) != GMMNLSE_OK) {
        cudaGetLastError();
        slot = gm_job::G();
      }
    }
    if (slot.exec) {
      CK(cudaGraphLaunch(slot.exec, s));
      ran = true;
    }
  }
  if (!ran) {
    // host-driven loop over the same kernels
    for (int it = 0; it < 4096; ++it) {
      launch_iteration<R>(jb, g, s, 0, 0);
      CK(cudaGetLastError());
      CK(cudaMemcpyAsync(jb->h_ls, jb->ls, Bact * sizeof(LoopState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      bool any = false;
      for (int k = 0; k < Bact; ++k) any = any || (!jb->h_ls[k].idle && !jb->h_ls[k].done);
      if (!any) break;
    }
    launch_advance<R>(jb, g, 0, s, 0, 0, 0);
    CK(cudaGetLastError());
  }
  CK(cudaMemcpyAsync(jb->h_ls, jb->ls, B * sizeof(LoopState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < B; ++k) {
    const LoopState& h = jb->h_ls[k];
    finished[k] = !h.idle && (h.status != ST_OK || h.step >= h.nsteps || h.tc_err) ? 1 : 0;
  }
  if (jb->h_ls[0].tc_err) {
    gm_set_last_error_text("tensor-core contraction: a wait for its operands timed out");
    return GMMNLSE_E_CUDA;
  }
  return GMMNLSE_OK;
}

template <typename R>
static int pack_retire(gm_job* jb, int b, double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  const int M = jb->Mcap;
  const size_t Nn = (size_t)c->N * c->n;
  double2* p0 = jb->psi0 + (size_t)b * Nn;
  k_spec_sums<<<elementwise_blocks(Nn), 256, 0, s>>>(p0, c->N, c->n, c->prm.dt, c->omega0, (jb->ls + b)->spec + 2);
  int rc = fft64(c, jb->io + Nn, p0, jb->io, c->N, -1, 1.0 / c->n, s);
  if (rc) return rc;
  CK(cudaMemcpyAsync(jb->h_io, jb->io, Nn * 16, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&jb->h_ls[b], jb->ls + b, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::memcpy(Aout, jb->h_io, Nn * 16);
  const LoopState hs = jb->h_ls[b];
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->long_steps = hs.step;
    st->z = (double)hs.step * M * (2.0 * hs.hdz);
    st->iters_total = hs.iters_total;
    st->iters_min = hs.step > 0 ? hs.iters_min : 0;
    st->iters_max = hs.iters_max;
    std::memcpy(st->iter_hist, hs.hist, sizeof(st->iter_hist));
    st->eps_max = hs.eps_max;
    st->eps_last = hs.eps;
    st->energy_in = hs.spec[0] * c->prm.dt / c->n;
    st->photons_in = hs.spec[1];
    st->energy_out = hs.spec[2] * c->prm.dt / c->n;
    st->photons_out = hs.spec[3];
    st->coupling_rank = c->lr ? c->r : c->K;
  }
  // the slot is empty again
  LoopState idle = {};
  idle.idle = 1;
  jb->h_ls[b] = idle;
  CK(cudaMemcpyAsync(jb->ls + b, &jb->h_ls[b], sizeof(LoopState), cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));
  if (hs.tc_err) {
    gm_set_last_error_text("tensor-core contraction: a wait for its operands timed out");
    return GMMNLSE_E_CUDA;
  }
  if (hs.status == ST_NOT_CONVERGED) return GMMNLSE_E_NOT_CONVERGED;
  if (hs.status == ST_NONFINITE) return GMMNLSE_E_NONFINITE;
  return GMMNLSE_OK;
}

// ---------------------------------------------------------------------------
// RK4IP on the same kernels (the split-step comparator of Sec. III.D): each
// step of h evaluates N four times, one after the other, as K1 -> K2/K3 ->
// K4 on a single slice of phase 1 (loop state at iteration 0, geometry of
// M = 0), with k_rk4_stage between them.  The field between steps is FP64.
// Host-driven launches, no graph; the phase tables are taken for (h/2, 1)
// and marked stale for the next MPA call.
// ---------------------------------------------------------------------------
template <typename R>
static int rk4ip_impl(gm_job* jb, const double* A0, bool dev_io, double L, double h, double* Aout,
                      gmmnlse_stats* st, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  long steps = 0;
  int rem = 0;
  int rc = gm_schedule(L, h, 1, &steps, &rem);
  if (rc) return rc;
  const size_t Nn = (size_t)c->N * c->n;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, s));
  double2* tin = jb->io;
  if (dev_io) {
    CK(cudaMemcpyAsync(tin, A0, Nn * 16, cudaMemcpyDeviceToDevice, s));
  } else {
    std::memcpy(jb->h_io, A0, Nn * 16);
    CK(cudaMemcpyAsync(tin, jb->h_io, Nn * 16, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemsetAsync(jb->flag, 0, sizeof(int), s));
  k_nonfinite<<<elementwise_blocks(Nn), 256, 0, s>>>(tin, Nn, jb->flag);
  int hflag = 0;
  CK(cudaMemcpyAsync(&hflag, jb->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (hflag) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return GMMNLSE_E_INVALID;
  }
  // RK4 state: field A, AI = Eh A, the stage sum (FP64 [N][Nt] each)
  double2* buf = nullptr;
  if (cudaMalloc(&buf, 3 * Nn * sizeof(double2)) != cudaSuccess) {
    cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return GMMNLSE_E_NOMEM;
  }
  double2 *Ast = buf, *AI = buf + Nn, *acc = buf + 2 * Nn;
  rc = fft64(c, jb->io + Nn, tin, jb->psi0, c->N, +1, 1.0, s);
  if (rc) {
    cudaFree(buf);
    return rc;
  }
  CK(cudaMemcpyAsync(Ast, jb->psi0, Nn * 16, cudaMemcpyDeviceToDevice, s));
  // E_1 and EM64[0] = exp(i beta h/2); the MPA's tables are rebuilt next time
  k_phase_tables<R><<<elementwise_blocks(2 * Nn), 256, 0, s>>>(c->beta, (int)Nn, 1, 0.5 * h, 0, (cplx<R>*)jb->E,
                                                               jb->EM64);
  CK(cudaGetLastError());
  jb->tab_dz = -1.0;
  jb->tab_M = -1;
  LoopState hl = {};
  hl.status = ST_OK;
  *jb->h_ls = hl;
  CK(cudaMemcpyAsync(jb->ls, jb->h_ls, sizeof(LoopState), cudaMemcpyHostToDevice, s));
  k_spec_sums<<<elementwise_blocks(Nn), 256, 0, s>>>(jb->psi0, c->N, c->n, c->prm.dt, c->omega0, jb->ls->spec);
  const Geo g = make_geo<R>(c, 0, 0.5 * h);
  const int eb = elementwise_blocks(Nn);
  cplx<R>* X = (cplx<R>*)jb->psiR;
  const cplx<R>* I0 = (const cplx<R>*)jb->I;
  k_rk4_stage<R><<<eb, 256, 0, s>>>(0, Nn, h, Ast, AI, acc, I0, jb->EM64, X);
  for (long k = 0; k < steps; ++k) {
    for (int q = 1; q <= 4; ++q) {
      launch_k1<R>(jb, g, s);
      if (c->sat != 0.0) launch_saturation<R>(jb, g, s);
      if (c->general) {
        launch_gen<R>(jb, g, s);
      } else if (c->lr) {
        launch_lr_z<R>(jb, g, s);
        if (c->raman_mode) launch_lr_raman<R>(jb, g, s);
        launch_lr_r<R>(jb, g, s);
      } else {
        if (c->raman_mode) launch_k2<R>(jb, g, s);
        if (c->tc) launch_tc<R>(jb, g, s);
        else launch_contract<R>(g, c, jb->A, jb->V, jb->NL, jb->ls, s);
      }
      launch_k4<R>(jb, g, s);
      // the stage's position: z, z + h/2, z + h/2, z + h
      if (extra_terms(c)) launch_linear_coupling<R>(jb, g, s, 0, h * (k + (q == 1 ? 0.0 : (q == 4 ? 1.0 : 0.5))));
      k_rk4_stage<R><<<eb, 256, 0, s>>>(q, Nn, h, Ast, AI, acc, I0, jb->EM64, X);
    }
    if (cudaGetLastError() != cudaSuccess) {
      cudaStreamSynchronize(s);
      cudaFree(buf);
      return GMMNLSE_E_CUDA;
    }
  }
  CK(cudaMemcpyAsync(jb->psi0, Ast, Nn * 16, cudaMemcpyDeviceToDevice, s));
  cudaStreamSynchronize(s);
  cudaFree(buf);
  k_spec_sums<<<elementwise_blocks(Nn), 256, 0, s>>>(jb->psi0, c->N, c->n, c->prm.dt, c->omega0,
                                                     jb->ls->spec + 2);
  CK(cudaMemsetAsync(jb->flag, 0, sizeof(int), s));
  k_nonfinite<<<elementwise_blocks(Nn), 256, 0, s>>>(jb->psi0, Nn, jb->flag);
  rc = fft64(c, jb->io + Nn, jb->psi0, jb->io, c->N, -1, 1.0 / c->n, s);
  if (rc) return rc;
  if (dev_io) {
    CK(cudaMemcpyAsync(Aout, jb->io, Nn * 16, cudaMemcpyDeviceToDevice, s));
  } else {
    CK(cudaMemcpyAsync(jb->h_io, jb->io, Nn * 16, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaMemcpyAsync(jb->h_ls, jb->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&hflag, jb->flag, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaEventRecord(e1, s));
  CK(cudaStreamSynchronize(s));
  if (!dev_io) std::memcpy(Aout, jb->h_io, Nn * 16);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const LoopState& hs = *jb->h_ls;
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->long_steps = (int)steps;
    st->z = (double)steps * h;
    st->iters_total = (int)(4 * steps);  // evaluations of N
    st->iters_min = steps > 0 ? 4 : 0;
    st->iters_max = steps > 0 ? 4 : 0;
    st->energy_in = hs.spec[0] * c->prm.dt / c->n;
    st->photons_in = hs.spec[1];
    st->energy_out = hs.spec[2] * c->prm.dt / c->n;
    st->photons_out = hs.spec[3];
    st->ms = ms;
    st->coupling_rank = c->lr ? c->r : c->K;
  }
  if (hs.tc_err) {
    gm_set_last_error_text("tensor-core contraction: a wait for its operands timed out");
    return GMMNLSE_E_CUDA;
  }
  if (hflag) return GMMNLSE_E_NONFINITE;
  return GMMNLSE_OK;
}

// ---------------------------------------------------------------------------
// Per-kernel timing of one MPA iteration (used for the roofline report)
// ---------------------------------------------------------------------------
template <typename R>
static int profile_impl(gmmnlse_ctx* c, gm_job* jb, int M, int reps, double* ms, double* bytes) {
  cudaStream_t s = c->stream;
  const double dz = jb->tab_dz > 0 ? jb->tab_dz : 1e-5;
  const Geo g = make_geo<R>(c, M, dz);
  const double rs = sizeof(R), cs = 2 * rs;
  const double Nn = (double)c->N * c->n;
  // algorithmic bytes per launch of an iteration (substeps j = 1..M)
  bytes[0] = M * Nn * 4 * cs;                     // psiR, dpsi, E -> A
  bytes[1] = c->raman_mode ? M * (Nn * cs + (double)c->K * c->n * rs) : 0.0;     // A -> Y
  bytes[2] = M * (double)c->n * (2 * c->N * cs + (c->raman_mode ? c->K * rs : 0.0));  // A, Y -> NL
  if (c->general) {
    // pair rows A -> Z, Raman on them (Z -> V); contraction A, Z, V -> NL
    bytes[1] = c->raman_mode ? M * 2.0 * c->gK * c->n * rs : 0.0;
    bytes[2] = M * (double)c->n * (3 * c->N * cs + (double)c->gK * rs * (c->raman_mode ? 3 : 2));
  }
  if (c->lr) {
    // Raman on the rows of Z (Z -> Y'); contraction: A -> Z (GEMM 1), A, Z, Y' -> NL (GEMM 2)
    bytes[1] = c->raman_mode ? M * 2.0 * c->r * c->n * rs : 0.0;
    bytes[2] = M * (double)c->n * (3 * c->N * cs + (double)c->r * rs * (c->raman_mode ? 3 : 2));
  }
  bytes[3] = M * Nn * 3 * cs + c->n * rs;         // NL, E -> I; prefactor table
  bytes[4] = Nn * ((M + 1) * cs + 2 * M * cs + cs); // I, dpsi old/new, psiR
  bytes[5] = Nn * (16 + cs + 16 + 16 + (c->fp64 ? 0 : cs));
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  const int one = 1;
  const size_t Nsz = (size_t)c->N * c->n;
  for (int k = 0; k < 6; ++k) {
    ms[k] = 0.0;
    if (k == 1 && !c->raman_mode) continue;
    // iteration state: iter = 1 (substeps 1..M, the shape of every iteration after the first)
    CK(cudaMemcpyAsync(&jb->ls->iter, &one, sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    for (int r = -1; r < reps; ++r) {
      if (r == 0) CK(cudaEventRecord(a, s));  // reps launches back to back after one warm-up
      switch (k) {
        case 0: launch_k1<R>(jb, g, s); break;
        case 1:
          if (c->general) launch_lr_raman<R>(jb, g, s, c->gK);
          else if (c->lr) launch_lr_raman<R>(jb, g, s);
          else launch_k2<R>(jb, g, s);
          break;
        case 2:
          if (c->general) {
            launch_gen<R>(jb, g, s);
          } else if (c->lr) {
            launch_lr_z<R>(jb, g, s);
            launch_lr_r<R>(jb, g, s);
          } else if (c->tc) {
            launch_tc<R>(jb, g, s);
          } else {
            launch_contract<R>(g, c, jb->A, jb->V, jb->NL, jb->ls, s);
          }
          break;
        case 3: launch_k4<R>(jb, g, s); break;
        case 4: launch_k5<R>(jb, g, s, 0, 0); break;
        default:
          k_advance<R><<<elementwise_blocks(Nsz), 256, 0, s>>>(g, jb->psi0, (cplx<R>*)jb->psiR,
                                                               (const cplx<R>*)jb->dpsi, jb->EM64, jb->ls, 0, 0, 0,
                                                               jb->part, 2 * Nsz);
          break;
      }
      CK(cudaGetLastError());
    }
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    ms[k] = t / reps;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return GMMNLSE_OK;
}


}  // namespace gm_prop
