// One long step of the MPA (Sec. III.D) as one cooperative kernel, for the
// register contraction (N <= 8) and one-block transforms of 16 elements per
// thread.  Every block loops over the iterations; inside one iteration the
// steps K1 .. K5 run as phases separated by grid barriers, each phase's
// tasks (a transform, a pair of Raman rows, a point, an element) spread over
// the blocks; the decision is taken by block 0 after the last phase, then
// every block reads it; after the loop the long-step advance (K6) and the
// bookkeeping.  This replaces some 22 kernel launches per long step, whose
// launch, ramp and tail dominate at small sizes, by one.
//
// The launch is cooperative, so every block is resident and the barriers
// cannot wait on a block that never runs.  A barrier counts arrivals in a
// device counter (zeroed before the launch) and every wait on it is bounded:
// on a timeout the block records the failure in the loop state and goes on.
// Data written by other blocks during the kernel is read through L2
// (__ldcg in the task functions), never from a stale L1 line.
#pragma once

#include "kernels.cuh"

namespace gm {

struct StepArgs {
  const void* psiR;    // [N][n] R
  void* dpsi;          // [M][N][n] R complex
  const void* E;       // [M+1][N][n]
  void* A;             // [M+1][N][n]
  void* Y;             // [M+1][K][n] R
  void* NL;            // [M+1][N][n]
  void* I;             // [M+1][N][n]
  const void* H;       // [n]
  const void* fac;     // [n] R
  const void* tw;      // twiddles + pass tables of n
  const int2* pairs;   // [K]
  const void* G;       // [K][KK] R
  double2* psi0;       // [N][n]
  const double2* EM;   // [N][n] exp(i beta M dz)
  double2* part;       // per-block sums
  unsigned* bar;       // barrier counter, zero at launch
};

constexpr unsigned kBarrierSpins = 1u << 22;

// Barrier k of the launch over all its blocks (bounded wait).
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned& k, LoopState* ls) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = (++k) * gridDim.x;
    __threadfence();
    atomicAdd(count, 1u);
    unsigned v = 0;
    for (unsigned spins = 0;; ++spins) {
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
      if (v >= target) break;
      if (spins >= kBarrierSpins) {
        atomicExch(&ls->sync_err, 1u);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

template <typename R, int N, int MODE>
__global__ void __launch_bounds__(512) k_long_step(Geo g, StepArgs a, LoopState* ls,
                                                   cudaGraphConditionalHandle hStep, int use_cond) {
  constexpr int EPT = 16;
  constexpr int K = N * (N + 1) / 2;
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smraw);
  __shared__ double red[64];
  const cplx<R>* psiR = (const cplx<R>*)a.psiR;
  cplx<R>* dpsi = (cplx<R>*)a.dpsi;
  const cplx<R>* E = (const cplx<R>*)a.E;
  cplx<R>* A = (cplx<R>*)a.A;
  R* Y = (R*)a.Y;
  cplx<R>* NL = (cplx<R>*)a.NL;
  cplx<R>* I = (cplx<R>*)a.I;
  const cplx<R>* tw = (const cplx<R>*)a.tw;
  const int n = g.n, M = g.M, T = blockDim.x, tid = threadIdx.x;
  const size_t Nn = (size_t)N * n, npts = (size_t)(M + 1) * n;
  const int pp = (K + 1) / 2;
  unsigned k = 0;

  for (int guard = 0; guard <= 4096; ++guard) {
    const int iter = __ldcg(&ls->iter);
    // K1: A_j = F^-1{(psi0 + dpsi_j) E_j}
    for (int task = blockIdx.x; task < N * (M + 1); task += gridDim.x) {
      const int j = task / N, p = task - j * N;
      if (iter > 0 && j == 0) continue;
      __syncthreads();
      ip_to_time_task<R, EPT, 1>(g, psiR, dpsi, E, A, tw, iter, p, j, sm);
    }
    grid_barrier(a.bar, k, ls);
    // K2: Y = h_R * U, two pair rows per task
    if (MODE != 0) {
      for (int task = blockIdx.x; task < pp * (M + 1); task += gridDim.x) {
        const int j = task / pp, kp = task - j * pp;
        if (iter > 0 && j == 0) continue;
        pairs_raman_task<R, EPT, 0>(g, A, Y, (const cplx<R>*)a.H, tw, a.pairs, (const R*)nullptr, K, kp, j, sm);
      }
      grid_barrier(a.bar, k, ls);
    }
    // K3: NL from A and Y, G staged in the (now free) transform buffer
    {
      R* Gs = reinterpret_cast<R*>(smraw);
      __syncthreads();
      stage_g<R, N, MODE>((const R*)a.G, Gs);
      __syncthreads();
      for (size_t pt = (size_t)blockIdx.x * T + tid; pt < npts; pt += (size_t)gridDim.x * T) {
        if (iter > 0 && pt < (size_t)n) continue;
        contract_reg_point<R, N, MODE>(g, A, Y, Gs, NL, pt);
      }
    }
    grid_barrier(a.bar, k, ls);
    // K4: I_j = i gamma0 s(w) F{NL} exp(-i beta j dz)
    for (int task = blockIdx.x; task < N * (M + 1); task += gridDim.x) {
      const int j = task / N, p = task - j * N;
      if (iter > 0 && j == 0) continue;
      __syncthreads();
      integrand_task<R, EPT, 1>(g, NL, E, (const R*)a.fac, I, tw, p, j, sm);
    }
    grid_barrier(a.bar, k, ls);
    // K5: trapezoid and the two sums, per block
    {
      double diff = 0.0, nrm = 0.0;
      const R hdz = (R)g.hdz;
      for (size_t e = (size_t)blockIdx.x * T + tid; e < Nn; e += (size_t)gridDim.x * T)
        trapz_element<R>(g, psiR, dpsi, I, iter, e, hdz, diff, nrm);
      block_sum2(diff, nrm, red);
      if (tid == 0) a.part[blockIdx.x] = make_double2(diff, nrm);
    }
    grid_barrier(a.bar, k, ls);
    // decision (block 0), seen by every block after the barrier
    if (blockIdx.x == 0) {
      double diff = 0.0, nrm = 0.0;
      for (int b = tid; b < (int)gridDim.x; b += T) {
        const double2 v = __ldcg(&a.part[b]);
        diff += v.x;
        nrm += v.y;
      }
      block_sum2(diff, nrm, red);
      if (tid == 0) decide(ls, diff, nrm, 0, 0);
    }
    grid_barrier(a.bar, k, ls);
    if (__ldcg(&ls->done) || __ldcg(&ls->sync_err)) break;
  }

  // K6: A(z0 + M dz) = (psi0 + dpsi_M) exp(i beta M dz) in FP64
  if (__ldcg(&ls->status) == ST_OK) {
    const cplx<R>* d = dpsi + (size_t)(M - 1) * Nn;
    for (size_t e = (size_t)blockIdx.x * T + tid; e < Nn; e += (size_t)gridDim.x * T) {
      const double2 p0 = __ldcg(a.psi0 + e);
      const cplx<R> dd = __ldcg(d + e);
      const double x = p0.x + (double)dd.x, y = p0.y + (double)dd.y;
      const double2 w = a.EM[e];
      const double2 v = make_double2(x * w.x - y * w.y, x * w.y + y * w.x);
      a.psi0[e] = v;
      if ((const void*)a.psiR != (const void*)a.psi0) ((cplx<R>*)a.psiR)[e] = mk<R>((R)v.x, (R)v.y);
    }
  }
  grid_barrier(a.bar, k, ls);
  if (blockIdx.x == 0 && tid == 0) step_end(ls, hStep, 0, use_cond, false);
}

}  // namespace gm
