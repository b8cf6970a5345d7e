// Device kernels of one MPA long step (Sec. III.D), templated on the working
// real type R (float or double) and on the FFT elements per thread EPT.
//
// Data (row-major, all resident on the device for the whole propagation):
//   psi0 [N][n]      double2  running spectrum A~(z0, w): FP64 between long steps
//   psiR [N][n]      cplx<R>  psi0 rounded to the working precision (= psi0 in FP64)
//   dpsi [M][N][n]   cplx<R>  psi_j - psi0, j = 1..M (the iterate)
//   E    [M+1][N][n] cplx<R>  exp(i beta_p(w) j dz), phase reduced in FP64
//   A    [M+1][N][n] cplx<R>  A_j(t) = F^-1{psi_j E_j}
//   V    [M+1][KK][n] R       pair products after the Raman convolution
//   NL   [M+1][N][n] cplx<R>  bracket of Eq. 1 at z_j
//   I    [M+1][N][n] cplx<R>  integrand of Eq. MPA_eq at z_j
// Substep j = 0 (z0 itself) is evaluated only in the first iteration of a
// long step: I_0 does not change while psi_j, j >= 1, is iterated.
#pragma once

#include <cooperative_groups.h>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

namespace gm {

constexpr double C_LIGHT = 299792458.0;

enum : int { ST_OK = 0, ST_NOT_CONVERGED = -4, ST_NONFINITE = -5 };

// Iteration control shared by the kernels of a propagation (device memory).
struct LoopState {
  double diff, nrm;        // sum |psi^(n+1) - psi^(n)|^2, sum |psi^(n+1)|^2 (this iteration)
  double eps, prev_eps;    // eps of this and the previous iteration
  double eps_max;          // largest final eps of a completed long step
  double tol, floor_eps;   // threshold; rounding floor of the working precision
  int iter;                // updates made in the current long step
  int done;                // current long step has stopped iterating
  int status;              // ST_*
  int step, nsteps;        // long steps completed / to do (in this launch)
  int max_iter, fixed_iters;
  int iters_total, iters_min, iters_max;
  int hist[33];
  double spec[4];          // sum |psi0|^2, photon sum (filled by k_spec_sums)
  unsigned tc_err;         // a tensor-core contraction wait timed out
  unsigned sync_err;       // a grid barrier of the long-step kernel timed out
  unsigned arrive;         // blocks of k_trapz<R, true> that have added their sums
  double spec_v;           // sum |psi0|^2 at the start of the current long step (0: take spec[0]),
                           // the bound of the FP16 operand scale (set by k_advance)
  double hdz;              // dz / 2 of this propagation (the trapezoid's weight)
  int idle;                // packed launches: 1 for a slot that holds no propagation
  unsigned batch_arrive;   // (slot 0) slots whose trapezoid decision is made in this iteration
};

struct Geo {
  int N, n, K, P, KK, M;  // modes, samples, pairs, unique (p,l) rows, V rows, substeps
  int raman_mode;         // 0: Kerr only; 1: V = (1-fR) U + fR h*U; 2: V = [U; h*U]
  int ss;                 // self-steepening
  double fR, gamma0, omega0, dt, hdz;  // hdz = dz / 2
  int B;                  // propagations packed in the launch (slots; 1 for one propagation)
};

// Packed launches stack B slots of M + 1 substep slices each: slice =
// b (M + 1) + j.  Every per-slice array (A, NL, I, E, Y, Z, the tensor-core
// operands) is laid out by slice; the per-propagation arrays (psi0, psiR:
// [B][N][n]; dpsi: [B][M][N][n]) by slot; the loop state is an array of B.
__device__ __forceinline__ void slot_of(const Geo& g, int slice, int& b, int& j) {
  b = slice / (g.M + 1);
  j = slice - b * (g.M + 1);
}
// A slice does no work when its slot is empty or has converged in this long
// step, and z0 (j = 0) after the first iteration (its integrand is known).
__device__ __forceinline__ bool slice_skipped(const LoopState* lb, int j) {
  return lb->idle || lb->done || (lb->iter > 0 && j == 0);
}

// Programmatic dependent launch: let the next kernel in the stream start
// launching now, then wait until every kernel this one depends on has
// finished and its writes are visible.  Both are no-ops for a kernel that
// was not launched as a programmatic dependent.
__device__ __forceinline__ void pdl_enter() {
  cudaTriggerProgrammaticLaunchCompletion();
  cudaGridDependencySynchronize();
}

__device__ __forceinline__ double omega_of(int q, int n, double dt) {
  const int s = (q < n / 2) ? q : q - n;
  return 2.0 * 3.14159265358979323846 * (double)s / ((double)n * dt);
}

// ---------------------------------------------------------------------------
// K0: phase tables E_j = exp(i beta (j dz)) for j = 0..M (argument formed in
// FP64 as beta * (j * dz); sincos reduces it mod 2 pi), plus FP64 copies of
// the long-step propagators exp(i beta M dz) and exp(i beta Mrem dz).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_phase_tables(const double* __restrict__ beta, int Nn, int M, double dz, int Mrem,
                               cplx<R>* __restrict__ E, double2* __restrict__ EM64) {
  const size_t total = (size_t)(M + 1) * Nn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / Nn);
    const size_t e = i - (size_t)j * Nn;
    const double zj = (double)j * dz;
    double s, c;
    sincos(beta[e] * zj, &s, &c);
    E[i] = mk<R>((R)c, (R)s);
    if (j == M) EM64[e] = make_double2(c, s);
    if (Mrem > 0 && j == Mrem) EM64[Nn + e] = make_double2(c, s);
  }
}

// ---------------------------------------------------------------------------
// K1: A_j(t) = F^-1{(psi0 + dpsi_j) E_j}   (Eq. cov), grid (N S, M+1); with
// S > 1 the S blocks of a cluster share one transform (fft_cluster).
// ---------------------------------------------------------------------------
// Data written by other blocks earlier in the same kernel (the persistent
// long-step kernel) is read through L2 (__ldcg), never a stale L1 line.
template <typename R, int EPT, int S>
__device__ __forceinline__ void ip_to_time_task(const Geo& g, const cplx<R>* __restrict__ psiR,
                                                const cplx<R>* __restrict__ dpsi, const cplx<R>* __restrict__ E,
                                                cplx<R>* __restrict__ A, const cplx<R>* __restrict__ tw, int iter,
                                                int p, int j, cplx<R>* sm, int slice = -1) {
  // psiR, dpsi: this slot's; E, A: by slice (= j for one propagation)
  const int n = g.n;
  const size_t off = ((size_t)(slice < 0 ? j : slice) * g.N + p) * n;
  const cplx<R>* ps = psiR + (size_t)p * n;
  const cplx<R>* dp = (iter > 0) ? dpsi + ((size_t)(j - 1) * g.N + p) * n : nullptr;
  const cplx<R>* e = E + off;
  const R inv_n = (R)1.0 / (R)n;
  auto load = [&](int q) {
    cplx<R> x = __ldcg(ps + q);
    if (dp) x = cadd<R>(x, __ldcg(dp + q));
    return cmul<R>(x, e[q]);
  };
  auto store = [&](int t, cplx<R> v) { A[off + t] = cscale<R>(v, inv_n); };
  if (S == 1) fft_block<R, -1, EPT>(sm, n, tw, load, store);
  else fft_cluster<R, -1, EPT, S>(sm + fft_smem_elems(n / S), sm, n, tw, load, store);
}

template <typename R, int EPT, int S>
__global__ void __launch_bounds__(512) k_ip_to_time(Geo g, const cplx<R>* __restrict__ psiR,
                                                     const cplx<R>* __restrict__ dpsi,
                                                     const cplx<R>* __restrict__ E, cplx<R>* __restrict__ A,
                                                     const cplx<R>* __restrict__ tw,
                                                     const LoopState* __restrict__ ls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smraw);
  pdl_enter();
  const int p = blockIdx.x / S, slice = blockIdx.y;
  int b, j;
  slot_of(g, slice, b, j);
  const LoopState* lb = ls + b;
  if (slice_skipped(lb, j)) return;
  const size_t Nn = (size_t)g.N * g.n;
  ip_to_time_task<R, EPT, S>(g, psiR + b * Nn, dpsi + (size_t)b * g.M * Nn, E, A, tw, lb->iter, p, j, sm, slice);
}

// U_k(t): |A_m|^2 for m == n, 2 Re(A_m A_n^*) for m < n (pairs k = (m <= n))
template <typename R>
__device__ __forceinline__ R pair_product(const cplx<R>* __restrict__ a, int n, int2 mn, int t) {
  const cplx<R> am = __ldcg(a + (size_t)mn.x * n + t);
  if (mn.x == mn.y) return am.x * am.x + am.y * am.y;
  const cplx<R> an = __ldcg(a + (size_t)mn.y * n + t);
  return (R)2.0 * (am.x * an.x + am.y * an.y);
}

// ---------------------------------------------------------------------------
// K2 of the general coupling: the N^2 real rows of the pair products,
// U_k = Re(A_m A_n^*) for the pairs m <= n and Im(A_m A_n^*) for m < n
// (gpairs[k] = (m, n), n + N for an imaginary row), to Ug [slices][N^2][n].
// grid (ceil(n / 256), slices)
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(256) k_gen_pairs(Geo g, const cplx<R>* __restrict__ A, R* __restrict__ Ug,
                                                   const int2* __restrict__ gpairs, const LoopState* __restrict__ ls) {
  pdl_enter();
  int b, j;
  slot_of(g, blockIdx.y, b, j);
  if (slice_skipped(ls + b, j)) return;
  const int n = g.n, N = g.N, NN = N * N;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const cplx<R>* a = A + (size_t)blockIdx.y * N * n;
  R* u = Ug + (size_t)blockIdx.y * NN * n + t;
  for (int k = 0; k < NN; ++k) {
    const int2 mn = gpairs[k];
    const bool im = mn.y >= N;
    const cplx<R> am = __ldcg(a + (size_t)mn.x * n + t);
    const cplx<R> an = __ldcg(a + (size_t)(im ? mn.y - N : mn.y) * n + t);
    // A_m A_n^* = (am.x an.x + am.y an.y) + i (am.y an.x - am.x an.y)
    u[(size_t)k * n] = im ? am.y * an.x - am.x * an.y : am.x * an.x + am.y * an.y;
  }
}

// ---------------------------------------------------------------------------
// K2: pair products and the Raman convolution Y_k = h_R * U_k for two rows
// at once (U_k1 + i U_k2 is transformed, multiplied by H = (dt/n) DFT(h_R),
// and transformed back; h_R is real so the real and imaginary parts stay
// apart).  SRC 0: the rows are the K pair products, formed from A; SRC 1
// (low-rank coupling): the rows are the cnt = r rows of Z = W U
// ([M+1][r][n]), read from Zs.  Only Y [M+1][cnt][n] is written: the
// contraction forms U from A.  grid (ceil(cnt/2), M+1)
// ---------------------------------------------------------------------------
template <typename R, int EPT, int SRC>
__device__ __forceinline__ void pairs_raman_task(const Geo& g, const cplx<R>* __restrict__ A, R* __restrict__ Y,
                                                 const cplx<R>* __restrict__ H, const cplx<R>* __restrict__ tw,
                                                 const int2* __restrict__ pairs, const R* __restrict__ Zs, int cnt,
                                                 int kp, int j, cplx<R>* sm) {
  const int n = g.n;
  const int k1 = 2 * kp, k2 = k1 + 1;
  const bool has2 = k2 < cnt;
  __syncthreads();  // the block's previous use of sm is over
  auto from_smem = [&](int q) { return sm[pad16(q)]; };
  auto to_smem = [&](int q, cplx<R> x) { sm[pad16(q)] = cmul<R>(x, H[q]); };
  if (SRC == 0) {
    // the pair products are staged in shared memory first: the transform's
    // first pass then reads no global memory, which keeps its registers free
    const int2 mn1 = pairs[k1];
    const int2 mn2 = has2 ? pairs[k2] : mn1;
    const cplx<R>* a = A + (size_t)j * g.N * n;
#pragma unroll 4
    for (int t = threadIdx.x; t < n; t += blockDim.x)
      sm[pad16(t)] = mk<R>(pair_product<R>(a, n, mn1, t), has2 ? pair_product<R>(a, n, mn2, t) : (R)0);
    fft_block<R, -1, EPT>(sm, n, tw, from_smem, to_smem);
  } else {
    // rows of Z: the first pass reads them straight from global memory
    // (every load of the pass in flight at once)
    const R* z1 = Zs + ((size_t)j * cnt + k1) * n;
    auto load = [&](int t) { return mk<R>(__ldcg(z1 + t), has2 ? __ldcg(z1 + n + t) : (R)0); };
    fft_block<R, -1, EPT>(sm, n, tw, load, to_smem);
  }
  R* y1 = Y + ((size_t)j * cnt + k1) * n;
  auto store = [&](int t, cplx<R> y) {
    y1[t] = y.x;
    if (has2) y1[n + t] = y.y;
  };
  fft_block<R, +1, EPT>(sm, n, tw, from_smem, store);
}

template <typename R, int EPT, int SRC>
__global__ void __launch_bounds__(512) k_pairs_raman(Geo g, const cplx<R>* __restrict__ A, R* __restrict__ Y,
                                                      const cplx<R>* __restrict__ H,
                                                      const cplx<R>* __restrict__ tw,
                                                      const int2* __restrict__ pairs, const R* __restrict__ Zs,
                                                      int cnt, const LoopState* __restrict__ ls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smraw);
  pdl_enter();
  int b, j;
  slot_of(g, blockIdx.y, b, j);
  if (slice_skipped(ls + b, j)) return;
  pairs_raman_task<R, EPT, SRC>(g, A, Y, H, tw, pairs, Zs, cnt, blockIdx.x, blockIdx.y, sm);
}

// K2 with the two transforms of a pair spread over an S-block cluster
// (fft_cluster): block s loads the rows of its time slice (SRC 0: the pair
// products of A; SRC 1: rows of Zs, cnt per substep), the spectrum slice it
// ends up holding is multiplied by H in place, and the inverse returns its
// time slice of h_R * U.  grid (S ceil(cnt/2), M+1).
template <typename R, int EPT, int S, int SRC>
__global__ void __launch_bounds__(512) k_pairs_raman_cl(Geo g, const cplx<R>* __restrict__ A, R* __restrict__ Y,
                                                        const cplx<R>* __restrict__ H,
                                                        const cplx<R>* __restrict__ tw,
                                                        const int2* __restrict__ pairs, const R* __restrict__ Zs,
                                                        int cnt, const LoopState* __restrict__ ls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smraw);
  pdl_enter();
  int b, jl;
  slot_of(g, blockIdx.y, b, jl);
  if (slice_skipped(ls + b, jl)) return;  // the same for every block of a cluster
  const int j = blockIdx.y;  // the slice
  const int n = g.n, np = n / S;
  const int s = (int)(blockIdx.x % S);
  cplx<R>* xbuf = sm + fft_smem_elems(np);
  const int k1 = 2 * (blockIdx.x / S), k2 = k1 + 1;
  const bool has2 = k2 < cnt;
  auto load = [&](int t) {
    if (SRC == 0) {
      const int2 mn1 = pairs[k1];
      const int2 mn2 = has2 ? pairs[k2] : mn1;
      const cplx<R>* a = A + (size_t)j * g.N * n;
      return mk<R>(pair_product<R>(a, n, mn1, t), has2 ? pair_product<R>(a, n, mn2, t) : (R)0);
    }
    const R* z1 = Zs + ((size_t)j * cnt + k1) * n;
    return mk<R>(z1[t], has2 ? z1[n + t] : (R)0);
  };
  auto spectrum = [&](int q, cplx<R> x) { xbuf[q - s * np] = cmul<R>(x, H[q]); };
  fft_cluster<R, -1, EPT, S>(xbuf, sm, n, tw, load, spectrum);
  auto own = [&](int q) { return xbuf[q - s * np]; };
  R* y1 = Y + ((size_t)j * cnt + k1) * n;
  auto store = [&](int t, cplx<R> y) {
    y1[t] = y.x;
    if (has2) y1[n + t] = y.y;
  };
  fft_cluster<R, +1, EPT, S>(xbuf, sm, n, tw, own, store);
}

// ---------------------------------------------------------------------------
// K3: NL_p(t) = sum_l A_l R_pl, R_pl = sum_k G[(p,l)][k] V_k  (Eq. 1 bracket,
// symmetry-reduced: rows (p <= l), columns (m <= n) or [U; h*U]).  V is
// formed from A and Y = h_R * U:
//   raman_mode 0: V = U;  1: V = (1 - fR) U + fR Y;  2: V = [U; Y].
// For N > 8 the tiled GEMM of contract_tile.cuh (CUDA cores) or
// tc_contract.cuh (tensor cores) computes it.
// ---------------------------------------------------------------------------
// K3 for N <= 8: the same contraction with every operand in registers
// (compile-time N and raman_mode); the reduced coupling matrix is read from
// shared memory as a broadcast, 16 bytes per load (rows padded to KKP).
// One thread per (j, t).
template <typename R, int N, int MODE>
struct RegShape {
  static constexpr int K = N * (N + 1) / 2;
  static constexpr int KK = MODE == 2 ? 2 * K : K;
  static constexpr int VW = 16 / (int)sizeof(R);       // values per 16-byte load
  static constexpr int KKP = (KK + VW - 1) / VW * VW;  // padded row length
};

// G [K][KK] to shared memory [K][KKP], zero padding (the whole block)
template <typename R, int N, int MODE>
__device__ __forceinline__ void stage_g(const R* __restrict__ Gm, R* Gs) {
  using S = RegShape<R, N, MODE>;
  for (int i = threadIdx.x; i < S::K * S::KKP; i += blockDim.x) {
    const int r = i / S::KKP, k = i - r * S::KKP;
    Gs[i] = k < S::KK ? Gm[r * S::KK + k] : (R)0;
  }
}

// NL of one point pt = j n + t (all N modes)
template <typename R, int N, int MODE>
__device__ __forceinline__ void contract_reg_point(const Geo& g, const cplx<R>* __restrict__ A,
                                                   const R* __restrict__ Y, const R* Gs, cplx<R>* __restrict__ NL,
                                                   size_t pt) {
  using S = RegShape<R, N, MODE>;
  constexpr int K = S::K, KK = S::KK, VW = S::VW, KKP = S::KKP;
  using V16 = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
  const int n = g.n;
  const int j = (int)(pt / n), t = (int)(pt - (size_t)j * n);
  const cplx<R>* a = A + (size_t)j * N * n + t;
  cplx<R> av[N];
#pragma unroll
  for (int l = 0; l < N; ++l) av[l] = __ldcg(a + (size_t)l * n);
  R v[KK];
  {
    const R* yp = Y + (size_t)j * K * n + t;
    const R fR = (R)g.fR, fK = (R)(1.0 - g.fR);
    int k = 0;
#pragma unroll
    for (int m = 0; m < N; ++m)
#pragma unroll
      for (int q = m; q < N; ++q, ++k) {
        const R u = (m == q) ? av[m].x * av[m].x + av[m].y * av[m].y
                             : (R)2 * (av[m].x * av[q].x + av[m].y * av[q].y);
        if (MODE == 0) v[k] = u;
        else if (MODE == 1) v[k] = fK * u + fR * __ldcg(yp + (size_t)k * n);
        else {
          v[k] = u;
          v[K + k] = __ldcg(yp + (size_t)k * n);
        }
      }
  }
  cplx<R> nl[N];
#pragma unroll
  for (int p = 0; p < N; ++p) nl[p] = mk<R>(0, 0);
  int r = 0;
#pragma unroll
  for (int p = 0; p < N; ++p)
#pragma unroll
    for (int l = p; l < N; ++l, ++r) {
      R acc = (R)0;
#pragma unroll
      for (int k4 = 0; k4 < KKP / VW; ++k4) {
        const V16 w = *reinterpret_cast<const V16*>(Gs + r * KKP + k4 * VW);
        const R* wv = reinterpret_cast<const R*>(&w);
#pragma unroll
        for (int i = 0; i < VW; ++i)
          if (k4 * VW + i < KK) acc += wv[i] * v[k4 * VW + i];
      }
      nl[p].x += av[l].x * acc;
      nl[p].y += av[l].y * acc;
      if (l != p) {
        nl[l].x += av[p].x * acc;
        nl[l].y += av[p].y * acc;
      }
    }
  cplx<R>* out = NL + (size_t)j * N * n + t;
#pragma unroll
  for (int p = 0; p < N; ++p) out[(size_t)p * n] = nl[p];
}

template <typename R, int N, int MODE>
__global__ void __launch_bounds__(128) k_contract_reg(Geo g, const cplx<R>* __restrict__ A,
                                                      const R* __restrict__ Y, const R* __restrict__ Gm,
                                                      cplx<R>* __restrict__ NL, const LoopState* __restrict__ ls) {
  using S = RegShape<R, N, MODE>;
  __shared__ __align__(16) R Gs[S::K * S::KKP];
  stage_g<R, N, MODE>(Gm, Gs);
  pdl_enter();
  __syncthreads();
  const int n = g.n;
  const size_t pt = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= (size_t)g.B * (g.M + 1) * n) return;
  int b, j;
  slot_of(g, (int)(pt / n), b, j);
  if (slice_skipped(ls + b, j)) return;
  contract_reg_point<R, N, MODE>(g, A, Y, Gs, NL, pt);
}

// ---------------------------------------------------------------------------
// K4: I_j(w) = i gamma0 s(w) F{NL_p}(w) exp(-i beta j dz)   (Eq. MPA_eq)
// grid (N S, M+1) as K1; fac[q] = gamma0 (1 + w_q/omega0) (or gamma0 without
// self-steepening), tabulated in FP64 and rounded once.
// ---------------------------------------------------------------------------
template <typename R, int EPT, int S>
__device__ __forceinline__ void integrand_task(const Geo& g, const cplx<R>* __restrict__ NL,
                                               const cplx<R>* __restrict__ E, const R* __restrict__ fac,
                                               cplx<R>* __restrict__ I, const cplx<R>* __restrict__ tw, int p, int j,
                                               cplx<R>* sm) {
  const int n = g.n;
  const size_t off = ((size_t)j * g.N + p) * n;
  const cplx<R>* src = NL + off;
  const cplx<R>* e = E + off;
  auto load = [&](int t) { return __ldcg(src + t); };
  auto store = [&](int q, cplx<R> X) {
    const R f = fac[q];  // gamma0 s(w_q)
    const cplx<R> iX = mk<R>(-X.y * f, X.x * f);
    I[off + q] = cmulc<R>(iX, e[q]);
  };
  // correctly rounded table twiddles: twiddles formed as products of table
  // entries (up to 4 ulp, with a bias in their magnitude) scale the
  // integrand by the same small factor in every long step, an error that
  // grows linearly along the fiber in FP32 (1.2e-5 against FP64 after the
  // 0.5 m of the 6-mode fiber, 4.4e-6 with the tables)
  if (S == 1) fft_block<R, +1, EPT, true>(sm, n, tw, 1, load, store);
  else fft_cluster<R, +1, EPT, S>(sm + fft_smem_elems(n / S), sm, n, tw, load, store);
}

template <typename R, int EPT, int S>
__global__ void __launch_bounds__(512) k_integrand(Geo g, const cplx<R>* __restrict__ NL,
                                                    const cplx<R>* __restrict__ E, const R* __restrict__ fac,
                                                    cplx<R>* __restrict__ I,
                                                    const cplx<R>* __restrict__ tw,
                                                    const LoopState* __restrict__ ls) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cplx<R>* sm = reinterpret_cast<cplx<R>*>(smraw);
  pdl_enter();
  const int p = blockIdx.x / S;
  int b, j;
  slot_of(g, blockIdx.y, b, j);
  if (slice_skipped(ls + b, j)) return;
  integrand_task<R, EPT, S>(g, NL, E, fac, I, tw, p, blockIdx.y, sm);
}


// Convergence decision (one thread): eps, stop rule, reset of the sums, and
// the while-node condition when running inside a graph.  Every path ends the
// loop after at most max_iter (or fixed_iters) updates.
__device__ __forceinline__ void decide(LoopState* ls, double diff, double nrm, cudaGraphConditionalHandle h,
                                       int use_cond) {
  const bool finite = isfinite(diff) && isfinite(nrm);
  const double eps = finite ? (nrm > 0.0 ? sqrt(diff / nrm) : 0.0) : nan("");
  const int it = ls->iter + 1;
  bool stop = false;
  if (!finite) {
    ls->status = ST_NONFINITE;
    stop = true;
  } else if (ls->fixed_iters > 0) {
    stop = it >= ls->fixed_iters;
  } else if (eps < ls->tol) {
    stop = true;
  } else if (eps < ls->floor_eps && eps > 0.5 * ls->prev_eps) {
    stop = true;  // rounding-limited: eps no longer contracts
  } else if (it >= ls->max_iter) {
    ls->status = ST_NOT_CONVERGED;
    stop = true;
  }
  if (it >= 4096) stop = true;  // hard cap, whatever the settings
  ls->eps = eps;
  ls->prev_eps = eps;
  ls->iter = it;
  ls->done = stop ? 1 : 0;
  ls->diff = 0.0;
  ls->nrm = 0.0;
  if (use_cond) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

static __global__ void k_decide(LoopState* ls, cudaGraphConditionalHandle h, int use_cond) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  decide(ls, ls->diff, ls->nrm, h, use_cond);
}

// ---------------------------------------------------------------------------
// K5: trapezoid over z' and the convergence sums (Sec. III.D)
//   dpsi_j <- (dz/2) sum_{k=1..j} (I_{k-1} + I_k),
//   diff = sum |new - old|^2, nrm = sum |psi0 + new|^2 over j, p, w: the
//   terms of one element in the working precision, the sums over elements
//   and blocks in FP64.
// One thread per element sweeps j in order; its loads are issued TRAPZ_JC
// substeps at a time (I_j and the previous dpsi_j into registers), so a
// long step of M <= TRAPZ_JC costs one round trip to L2.  Each block writes
// its two sums to part[blockIdx.x]; the last block to finish adds them in a
// fixed order (the result does not depend on block timing) and, with
// DECIDE, takes the convergence decision, else leaves the sums in
// ls->diff / ls->nrm.  Every block reads iter before it arrives, so the last
// one may update it.
// ---------------------------------------------------------------------------
constexpr int TRAPZ_T = 128;
constexpr int TRAPZ_MAX_BLOCKS = 148 * 8;  // partial-sum slots per propagation slot
// K5's grid: at most one wave of resident blocks, four 128-thread blocks per
// SM (the FP32 and FP64 forms take 128 and 119 registers a thread); a second,
// mostly idle wave of blocks cost a third of its time at 42 modes (0.0129
// against 0.0086 ms per iteration)
constexpr int TRAPZ_WAVE = 148 * 4;
template <typename R> struct TrapzJC { static constexpr int value = sizeof(R) == 4 ? 16 : 8; };

inline int trapz_blocks(size_t Nn) {
  const size_t b = (Nn + TRAPZ_T - 1) / TRAPZ_T;
  return (int)(b < 1 ? 1 : (b > (size_t)TRAPZ_WAVE ? TRAPZ_WAVE : b));
}

// Sum of (a, b) over the block (any shape, at most 32 warps); valid in
// thread 0.  red: 64 doubles.
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nw = (blockDim.x * blockDim.y + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if ((tid & 31) == 0) {
    red[tid >> 5] = a;
    red[32 + (tid >> 5)] = b;
  }
  __syncthreads();
  if (tid < 32) {
    a = tid < nw ? red[tid] : 0.0;
    b = tid < nw ? red[32 + tid] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

// The sweep over j of one element; its two terms added to diff and nrm.
template <typename R>
__device__ __forceinline__ void trapz_element(const Geo& g, const cplx<R>* __restrict__ psiR,
                                              cplx<R>* __restrict__ dpsi, const cplx<R>* __restrict__ I, int iter,
                                              size_t e, R hdz, double& diff, double& nrm) {
  constexpr int JC = TrapzJC<R>::value;
  const size_t Nn = (size_t)g.N * g.n;
  const int M = g.M;
  const cplx<R> p0 = __ldcg(psiR + e);
  cplx<R> Ip = __ldcg(I + e);
  cplx<R> acc = mk<R>(0, 0);
  R dsum = 0, nsum = 0;  // this element's terms in the working precision
  for (int j0 = 1; j0 <= M; j0 += JC) {
    cplx<R> ij[JC], old[JC];
#pragma unroll
    for (int i = 0; i < JC; ++i) {
      const int j = j0 + i;
      ij[i] = j <= M ? __ldcg(I + (size_t)j * Nn + e) : mk<R>(0, 0);
      old[i] = (j <= M && iter > 0) ? __ldcg(dpsi + (size_t)(j - 1) * Nn + e) : mk<R>(0, 0);
    }
#pragma unroll
    for (int i = 0; i < JC; ++i) {
      const int j = j0 + i;
      if (j > M) break;
      acc = cadd<R>(acc, cscale<R>(cadd<R>(Ip, ij[i]), hdz));
      Ip = ij[i];
      const R dx = acc.x - old[i].x, dy = acc.y - old[i].y;
      dsum += dx * dx + dy * dy;
      const R px = p0.x + acc.x, py = p0.y + acc.y;
      nsum += px * px + py * py;
      dpsi[(size_t)(j - 1) * Nn + e] = acc;
    }
  }
  diff += (double)dsum;
  nrm += (double)nsum;
}

// Packed launches: grid (blocks, B), one row of blocks per slot (per-slot
// partial sums part[b][block] and arrival counter); a slot that is empty or
// has converged in this long step adds nothing; the last slot to decide sets
// the graph's loop condition: continue while any slot iterates.
template <typename R, bool DECIDE>
__global__ void __launch_bounds__(TRAPZ_T) k_trapz(Geo g, const cplx<R>* __restrict__ psiR, cplx<R>* __restrict__ dpsi,
                                                   const cplx<R>* __restrict__ I, LoopState* ls, double2* part,
                                                   cudaGraphConditionalHandle h, int use_cond) {
  __shared__ double red[64];
  __shared__ bool last;
  pdl_enter();
  const int b = blockIdx.y;
  LoopState* lb = ls + b;
  const size_t Nn = (size_t)g.N * g.n;
  const bool work = !lb->idle && !lb->done;
  const int iter = lb->iter;
  const int tid = threadIdx.x;
  double diff = 0.0, nrm = 0.0;
  if (work) {
    const R hdz = (R)lb->hdz;
    const cplx<R>* pR = psiR + b * Nn;
    cplx<R>* dp = dpsi + (size_t)b * g.M * Nn;
    const cplx<R>* Ib = I + (size_t)b * (g.M + 1) * Nn;
    for (size_t e = (size_t)blockIdx.x * TRAPZ_T + tid; e < Nn; e += (size_t)gridDim.x * TRAPZ_T)
      trapz_element<R>(g, pR, dp, Ib, iter, e, hdz, diff, nrm);
  }
  block_sum2(diff, nrm, red);
  double2* pb = part + (size_t)b * TRAPZ_MAX_BLOCKS;
  if (tid == 0) {
    pb[blockIdx.x] = make_double2(diff, nrm);
    __threadfence();
    last = atomicAdd(&lb->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  diff = 0.0;
  nrm = 0.0;
  for (int k = tid; k < (int)gridDim.x; k += TRAPZ_T) {
    const double2 v = __ldcg(&pb[k]);
    diff += v.x;
    nrm += v.y;
  }
  block_sum2(diff, nrm, red);
  if (tid == 0) {
    lb->arrive = 0;
    if (work) {
      if (DECIDE) {
        decide(lb, diff, nrm, h, use_cond && g.B == 1);
      } else {
        lb->diff = diff;
        lb->nrm = nrm;
      }
    }
    if (DECIDE && use_cond && g.B > 1) {
      __threadfence();
      if (atomicAdd(&ls->batch_arrive, 1u) == gridDim.y - 1) {
        __threadfence();
        ls->batch_arrive = 0;
        bool any = false;
        for (int k = 0; k < g.B; ++k) {
          const volatile LoopState* v = ls + k;
          if (!v->idle && !v->done) any = true;
        }
        cudaGraphSetConditional(h, any ? 1u : 0u);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Long-step bookkeeping (one thread): statistics, the reset of the iteration
// state, and in a graph the outer while-node condition (continue while the
// step succeeded and steps remain) and the inner one re-armed for the next
// long step.
__device__ __forceinline__ void step_end(LoopState* ls, cudaGraphConditionalHandle hStep,
                                         cudaGraphConditionalHandle hIter, int use_cond, bool rearm_iter = true) {
  const int status = ls->status, it = ls->iter;
  if (status == ST_OK) {
    ls->step += 1;
    ls->iters_total += it;
    ls->iters_min = min(ls->iters_min, it);
    ls->iters_max = max(ls->iters_max, it);
    ls->hist[min(it, 32)] += 1;
    ls->eps_max = fmax(ls->eps_max, ls->eps);
  }
  ls->iter = 0;
  ls->done = 0;
  ls->prev_eps = INFINITY;
  if (use_cond) {
    cudaGraphSetConditional(hStep, (status == ST_OK && ls->step < ls->nsteps) ? 1u : 0u);
    if (rearm_iter) cudaGraphSetConditional(hIter, 1u);
  }
}

// K6: end of a long step (Sec. III.D): A~(z0 + L) = (psi0 + dpsi_M) exp(i beta M dz)
// in FP64; becomes the next psi0.  Skipped when the long step failed.  Each
// block also sums |psi0|^2 of its elements (FP64) into part[blockIdx.x]; the
// last block to finish adds those in a fixed order into ls->spec_v (the
// energy bound of the next long step's FP16 operand scale, which a gain can
// raise) and does the long-step bookkeeping (every block reads the status
// before it arrives).
// Packed launches: grid (blocks, B), slot b's psi0, psiR, dpsi and EM at
// their slot offsets (EM + b em_stride); the graph conditions are set only
// for one propagation (a packed launch runs one long step per launch).
template <typename R>
__global__ void __launch_bounds__(256) k_advance(Geo g, double2* __restrict__ psi0, cplx<R>* psiR,
                                                 const cplx<R>* __restrict__ dpsi,
                                                 const double2* __restrict__ EM, LoopState* ls,
                                                 cudaGraphConditionalHandle hStep, cudaGraphConditionalHandle hIter,
                                                 int use_cond, double2* part, size_t em_stride) {
  __shared__ bool last;
  __shared__ double red[32];
  pdl_enter();
  const int b = blockIdx.y;
  LoopState* lb = ls + b;
  const size_t Nn = (size_t)g.N * g.n;
  double2* p0 = psi0 + b * Nn;
  cplx<R>* pR = psiR + b * Nn;
  const double2* em = EM + b * em_stride;
  double e2 = 0.0;
  if (!lb->idle && lb->status == ST_OK) {
    const cplx<R>* d = dpsi + ((size_t)b * g.M + (g.M - 1)) * Nn;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < Nn; e += (size_t)gridDim.x * blockDim.x) {
      const double2 q0 = p0[e];
      const cplx<R> dd = d[e];
      const double x = q0.x + (double)dd.x, y = q0.y + (double)dd.y;
      const double2 w = em[e];
      const double2 v = make_double2(x * w.x - y * w.y, x * w.y + y * w.x);
      p0[e] = v;
      e2 += v.x * v.x + v.y * v.y;
      if ((const void*)psiR != (const void*)psi0) pR[e] = mk<R>((R)v.x, (R)v.y);
    }
  }
  e2 = block_sum(e2, red);
  double2* pb = part + (size_t)b * TRAPZ_MAX_BLOCKS;
  if (threadIdx.x == 0) {
    pb[blockIdx.x] = make_double2(e2, 0.0);
    __threadfence();
    last = atomicAdd(&lb->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double tot = 0.0;
  for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) tot += __ldcg(&pb[k]).x;
  tot = block_sum(tot, red);
  if (threadIdx.x == 0) {
    lb->arrive = 0;
    if (!lb->idle) {
      if (lb->status == ST_OK) lb->spec_v = tot;
      step_end(lb, hStep, hIter, use_cond && g.B == 1);
    }
  }
}

// psiR = psi0 rounded to the working precision (start of a propagation).
template <typename R>
__global__ void k_round_psi(const double2* __restrict__ psi0, cplx<R>* __restrict__ psiR, size_t count) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    psiR[e] = mk<R>((R)psi0[e].x, (R)psi0[e].y);
}

// ---------------------------------------------------------------------------
// Terms of Sec. IV added to the right-hand side of Eq. 1, none of which
// depends on time within a substep, so each acts on every frequency alike
// and joins the integrand after K4: the linear mode coupling
// C_p = i sum_n Q_np(z) A_n with Q_np(z) = Q_np f(z), the small-signal gain
// g_p A_p, and its saturation - sat sum_l R_pl A_l with
// R_pl = sum_mn S^R_plmn int A_m A_n^* dtau (real and symmetric for an S^R
// of Eq. 2).  In the interaction picture
//   I_j,p += exp(-i beta_p j dz) (i f(z_j) sum_n Q_np - sat R_pl(j)) A~_n,j
//            + g_p (psi_p + dpsi_p,j),
// with A~_n,j = (psi_n + dpsi_n,j) E_n,j the spectrum K1 transforms (the
// gain's phase and the interaction picture's cancel).  Slices follow K1:
// j = 0 only in the first iteration, dpsi only after it.  One thread per
// (substep, frequency), all modes; the coefficients FP64, used in R.
// ---------------------------------------------------------------------------
struct LinTerms {
  const double* Q;       // [N][N] Q[n][p], or null
  const double* gain;    // [N] g_p, or null
  const double* fprof;   // f(z) at z = k fdz, k < fcount (linear interpolation), or null (f = 1)
  int fcount;
  double fdz;
  const double* Rs;      // [M+1][P] saturation rows R_(p<=l)(j), or null
  double sat;            // the saturation's coefficient (1/I_sat)
  int Mfull;             // substeps of a full long step: z0 = (long steps done) Mfull dz
  int use_step;          // 1: z0 from the loop state; 0: z0 = zoff
  double zoff;
};

__device__ __forceinline__ double profile_at(const LinTerms& t, double z) {
  if (!t.fprof) return 1.0;
  const double u = z / t.fdz;
  if (!(u > 0.0)) return t.fprof[0];
  const int k = (int)u;
  if (k >= t.fcount - 1) return t.fprof[t.fcount - 1];
  const double w = u - (double)k;
  return t.fprof[k] + w * (t.fprof[k + 1] - t.fprof[k]);
}

template <typename R>
__global__ void k_linear_coupling(Geo g, LinTerms lt, const cplx<R>* __restrict__ psiR,
                                  const cplx<R>* __restrict__ dpsi, const cplx<R>* __restrict__ E,
                                  cplx<R>* __restrict__ I, const LoopState* __restrict__ ls) {
  const int N = g.N, n = g.n, iter = ls->iter;
  const double dz = 2.0 * g.hdz;
  const double z0 = lt.use_step ? (double)ls->step * lt.Mfull * dz : lt.zoff;
  const size_t total = (size_t)(g.M + 1) * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / n), q = (int)(i - (size_t)j * n);
    if (iter > 0 && j == 0) continue;
    const R fq = lt.Q ? (R)profile_at(lt, z0 + j * dz) : (R)0;
    const double* rs = lt.Rs ? lt.Rs + (size_t)j * g.P : nullptr;
    for (int p = 0; p < N; ++p) {
      cplx<R>* o = I + ((size_t)j * N + p) * n + q;
      if (lt.gain) {
        cplx<R> a = psiR[(size_t)p * n + q];
        if (iter > 0) {
          const cplx<R> d = dpsi[((size_t)(j - 1) * N + p) * n + q];
          a.x += d.x;
          a.y += d.y;
        }
        const R gp = (R)lt.gain[p];
        o->x += gp * a.x;
        o->y += gp * a.y;
      }
      if (!lt.Q && !rs) continue;
      // c = sum_m (i f Q_mp - sat R_pm) A~_m: cq from the coupling, cs from the saturation
      R cqx = 0, cqy = 0, csx = 0, csy = 0;
      for (int m = 0; m < N; ++m) {
        cplx<R> a = psiR[(size_t)m * n + q];
        if (iter > 0) {
          const cplx<R> d = dpsi[((size_t)(j - 1) * N + m) * n + q];
          a.x += d.x;
          a.y += d.y;
        }
        const cplx<R> e = E[((size_t)j * N + m) * n + q];
        const R ax = a.x * e.x - a.y * e.y, ay = a.x * e.y + a.y * e.x;
        if (lt.Q) {
          const R w = fq * (R)lt.Q[(size_t)m * N + p];
          cqx += w * ax;
          cqy += w * ay;
        }
        if (rs) {
          const int lo = p < m ? p : m, hi = p < m ? m : p;
          const R w = (R)(lt.sat * rs[lo * N - lo * (lo - 1) / 2 + (hi - lo)]);
          csx += w * ax;
          csy += w * ay;
        }
      }
      // i (cqx + i cqy) - (csx + i csy), times conj(E_p,j)
      const cplx<R> e = E[((size_t)j * N + p) * n + q];
      const R tx = -cqy - csx, ty = cqx - csy;
      o->x += tx * e.x + ty * e.y;
      o->y += ty * e.x - tx * e.y;
    }
  }
}

// The time integrals of the pair products at every substep, for the
// saturation: Ubar[j][k(m,n)] = dt sum_t U_mn(t) with U_mm = |A_m|^2 and
// U_mn = 2 Re(A_m A_n^*) (m < n), so that sum_{m<=n} S^R_pl,mn Ubar_mn =
// sum_mn S^R_plmn int A_m A_n^* dtau for an S^R symmetric in m, n.  FP64
// sums; block (m, j) takes the pairs (m, n >= m).
template <typename R>
__global__ void __launch_bounds__(256) k_sat_gram(Geo g, const cplx<R>* __restrict__ A, double* __restrict__ Ubar,
                                                  const LoopState* __restrict__ ls) {
  __shared__ double red[32];
  const int m = blockIdx.x, j = blockIdx.y, N = g.N, n = g.n;
  if (ls->iter > 0 && j == 0) return;
  const cplx<R>* a = A + (size_t)j * N * n;
  const int k0 = m * N - m * (m - 1) / 2;
  for (int q = m; q < N; ++q) {
    double acc = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
      const cplx<R> am = a[(size_t)m * n + t], aq = a[(size_t)q * n + t];
      acc += (double)am.x * (double)aq.x + (double)am.y * (double)aq.y;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) Ubar[(size_t)j * g.K + k0 + (q - m)] = g.dt * (q == m ? acc : 2.0 * acc);
  }
}

// R_r(j) = sum_k S^R[r][k] Ubar[j][k] for the rows r = (p <= l): GRt is the
// reduced S^R transposed, [K][P] (FP64).  One thread per (row, substep).
static __global__ void k_sat_rows(int P, int K, const double* __restrict__ GRt, const double* __restrict__ Ubar,
                                  double* __restrict__ Rs, const LoopState* __restrict__ ls) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (r >= P || (ls->iter > 0 && j == 0)) return;
  const double* u = Ubar + (size_t)j * K;
  double acc = 0.0;
  for (int k = 0; k < K; ++k) acc += GRt[(size_t)k * P + r] * u[k];
  Rs[(size_t)j * P + r] = acc;
}

// ---------------------------------------------------------------------------
// RK4IP, the split-step comparator of the MPA (Sec. III.D, Fig. 3): fourth-
// order Runge-Kutta in the interaction picture with its origin half a step
// in, so exp(D h/2) is applied three times per step.  The nonlinear operator
// N(X) = i gamma0 s(w) F{NL(F^-1 X)} is K1-K4 on slice 0 (phase 1); this
// kernel makes the elementwise combinations around its four evaluations.  A
// is the FP64 spectral field at the start of the step, Eh = exp(i beta h/2)
// (FP64), AI = Eh A, acc the running combination, I = N(X) of the last
// evaluation, X the next argument of N in the working precision.
//   stage 0: X = A
//   stage 1: k1 = Eh N(A); AI = Eh A; acc = AI + h/6 k1; X = AI + h/2 k1
//   stage 2: k2 = N(X); acc += h/3 k2; X = AI + h/2 k2
//   stage 3: k3 = N(X); acc += h/3 k3; X = Eh (AI + h k3)
//   stage 4: k4 = N(X); A = Eh acc + h/6 k4; X = A
// ---------------------------------------------------------------------------
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zaxpy(double2 y, double a, double2 x) {
  return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y));
}

template <typename R>
__global__ void k_rk4_stage(int stage, size_t count, double h, double2* __restrict__ A, double2* __restrict__ AI,
                            double2* __restrict__ acc, const cplx<R>* __restrict__ I,
                            const double2* __restrict__ Eh, cplx<R>* __restrict__ X) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    double2 x;
    if (stage == 0) {
      x = A[e];
    } else {
      const double2 k = make_double2((double)I[e].x, (double)I[e].y);
      const double2 eh = Eh[e];
      if (stage == 1) {
        const double2 k1 = zmul(eh, k), ai = zmul(eh, A[e]);
        AI[e] = ai;
        acc[e] = zaxpy(ai, h / 6.0, k1);
        x = zaxpy(ai, 0.5 * h, k1);
      } else if (stage == 2) {
        acc[e] = zaxpy(acc[e], h / 3.0, k);
        x = zaxpy(AI[e], 0.5 * h, k);
      } else if (stage == 3) {
        acc[e] = zaxpy(acc[e], h / 3.0, k);
        x = zmul(eh, zaxpy(AI[e], h, k));
      } else {
        x = zaxpy(zmul(eh, acc[e]), h / 6.0, k);
        A[e] = x;
      }
    }
    X[e] = mk<R>((R)x.x, (R)x.y);
  }
}

// ---------------------------------------------------------------------------
// FP64 helpers used once per propagation
// ---------------------------------------------------------------------------
// out_p = scale * DFT_DIR(in_p) for each mode row p (grid N), n <= 8192.
template <int DIR, int EPT>
__global__ void __launch_bounds__(512) k_fft64_rows(const double2* __restrict__ in, double2* __restrict__ out,
                                                     int n, double scale, const double2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const size_t off = (size_t)blockIdx.x * n;
  auto load = [&](int i) { return in[off + i]; };
  auto store = [&](int i, double2 v) { out[off + i] = make_double2(v.x * scale, v.y * scale); };
  fft_block<double, DIR, EPT>(sm, n, tw, load, store);
}

// Half-length transforms of the even and odd samples (for n = 16384 in FP64):
// out[2][rows][n/2]; blockIdx.y selects even (0) / odd (1).
template <int DIR, int EPT>
__global__ void __launch_bounds__(512) k_fft64_halves(const double2* __restrict__ in, double2* __restrict__ out,
                                                       int n, const double2* __restrict__ tw_half) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double2* sm = reinterpret_cast<double2*>(smraw);
  const int h = n / 2, par = blockIdx.y;
  const double2* src = in + (size_t)blockIdx.x * n;
  double2* dst = out + ((size_t)par * gridDim.x + blockIdx.x) * h;
  auto load = [&](int i) { return src[2 * i + par]; };
  auto store = [&](int i, double2 v) { dst[i] = v; };
  fft_block<double, DIR, EPT>(sm, h, tw_half, load, store);
}

// X_q = scale (Y_e[q mod h] + W^q Y_o[q mod h]), W = exp(DIR 2 pi i / n); tw[m] = exp(-2 pi i m/n)
template <int DIR>
__global__ void k_fft64_combine(const double2* __restrict__ half, double2* __restrict__ out, int rows, int n,
                                double scale, const double2* __restrict__ tw) {
  const int h = n / 2;
  const size_t total = (size_t)rows * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / n), q = (int)(i - (size_t)r * n);
    const int qm = q & (h - 1);
    const double2 ye = half[(size_t)r * h + qm];
    const double2 yo = half[((size_t)rows + r) * h + qm];
    double2 w = tw[q];
    if (DIR > 0) w.y = -w.y;
    out[i] = make_double2(scale * (ye.x + w.x * yo.x - w.y * yo.y), scale * (ye.y + w.x * yo.y + w.y * yo.x));
  }
}

// Energy-like sums of the spectrum: spec[0] = sum |psi|^2,
// spec[1] = sum_{w0 + w > 0} |psi|^2 / (w0 + w).
static __global__ void k_spec_sums(const double2* __restrict__ psi, int N, int n, double dt, double omega0,
                            double* __restrict__ spec) {
  __shared__ double red[32];
  double s0 = 0.0, s1 = 0.0;
  const size_t total = (size_t)N * n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % n);
    const double a2 = psi[i].x * psi[i].x + psi[i].y * psi[i].y;
    s0 += a2;
    const double w = omega0 + omega_of(q, n, dt);
    if (w > 0.0) s1 += a2 / w;
  }
  s0 = block_sum(s0, red);
  s1 = block_sum(s1, red);
  if (threadIdx.x == 0) {
    atomicAdd(&spec[0], s0);
    atomicAdd(&spec[1], s1);
  }
}

// Raman transfer function H[q] = (dt/n) DFT_-(h_R)[q] from an FP64 spectrum,
// and (when Hv is given) Hv[q] = (1 - fR)/n + fR H[q], the transfer function
// of (1 - fR) x + fR h_R * x, both formed in FP64 and rounded once.
template <typename R>
__global__ void k_raman_H(const double2* __restrict__ hspec, cplx<R>* __restrict__ H, float2* __restrict__ Hv,
                          int n, double dt, double fR) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const double hx = hspec[q].x * dt / n, hy = hspec[q].y * dt / n;
  H[q] = mk<R>((R)hx, (R)hy);
  if (Hv) Hv[q] = make_float2((float)((1.0 - fR) / n + fR * hx), (float)(fR * hy));
}

// Check a field for NaN / Inf (flag set to 1 if any).
static __global__ void k_nonfinite(const double2* __restrict__ x, size_t count, int* flag) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i].x) || !isfinite(x[i].y)) *flag = 1;
}

}  // namespace gm
