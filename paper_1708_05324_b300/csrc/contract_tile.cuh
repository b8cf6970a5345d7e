// Coupling contraction on the CUDA cores for any N (FP32 / FP64).
//
// Per point (j, t) of the MPA iteration (Eq. 1 bracket after the symmetry
// rewrite):  R_r = sum_k G[r][k] V_k   (rows r = (p <= l)),
//            NL_p = sum_l A_l R_pl.
// Over a tile of TP points and a block of TR rows this is the GEMM
//   D[TP x TR] = V[TP x KK] . Gt[KK x TR]
// computed in registers (TM x TN per thread, 16 x 16 threads; thread (x, y)
// holds points y TM + i and rows x + 16 j) from K chunks of KC staged in
// shared memory; the global loads of the next chunk are issued before the
// products of the current one.  V is formed while it is staged, from the
// tile's mode values A (held in shared memory for the whole block) and from
// Y = h_R * U:  raman_mode 0: V = U;  1: V = (1 - fR) U + fR Y;  2: V = [U; Y]
// (U_mm = |A_m|^2, U_mn = 2 Re(A_m A_n^*)).  A block loops over every row
// block of its points, so NL is complete in the block: each D element adds
// A_l R_r into NL_p (and A_p R_r into NL_l) with shared-memory atomics.
//
// Gt is the reduced coupling matrix transposed and zero-padded:
// [KKp][Pp], KKp a multiple of KC and Pp a multiple of TR.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace gm {

template <typename R> struct TileCfg;
template <> struct TileCfg<float> {
  static constexpr int TP = 128, TR = 128, TM = 8, TN = 8, KC = 16;
};
template <> struct TileCfg<double> {
  static constexpr int TP = 64, TR = 128, TM = 4, TN = 8, KC = 16;
};

// dynamic shared memory of k_contract_tile: A and NL tiles ([N][TP] complex)
// plus the V and G chunks
template <typename R> __host__ __device__ constexpr size_t contract_tile_smem(int N) {
  return (size_t)2 * N * TileCfg<R>::TP * 2 * sizeof(R) +
         (size_t)TileCfg<R>::KC * (TileCfg<R>::TP + TileCfg<R>::TR) * sizeof(R);
}

template <typename R, int MODE>
__global__ void __launch_bounds__(256) k_contract_tile(Geo g, const cplx<R>* __restrict__ A, const R* __restrict__ Y,
                                                       const R* __restrict__ Gt, int KKp, int Pp,
                                                       const int2* __restrict__ rows, const int2* __restrict__ pairs,
                                                       cplx<R>* __restrict__ NL, const LoopState* __restrict__ ls) {
  using C = TileCfg<R>;
  constexpr int TP = C::TP, TR = C::TR, TM = C::TM, TN = C::TN, KC = C::KC;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.N, n = g.n, K = g.K, KK = g.KK;
  cplx<R>* As = reinterpret_cast<cplx<R>*>(smraw);  // [N][TP]
  cplx<R>* Ns = As + (size_t)N * TP;                // [N][TP]
  R* Vs = reinterpret_cast<R*>(Ns + (size_t)N * TP);  // [KC][TP]
  R* Gs = Vs + KC * TP;                               // [KC][TR]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  pdl_enter();
  const int iter = ls->iter;
  const size_t npts = (size_t)(g.M + 1) * n;
  const size_t pt0 = (size_t)blockIdx.x * TP;
  // the z0 points are known after the first iteration
  if (iter > 0 && pt0 + TP <= (size_t)n) return;

  // this block's mode values; NL accumulators cleared
  for (int i = tid; i < N * TP; i += 256) {
    const int l = i / TP, q = i - l * TP;
    const size_t pt = pt0 + q;
    cplx<R> a = mk<R>(0, 0);
    if (pt < npts) {
      const size_t j = pt / n, t = pt - j * n;
      if (!(iter > 0 && j == 0)) a = A[(j * N + l) * n + t];
    }
    As[i] = a;
    Ns[i] = mk<R>(0, 0);
  }
  // the V-chunk elements this thread stages: point q, chunk rows
  // kk = kq + KSTEP i; the G-chunk elements: tid + 256 i
  const int q = tid % TP, kq = tid / TP;
  constexpr int KSTEP = 256 / TP, NV = KC / KSTEP, NG = KC * TR / 256;
  const size_t ptq = pt0 + q;
  const bool okq = ptq < npts && !(iter > 0 && ptq < (size_t)n);
  const size_t jq = ptq < npts ? ptq / n : 0, tq = ptq < npts ? ptq - jq * n : 0;
  const R* yq = Y + jq * (size_t)K * n + tq;
  const R fR = (R)g.fR, fK = (R)(1.0 - g.fR);
  R yreg[NV], greg[NG];
  // global loads of chunk k0 into registers (issued one chunk ahead)
  auto fetch = [&](int rb, int k0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int k = k0 + kq + KSTEP * i;
      const bool need = okq && k < KK && (MODE == 1 || (MODE == 2 && k >= K));
      yreg[i] = need ? yq[(size_t)(MODE == 2 ? k - K : k) * n] : (R)0;
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      const int e = tid + 256 * i, kk = e / TR, r = e - kk * TR;
      greg[i] = Gt[(size_t)(k0 + kk) * Pp + rb + r];
    }
  };
  // V from U (shared memory) and the fetched Y; G as fetched
  auto stage = [&](int k0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int kk = kq + KSTEP * i, k = k0 + kk;
      R v = (R)0;
      if (okq && k < KK) {
        R u = (R)0;
        if (MODE != 2 || k < K) {
          const int2 mn = pairs[k];
          const cplx<R> am = As[mn.x * TP + q];
          if (mn.x == mn.y) u = am.x * am.x + am.y * am.y;
          else {
            const cplx<R> an = As[mn.y * TP + q];
            u = (R)2 * (am.x * an.x + am.y * an.y);
          }
        }
        if (MODE == 0) v = u;
        else if (MODE == 1) v = fK * u + fR * yreg[i];
        else v = k < K ? u : yreg[i];
      }
      Vs[kk * TP + q] = v;
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) Gs[tid + 256 * i] = greg[i];
  };
  __syncthreads();

  for (int rb = 0; rb < Pp; rb += TR) {
    R acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int jn = 0; jn < TN; ++jn) acc[i][jn] = (R)0;
    fetch(rb, 0);
    for (int k0 = 0; k0 < KKp; k0 += KC) {
      stage(k0);
      __syncthreads();
      if (k0 + KC < KKp) fetch(rb, k0 + KC);  // in flight during the products below
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        R a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = Vs[kk * TP + ty * TM + i];
#pragma unroll
        for (int jn = 0; jn < TN; ++jn) b[jn] = Gs[kk * TR + tx + 16 * jn];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int jn = 0; jn < TN; ++jn) acc[i][jn] += a[i] * b[jn];
      }
      __syncthreads();
    }
    // l-sum: NL_p += A_l R_(p,l), NL_l += A_p R_(p,l)
#pragma unroll
    for (int jn = 0; jn < TN; ++jn) {
      const int r = rb + tx + 16 * jn;
      if (r >= g.P) continue;
      const int2 pl = rows[r];
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int qq = ty * TM + i;
        const R v = acc[i][jn];
        const cplx<R> al = As[pl.y * TP + qq];
        atomicAdd(&Ns[pl.x * TP + qq].x, al.x * v);
        atomicAdd(&Ns[pl.x * TP + qq].y, al.y * v);
        if (pl.x != pl.y) {
          const cplx<R> ap = As[pl.x * TP + qq];
          atomicAdd(&Ns[pl.y * TP + qq].x, ap.x * v);
          atomicAdd(&Ns[pl.y * TP + qq].y, ap.y * v);
        }
      }
    }
  }
  __syncthreads();
  for (int i = tid; i < N * TP; i += 256) {
    const int p = i / TP, qq = i - p * TP;
    const size_t pt = pt0 + qq;
    if (pt >= npts) continue;
    const size_t j = pt / n, t = pt - j * n;
    if (iter > 0 && j == 0) continue;
    NL[(j * N + p) * n + t] = Ns[i];
  }
}

}  // namespace gm
