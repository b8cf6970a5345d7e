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
// products of the current one.  A block loops over every row block of its
// points, so each point's result is complete in the block.
//
// The operand V is formed while it is staged:
//   SRC 0, from the tile's mode values A (held in shared memory for the whole
//     block) and from Y = h_R * U ([M+1][K][n]):
//     MODE 0: V = U;  1: V = (1 - fR) U + fR Y;  2: V = [U; Y]
//     (U_mm = |A_m|^2, U_mn = 2 Re(A_m A_n^*));
//   SRC 1 (second GEMM of the low-rank coupling; the general coupling),
//     from the rows of Z and Y' = h_R * Z ([slices][cnt][n]):  MODE 0:
//     V = Z;  1: V = (1 - fR) Z + fR Y';  2: V = [Z; Y'] (KK = 2 cnt).
// The result goes:
//   OUT 0: to the l-sum NL_p = sum_l A_l R_(p,l), formed per (point, p) in a
//     fixed order from the accumulators staged in shared memory (rows
//     ordered by diagonal l - p); NL written at the end;
//   OUT 1 (first GEMM of the low-rank coupling): D rows stored as Z
//     ([M+1][rows][n]);
//   OUT 2 (general coupling): the rows are the real and imaginary parts of
//     a complex R_pl for every (p, l), row 2 (p N + l) + {0, 1}, and
//     NL_p = sum_l A_l R_pl, formed per (point, p) in increasing l.
//
// Gt is the coupling matrix transposed and zero-padded: [KKp][Pp], KKp a
// multiple of KC and Pp a multiple of TR.
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

// Operands of one launch.  KK: the K dimension (K, KK or r); rows: the rows
// with a result (P, or r for OUT 1); Ys: Y (SRC 0) or Y' (SRC 1); Zs: Z
// (SRC 1); Zout: Z (OUT 1); cnt: the row count of Ys / Zs / Zout.
template <typename R>
struct TileArgs {
  const cplx<R>* A;
  const R* Ys;
  const R* Zs;
  const R* Gt;
  int KK, KKp, Pp, rows, cnt;
  const int2* rowpl;  // (p, l) of each row (OUT 0)
  const int2* pairs;  // (m, n) of each pair term (SRC 0)
  cplx<R>* NL;
  R* Zout;
};

template <typename R, int MODE, int SRC, int OUT>
__global__ void __launch_bounds__(256) k_contract_tile(Geo g, TileArgs<R> a, const LoopState* __restrict__ ls) {
  using C = TileCfg<R>;
  constexpr int TP = C::TP, TR = C::TR, TM = C::TM, TN = C::TN, KC = C::KC;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = g.N, n = g.n, K = g.K, KK = a.KK;
  cplx<R>* As = reinterpret_cast<cplx<R>*>(smraw);  // [N][TP]
  cplx<R>* Ns = As + (size_t)N * TP;                // [N][TP]
  R* Vs = reinterpret_cast<R*>(Ns + (size_t)N * TP);  // [KC][TP]
  R* Gs = Vs + KC * TP;                               // [KC][TR]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  pdl_enter();
  const size_t npts = (size_t)g.B * (g.M + 1) * n;
  const size_t pt0 = (size_t)blockIdx.x * TP;
  // points whose slice does no work (the z0 points after the first
  // iteration; in a packed launch, empty and converged slots)
  auto skip = [&](size_t pt) {
    int b, j;
    slot_of(g, (int)(pt / n), b, j);
    return slice_skipped(ls + b, j);
  };
  {
    const size_t ptl = (pt0 + TP <= npts ? pt0 + TP : npts) - 1;
    if (pt0 / n == ptl / n && skip(pt0)) return;  // the tile lies in one such slice
  }

  // this block's mode values; NL accumulators cleared
  for (int i = tid; i < N * TP; i += 256) {
    const int l = i / TP, q = i - l * TP;
    const size_t pt = pt0 + q;
    cplx<R> v = mk<R>(0, 0);
    if (pt < npts) {
      const size_t j = pt / n, t = pt - j * n;
      if (!skip(pt)) v = a.A[(j * N + l) * n + t];
    }
    As[i] = v;
    Ns[i] = mk<R>(0, 0);
  }
  // the V-chunk elements this thread stages: point q, chunk rows
  // kk = kq + KSTEP i; the G-chunk elements: tid + 256 i
  const int q = tid % TP, kq = tid / TP;
  constexpr int KSTEP = 256 / TP, NV = KC / KSTEP, NG = KC * TR / 256;
  const size_t ptq = pt0 + q;
  const bool okq = ptq < npts && !skip(ptq);
  const size_t jq = ptq < npts ? ptq / n : 0, tq = ptq < npts ? ptq - jq * n : 0;
  const R* yq = a.Ys + (jq * (size_t)a.cnt) * n + tq;
  const R* zq = SRC == 1 ? a.Zs + (jq * (size_t)a.cnt) * n + tq : nullptr;
  const R fR = (R)g.fR, fK = (R)(1.0 - g.fR);
  R yreg[NV], zreg[NV], greg[NG];
  // global loads of chunk k0 into registers (issued one chunk ahead)
  auto fetch = [&](int rb, int k0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int k = k0 + kq + KSTEP * i;
      const bool ok = okq && k < KK;
      if (SRC == 0) {
        const bool need = ok && (MODE == 1 || (MODE == 2 && k >= K));
        yreg[i] = need ? yq[(size_t)(MODE == 2 ? k - K : k) * n] : (R)0;
      } else if (MODE == 2) {
        zreg[i] = ok ? (k < a.cnt ? zq[(size_t)k * n] : yq[(size_t)(k - a.cnt) * n]) : (R)0;
      } else {
        zreg[i] = ok ? zq[(size_t)k * n] : (R)0;
        yreg[i] = (ok && MODE == 1) ? yq[(size_t)k * n] : (R)0;
      }
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) {
      const int e = tid + 256 * i, kk = e / TR, r = e - kk * TR;
      greg[i] = a.Gt[(size_t)(k0 + kk) * a.Pp + rb + r];
    }
  };
  // V from U (shared memory) and the fetched rows; G as fetched
  auto stage = [&](int k0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      const int kk = kq + KSTEP * i, k = k0 + kk;
      R v = (R)0;
      if (okq && k < KK) {
        if (SRC == 0) {
          R u = (R)0;
          if (MODE != 2 || k < K) {
            const int2 mn = a.pairs[k];
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
        } else {
          v = MODE == 1 ? fK * zreg[i] + fR * yreg[i] : zreg[i];
        }
      }
      Vs[kk * TP + q] = v;
    }
#pragma unroll
    for (int i = 0; i < NG; ++i) Gs[tid + 256 * i] = greg[i];
  };
  __syncthreads();

  for (int rb = 0; rb < a.Pp; rb += TR) {
    R acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int jn = 0; jn < TN; ++jn) acc[i][jn] = (R)0;
    fetch(rb, 0);
    for (int k0 = 0; k0 < a.KKp; k0 += KC) {
      stage(k0);
      __syncthreads();
      if (k0 + KC < a.KKp) fetch(rb, k0 + KC);  // in flight during the products below
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        R av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = Vs[kk * TP + ty * TM + i];
#pragma unroll
        for (int jn = 0; jn < TN; ++jn) bv[jn] = Gs[kk * TR + tx + 16 * jn];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int jn = 0; jn < TN; ++jn) acc[i][jn] += av[i] * bv[jn];
      }
      __syncthreads();
    }
    if (OUT == 0) {
      // l-sum NL_p = sum_l A_l R_(p,l) over this block's rows, 32 rows at a
      // time: the accumulators go to shared memory (the V and G chunks, free
      // now), then each thread adds, for the (point, p) items it owns, the
      // rows (p, p + d) and (p - d, p) of the diagonals d the 32 rows cover
      // (rows are ordered by diagonal; row (p, p + d) is dstart(d) + p).
      R* Ds = Vs;  // [32][TP]
      static_assert(KC * (TP + TR) >= 32 * TP, "the row chunk fits in the V and G chunks");
#pragma unroll
      for (int c = 0; c < TR / 32; ++c) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int i = 0; i < TM; ++i) Ds[(tx + 16 * h) * TP + ty * TM + i] = acc[i][2 * c + h];
        __syncthreads();
        const int r0 = rb + 32 * c;
        if (r0 < a.rows) {
          const int r1 = min(r0 + 32, a.rows) - 1;
          const int2 first = a.rowpl[r0], last = a.rowpl[r1];
          const int d_lo = first.y - first.x, d_hi = last.y - last.x;
          for (int item = tid; item < N * TP; item += 256) {
            const int p = item / TP, qq = item - p * TP;
            cplx<R> v = Ns[item];
            for (int d = d_lo; d <= d_hi; ++d) {
              const int ds = d * N - d * (d - 1) / 2;
              if (p + d < N) {
                const int rr = ds + p;
                if (rr >= r0 && rr <= r1) {
                  const R x = Ds[(rr - r0) * TP + qq];
                  const cplx<R> al = As[(p + d) * TP + qq];
                  v.x += al.x * x;
                  v.y += al.y * x;
                }
              }
              if (d > 0 && p >= d) {
                const int rr = ds + p - d;
                if (rr >= r0 && rr <= r1) {
                  const R x = Ds[(rr - r0) * TP + qq];
                  const cplx<R> al = As[(p - d) * TP + qq];
                  v.x += al.x * x;
                  v.y += al.y * x;
                }
              }
            }
            Ns[item] = v;
          }
        }
        __syncthreads();
      }
    } else if (OUT == 2) {
      // complex l-sum: row rr = 2 (p N + l) + c holds Re (c = 0) or Im
      // (c = 1) of R_pl; 32 rows at a time through shared memory, each
      // (point, p) item adding the rows of its p in increasing order
      R* Ds = Vs;  // [32][TP]
      static_assert(KC * (TP + TR) >= 32 * TP, "the row chunk fits in the V and G chunks");
#pragma unroll
      for (int c = 0; c < TR / 32; ++c) {
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int i = 0; i < TM; ++i) Ds[(tx + 16 * h) * TP + ty * TM + i] = acc[i][2 * c + h];
        __syncthreads();
        const int r0 = rb + 32 * c;
        if (r0 < a.rows) {
          const int r1 = min(r0 + 32, a.rows) - 1;
          for (int item = tid; item < N * TP; item += 256) {
            const int p = item / TP, qq = item - p * TP;
            const int lo = max(r0, 2 * p * N), hi = min(r1, 2 * p * N + 2 * N - 1);
            if (lo > hi) continue;
            cplx<R> v = Ns[item];
            for (int rr = lo; rr <= hi; ++rr) {
              const R x = Ds[(rr - r0) * TP + qq];
              const cplx<R> al = As[((rr >> 1) - p * N) * TP + qq];
              if (rr & 1) {  // i Im(R_pl) A_l
                v.x -= al.y * x;
                v.y += al.x * x;
              } else {
                v.x += al.x * x;
                v.y += al.y * x;
              }
            }
            Ns[item] = v;
          }
        }
        __syncthreads();
      }
    } else {
      // rows of Z: [M+1][cnt][n]
      bool vec = false;
      if constexpr (sizeof(R) == 4 && TM % 4 == 0) {
        // the tile lies in one substep: each thread writes its TM
        // consecutive points of a row as 16-byte vectors
        vec = pt0 / n == (pt0 + TP - 1) / n && pt0 + TP <= npts;
        if (vec) {
          const size_t j = pt0 / n, t0 = pt0 - j * n + ty * TM;
          R* z = a.Zout + (j * (size_t)a.cnt) * n + t0;
#pragma unroll
          for (int jn = 0; jn < TN; ++jn) {
            const int r = rb + tx + 16 * jn;
            if (r >= a.rows) continue;
#pragma unroll
            for (int i = 0; i < TM; i += 4)
              *reinterpret_cast<float4*>(z + (size_t)r * n + i) =
                  make_float4(acc[i][jn], acc[i + 1][jn], acc[i + 2][jn], acc[i + 3][jn]);
          }
        }
      }
      if (!vec) {
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const size_t pt = pt0 + ty * TM + i;
          if (pt >= npts) continue;
          const size_t j = pt / n, t = pt - j * n;
          if (skip(pt)) continue;
          R* z = a.Zout + (j * (size_t)a.cnt) * n + t;
#pragma unroll
          for (int jn = 0; jn < TN; ++jn) {
            const int r = rb + tx + 16 * jn;
            if (r < a.rows) z[(size_t)r * n] = acc[i][jn];
          }
        }
      }
    }
  }
  if (OUT == 1) return;
  __syncthreads();
  for (int i = tid; i < N * TP; i += 256) {
    const int p = i / TP, qq = i - p * TP;
    const size_t pt = pt0 + qq;
    if (pt >= npts) continue;
    const size_t j = pt / n, t = pt - j * n;
    if (skip(pt)) continue;
    a.NL[(j * N + p) * n + t] = Ns[i];
  }
}

}  // namespace gm
