// One-block, shared-memory Stockham auto-sort FFT of length n = 2^k
// (16 <= n <= 16384): one leading radix-2/4/8 pass when log2 n is not a
// multiple of 4, then radix-16 passes; with 32 elements per thread, 8192
// points take a leading radix-32 pass and two radix-16 passes, 16384 points
// two radix-32 passes and a radix-16 one.
//
// Formulation: the radix-R Stockham iteration of Govindaraju et al.
// ("High performance discrete Fourier transforms on graphics processors",
// SC 2008).  A pass with sub-transform size Ns reads x[j + r n/R], applies
// the twiddles exp(DIR 2 pi i r (j mod Ns) / (Ns R)), does an R-point DFT in
// registers and writes y[(j/Ns) Ns R + (j mod Ns) + r Ns].
//
// DIR = +1 computes X_q = sum_k x_k exp(+2 pi i q k / n), DIR = -1 the
// conjugate kernel; neither is scaled.  The first pass reads through a caller
// functor (fusing whatever produces the input), the last pass writes through
// another (fusing whatever consumes the output); both see natural indices and
// their global accesses are coalesced.  Each thread holds EPT elements; the
// block must have exactly n / EPT threads.
//
// Shared memory: n + n/16 elements (one padding slot per 16 removes the
// stride-16 bank pattern of the Ns = 1 radix-16 pass; the radix-32 leading
// pass keeps a 4-way pattern on its stores, which measured cheaper than a
// padding of one slot per 32 for the other passes).  The functors may read
// or write that same shared buffer (by pad16 of the natural index): every
// pass separates its reads from its writes with a barrier.
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace gm {

__host__ __device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int fft_smem_elems(int n) { return n + (n >> 4); }

// Entries of the radix-16 pass tables of an n-point transform (the passes
// after the leading radix-2/4/8 pass with Ns > 1: 15 Ns each; fewer than n),
// followed for n = 16384 by the table of the radix-32 pass with Ns = 32 of
// the 32 x 32 x 16 schedule (31 x 32 entries, [r-1][k]).
__host__ __device__ inline int fft_pass_table_len(int n) {
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  int Ns = 1 << (logn & 3), len = 0;
  for (; Ns < n; Ns <<= 4)
    if (Ns > 1) len += 15 * Ns;
  return logn == 14 ? len + 31 * 32 : len;
}

template <typename R, int DIR, int RAD> struct Dft;

template <typename R, int DIR> struct Dft<R, DIR, 2> {
  __device__ __forceinline__ static void run(cplx<R>* v) {
    cplx<R> a = v[0], b = v[1];
    v[0] = cadd<R>(a, b);
    v[1] = csub<R>(a, b);
  }
};

template <typename R, int DIR> struct Dft<R, DIR, 4> {
  __device__ __forceinline__ static void run(cplx<R>* v) {
    cplx<R> s02 = cadd<R>(v[0], v[2]), d02 = csub<R>(v[0], v[2]);
    cplx<R> s13 = cadd<R>(v[1], v[3]), d13 = mul_i<R, DIR>(csub<R>(v[1], v[3]));
    v[0] = cadd<R>(s02, s13);
    v[2] = csub<R>(s02, s13);
    v[1] = cadd<R>(d02, d13);
    v[3] = csub<R>(d02, d13);
  }
};

// a * exp(DIR 2 pi i m / 8), m = 0..3
template <typename R, int DIR, int m> __device__ __forceinline__ cplx<R> w8(cplx<R> a) {
  const R h = (R)0.70710678118654752440;
  if (m == 0) return a;
  if (m == 2) return mul_i<R, DIR>(a);
  if (m == 1)  // (1 + DIR i) / sqrt 2
    return DIR > 0 ? mk<R>((a.x - a.y) * h, (a.x + a.y) * h) : mk<R>((a.x + a.y) * h, (a.y - a.x) * h);
  // m == 3: (-1 + DIR i) / sqrt 2
  return DIR > 0 ? mk<R>((-a.x - a.y) * h, (a.x - a.y) * h) : mk<R>((a.y - a.x) * h, (-a.x - a.y) * h);
}

template <typename R, int DIR> struct Dft<R, DIR, 8> {
  // 8 = 2 x 4: X[k1 + 2 k2] = sum_n2 W4^{n2 k2} W8^{n2 k1} sum_n1 x[4 n1 + n2] W2^{n1 k1}
  __device__ __forceinline__ static void run(cplx<R>* v) {
    cplx<R> y0[4], y1[4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      y0[n2] = cadd<R>(v[n2], v[n2 + 4]);
      y1[n2] = csub<R>(v[n2], v[n2 + 4]);
    }
    y1[1] = w8<R, DIR, 1>(y1[1]);
    y1[2] = w8<R, DIR, 2>(y1[2]);
    y1[3] = w8<R, DIR, 3>(y1[3]);
    Dft<R, DIR, 4>::run(y0);
    Dft<R, DIR, 4>::run(y1);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) {
      v[2 * k2] = y0[k2];
      v[2 * k2 + 1] = y1[k2];
    }
  }
};

// exp(DIR 2 pi i m / 16), m = 0..15, from the first-octant values
template <typename R, int DIR> __device__ __forceinline__ cplx<R> w16(int m) {
  const R c0 = (R)1.0, c1 = (R)0.92387953251128675613, c2 = (R)0.70710678118654752440,
          c3 = (R)0.38268343236508977173;
  R cs, sn;
  switch (m & 3) {
    case 0: cs = c0; sn = (R)0; break;
    case 1: cs = c1; sn = c3; break;
    case 2: cs = c2; sn = c2; break;
    default: cs = c3; sn = c1; break;
  }
  R x, y;
  switch ((m >> 2) & 3) {
    case 0: x = cs; y = sn; break;
    case 1: x = -sn; y = cs; break;
    case 2: x = -cs; y = -sn; break;
    default: x = sn; y = -cs; break;
  }
  return mk<R>(x, DIR > 0 ? y : -y);
}

template <typename R, int DIR> struct Dft<R, DIR, 16> {
  // 16 = 4 x 4: X[k1 + 4 k2] = sum_n2 W4^{n2 k2} [W16^{n2 k1} sum_n1 x[4 n1 + n2] W4^{n1 k1}]
  __device__ __forceinline__ static void run(cplx<R>* v) {
    cplx<R> y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[4 * n1 + n2];
      Dft<R, DIR, 4>::run(y[n2]);
    }
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) {
        const int m = n2 * k1;
        if (m == 4) y[n2][k1] = mul_i<R, DIR>(y[n2][k1]);
        else if (m == 2) y[n2][k1] = w8<R, DIR, 1>(y[n2][k1]);
        else if (m == 6) y[n2][k1] = w8<R, DIR, 3>(y[n2][k1]);
        else y[n2][k1] = cmul<R>(y[n2][k1], w16<R, DIR>(m));
      }
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cplx<R> t[4];
#pragma unroll
      for (int n2 = 0; n2 < 4; ++n2) t[n2] = y[n2][k1];
      Dft<R, DIR, 4>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
  }
};

// exp(DIR 2 pi i m / 32) for odd m = 1..15 (the even ones are w16(m/2))
template <typename R, int DIR, int m> __device__ __forceinline__ cplx<R> w32odd() {
  const R c1 = (R)0.98078528040323044913, s1 = (R)0.19509032201612826785, c3 = (R)0.83146961230254523708,
          s3 = (R)0.55557023301960222474;
  R x, y;
  switch (m) {
    case 1: x = c1; y = s1; break;
    case 3: x = c3; y = s3; break;
    case 5: x = s3; y = c3; break;
    case 7: x = s1; y = c1; break;
    case 9: x = -s1; y = c1; break;
    case 11: x = -s3; y = c3; break;
    case 13: x = -c3; y = s3; break;
    default: x = -c1; y = s1; break;  // 15
  }
  return mk<R>(x, DIR > 0 ? y : -y);
}

template <typename R, int DIR> struct Dft<R, DIR, 32> {
  // 32 = 2 x 16: X[2 k2 + k1] = sum_n2 W16^{n2 k2} [W32^{n2 k1} (x[n2] + (-1)^k1 x[n2 + 16])]
  template <int n2>
  __device__ __forceinline__ static cplx<R> tw32(cplx<R> a) {
    if constexpr (n2 == 0) return a;
    else if constexpr (n2 == 8) return mul_i<R, DIR>(a);
    else if constexpr (n2 == 4) return w8<R, DIR, 1>(a);
    else if constexpr (n2 == 12) return w8<R, DIR, 3>(a);
    else if constexpr (n2 % 2 == 0) return cmul<R>(a, w16<R, DIR>(n2 / 2));
    else return cmul<R>(a, w32odd<R, DIR, n2>());
  }
  template <int n2>
  __device__ __forceinline__ static void first(cplx<R>* v, cplx<R>* y0, cplx<R>* y1) {
    if constexpr (n2 < 16) {
      y0[n2] = cadd<R>(v[n2], v[n2 + 16]);
      y1[n2] = tw32<n2>(csub<R>(v[n2], v[n2 + 16]));
      first<n2 + 1>(v, y0, y1);
    }
  }
  __device__ __forceinline__ static void run(cplx<R>* v) {
    cplx<R> y0[16], y1[16];
    first<0>(v, y0, y1);
    Dft<R, DIR, 16>::run(y0);
    Dft<R, DIR, 16>::run(y1);
#pragma unroll
    for (int k2 = 0; k2 < 16; ++k2) {
      v[2 * k2] = y0[k2];
      v[2 * k2 + 1] = y1[k2];
    }
  }
};

// One radix-RAD pass.  Twiddles exp(DIR 2 pi i r k / (RAD Ns)) of the
// butterfly at k = j mod Ns: for a radix-16 pass with a per-pass table
// (tab[(r-1) Ns + k], r = 1..15), read from it after the barrier; otherwise
// from tw[m] = exp(-2 pi i m / n) (W, W^2, W^4, W^8 for radix 16, the rest
// by at most three products), issued before the data reads so that their
// latency overlaps them and the barrier.  The table form measured ~1.4x the
// throughput of the product form (fewer instructions, no registers held
// across the barrier).
template <typename R, int DIR, int RAD, int EPT, bool FIRST, bool LAST, bool TAB, class Load, class Store>
__device__ __forceinline__ void fft_pass(cplx<R>* sm, int n, int Ns, const cplx<R>* __restrict__ tw, int tws,
                                         const cplx<R>* __restrict__ tab, const Load& load, const Store& store) {
  static_assert(RAD != 32 || (!LAST && (FIRST || TAB)), "a radix-32 pass leads (Ns = 1) or reads a table");
  constexpr int B = EPT / RAD;  // butterflies per thread
  constexpr int NW = RAD == 16 ? 4 : (RAD == 32 ? 1 : RAD - 1);  // table reads per butterfly
  const int T = blockDim.x;
  const int stride = n / RAD;
  constexpr bool use_tab = (RAD == 16 || RAD == 32) && TAB;
  cplx<R> wt[B][NW];
  if (RAD != 32 && Ns > 1 && !use_tab) {
#pragma unroll
    for (int b = 0; b < B; ++b) {
      const int j = threadIdx.x + b * T;
      const int step = (j & (Ns - 1)) * (n / (Ns * RAD)) * tws;
      if (RAD == 16) {
        wt[b][0] = tw[step];
        wt[b][1] = tw[2 * step];
        wt[b][2] = tw[4 * step];
        wt[b][3] = tw[8 * step];
      } else {
#pragma unroll
        for (int r = 1; r < (RAD == 32 ? 2 : RAD); ++r) wt[b][r - 1] = tw[r * step];
      }
    }
  }
  cplx<R> v[B][RAD];
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = threadIdx.x + b * T;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int idx = j + r * stride;
      v[b][r] = FIRST ? load(idx) : sm[pad16(idx)];
    }
  }
  __syncthreads();  // every read of this pass precedes every write
#pragma unroll
  for (int b = 0; b < B; ++b) {
    const int j = threadIdx.x + b * T;
    const int k = j & (Ns - 1);
    if (Ns > 1 && use_tab) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        cplx<R> x = tab[(r - 1) * Ns + k];
        if (DIR > 0) x.y = -x.y;
        v[b][r] = cmul<R>(v[b][r], x);
      }
    } else if (RAD != 32 && Ns > 1) {
      cplx<R> w[RAD];
      if (RAD == 16) {
        // W^r for r = 1..15 from W, W^2, W^4, W^8 with at most three
        // products each (error <= 4 ulp)
        w[1] = wt[b][0];
        w[2] = wt[b][1];
        w[4] = wt[b][2];
        w[8] = wt[b][3];
        w[3] = cmul<R>(w[1], w[2]);
        w[5] = cmul<R>(w[1], w[4]);
        w[6] = cmul<R>(w[2], w[4]);
        w[7] = cmul<R>(w[3], w[4]);
#pragma unroll
        for (int r = 9; r < 16; ++r) w[r] = cmul<R>(w[r - 8], w[8]);
      } else {
#pragma unroll
        for (int r = 1; r < (RAD == 32 ? 1 : RAD); ++r) w[r] = wt[b][r - 1];
      }
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        cplx<R> x = w[r];
        if (DIR > 0) x.y = -x.y;
        v[b][r] = cmul<R>(v[b][r], x);
      }
    }
    Dft<R, DIR, RAD>::run(v[b]);
    const int base = (j - k) * RAD + k;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int idx = base + r * Ns;
      if (LAST) store(idx, v[b][r]);
      else sm[pad16(idx)] = v[b][r];
    }
  }
  if (!LAST) __syncthreads();
}

// Full transform: load(i) gives input element i (natural order), store(i, x)
// takes output element i.  tw is the table exp(-2 pi i m / (n tws)); tws > 1
// uses every tws-th entry of a longer table.  With TAB (tws == 1) the table
// must be followed by the radix-16 pass tables of n: tw[n + ...].
// Starts with a barrier, so the buffer may have been used just before by the
// same block.
template <typename R, int DIR, int EPT, bool TAB, class Load, class Store>
__device__ __forceinline__ void fft_block(cplx<R>* sm, int n, const cplx<R>* __restrict__ tw, int tws,
                                          const Load& load, const Store& store) {
  __syncthreads();
  const int logn = 31 - __clz(n);
  const int lead = logn & 3;
  const int passes = (logn >> 2) + (lead ? 1 : 0);
  auto no_load = [](int) { return mk<R>(0, 0); };
  auto no_store = [](int, cplx<R>) {};
  const cplx<R>* tabs = TAB ? tw + n : nullptr;
  const cplx<R>* none = nullptr;
  int Ns = 1, p = 0;
  int off = 0;  // the current pass's table in tabs
  if constexpr (EPT == 32) if (logn == 13) {
    // 8192 = 32 x 16 x 16: a radix-32 leading pass (no twiddles) in place of
    // the radix-2 one and the first radix-16 pass; the radix-16 passes that
    // follow (Ns = 32, 512) use the tables of the radix-2 schedule, past
    // its Ns = 2 table
    fft_pass<R, DIR, 32, EPT, true, false, false>(sm, n, Ns, tw, tws, none, load, no_store);
    Ns = 32;
    off = 15 * 2;
    const cplx<R>* tab = tabs ? tabs + off : nullptr;
    fft_pass<R, DIR, 16, EPT, false, false, TAB>(sm, n, Ns, tw, tws, tab, no_load, no_store);
    off += 15 * Ns;
    Ns <<= 4;
    tab = tabs ? tabs + off : nullptr;
    fft_pass<R, DIR, 16, EPT, false, true, TAB>(sm, n, Ns, tw, tws, tab, no_load, store);
    return;
  }
  if constexpr (EPT == 32 && TAB) if (logn == 14 && tws == 1) {
    // 16384 = 32 x 32 x 16: radix-32 (Ns = 1, no twiddles), radix-32 (Ns =
    // 32, its own table after the radix-16 ones), radix-16 (Ns = 1024, the
    // table of the radix-4 schedule's last pass)
    fft_pass<R, DIR, 32, EPT, true, false, false>(sm, n, Ns, tw, tws, none, load, no_store);
    Ns = 32;
    fft_pass<R, DIR, 32, EPT, false, false, TAB>(sm, n, Ns, tw, tws, tabs + (fft_pass_table_len(n) - 31 * 32),
                                                 no_load, no_store);
    Ns = 1024;
    fft_pass<R, DIR, 16, EPT, false, true, TAB>(sm, n, Ns, tw, tws, tabs + 15 * 4 + 15 * 64, no_load, store);
    return;
  }
  if (lead) {
    const bool last = (passes == 1);
    if (lead == 1) {
      if (last) fft_pass<R, DIR, 2, EPT, true, true, false>(sm, n, Ns, tw, tws, none, load, store);
      else fft_pass<R, DIR, 2, EPT, true, false, false>(sm, n, Ns, tw, tws, none, load, no_store);
    } else if (lead == 2) {
      if (last) fft_pass<R, DIR, 4, EPT, true, true, false>(sm, n, Ns, tw, tws, none, load, store);
      else fft_pass<R, DIR, 4, EPT, true, false, false>(sm, n, Ns, tw, tws, none, load, no_store);
    } else {
      if (last) fft_pass<R, DIR, 8, EPT, true, true, false>(sm, n, Ns, tw, tws, none, load, store);
      else fft_pass<R, DIR, 8, EPT, true, false, false>(sm, n, Ns, tw, tws, none, load, no_store);
    }
    Ns <<= lead;
    ++p;
  }
  for (; p < passes; ++p) {
    const bool first = (p == 0), last = (p == passes - 1);
    const cplx<R>* tab = tabs ? tabs + off : nullptr;
    if (first && last) fft_pass<R, DIR, 16, EPT, true, true, TAB>(sm, n, Ns, tw, tws, tab, load, store);
    else if (first) fft_pass<R, DIR, 16, EPT, true, false, TAB>(sm, n, Ns, tw, tws, tab, load, no_store);
    else if (last) fft_pass<R, DIR, 16, EPT, false, true, TAB>(sm, n, Ns, tw, tws, tab, no_load, store);
    else fft_pass<R, DIR, 16, EPT, false, false, TAB>(sm, n, Ns, tw, tws, tab, no_load, no_store);
    if (Ns > 1) off += 15 * Ns;
    Ns <<= 4;
  }
}

template <typename R, int DIR, int EPT, class Load, class Store>
__device__ __forceinline__ void fft_block(cplx<R>* sm, int n, const cplx<R>* __restrict__ tw, const Load& load,
                                          const Store& store) {
  fft_block<R, DIR, EPT, true>(sm, n, tw, 1, load, store);
}

// Output-residue split of an n-point transform over S blocks (radix-S
// decimation in frequency): block s (0 <= s < S) computes X[S k + s],
// k < n/S, as the (n/S)-point transform of
//   y_s[t] = W^{DIR t s} sum_{u<S} x[t + u n/S] W_S^{DIR u s},  W = exp(2 pi i / n).
// x_at(u, t) supplies x[t + u n/S].
template <typename R, int DIR, int S, class XAt>
__device__ __forceinline__ cplx<R> dif_input(int s, int t, const cplx<R>* __restrict__ tw, const XAt& x_at) {
  cplx<R> acc = x_at(0, t);
  if (S == 2) {
    const cplx<R> b = x_at(1, t);
    acc = s ? csub<R>(acc, b) : cadd<R>(acc, b);
  } else if (S == 4) {  // W_4^{DIR u s} = (DIR i)^{u s}
    const cplx<R> b = x_at(1, t), c = x_at(2, t), d = x_at(3, t);
    const cplx<R> ac = cadd<R>(acc, c), amc = csub<R>(acc, c);
    const cplx<R> bd = cadd<R>(b, d), ibmd = mul_i<R, DIR>(csub<R>(b, d));
    switch (s) {
      case 0: acc = cadd<R>(ac, bd); break;
      case 1: acc = cadd<R>(amc, ibmd); break;
      case 2: acc = csub<R>(ac, bd); break;
      default: acc = csub<R>(amc, ibmd); break;
    }
  }
  if (s) {
    cplx<R> w = tw[t * s];
    if (DIR > 0) w.y = -w.y;
    acc = cmul<R>(acc, w);
  }
  return acc;
}

// An n-point transform spread over the S blocks of a thread-block cluster
// (S = 2 or 4).  Block s reads only the input slice t in [s n/S, (s+1) n/S)
// (load(t), into xbuf), forms its residue-s input of the radix-S first stage
// from all slices through distributed shared memory, transforms n/S points
// locally, and finally gathers the output slice q in [s n/S, (s+1) n/S)
// (X[q] = Y_{q mod S}[q div S]) from the blocks' results, handing each to
// store(q).  xbuf: n/S elements; sm: fft_smem_elems(n/S) elements.  Every
// block of the cluster must call it.
template <typename R, int DIR, int EPT, int S, class Load, class Store>
__device__ __forceinline__ void fft_cluster(cplx<R>* xbuf, cplx<R>* sm, int n, const cplx<R>* __restrict__ tw,
                                            const Load& load, const Store& store) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int s = (int)cluster.block_rank();
  const int np = n / S;
  for (int t = threadIdx.x; t < np; t += blockDim.x) xbuf[t] = load(s * np + t);
  cluster.sync();  // every slice loaded
  const cplx<R>* xs[S];
  const cplx<R>* ys[S];
#pragma unroll
  for (int u = 0; u < S; ++u) {
    xs[u] = cluster.map_shared_rank(xbuf, u);
    ys[u] = cluster.map_shared_rank(sm, u);
  }
  auto x_at = [&](int u, int t) { return xs[u][t]; };
  auto first = [&](int t) { return dif_input<R, DIR, S>(s, t, tw, x_at); };
  auto keep = [&](int k, cplx<R> v) { sm[pad16(k)] = v; };
  fft_block<R, DIR, EPT, false>(sm, np, tw, S, first, keep);
  cluster.sync();  // every block's Y_s complete
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const int q = s * np + i;
    store(q, ys[q % S][pad16(q / S)]);
  }
  cluster.sync();  // partners are done reading this block's buffers
}

}  // namespace gm
