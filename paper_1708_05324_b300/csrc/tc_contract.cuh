// Coupling contraction on the 5th-generation tensor cores (mixed precision,
// BF16 or FP16 operands).
//
// Per point (j, t) of the MPA iteration (Eq. 1 bracket after the symmetry
// rewrite):  R_r = sum_k G[r][k] V_k   (rows r = (p <= l), k over pair terms),
//            NL_p = sum_l A_l R_pl.
// Over a tile of 128 points and a block of NB rows this is the GEMM
//   D[128 x NB] = V[128 x K] . G[NB x K]^T
// with V and G split into 16-bit hi + lo parts; D accumulates hi.hi + lo.hi +
// hi.lo in FP32 in TMEM (lo.lo lies below the FP32 rounding of the result).
// BF16 needs no scaling.  FP16 (11-bit significands, range 2^-24 .. 65504)
// takes power-of-two scales: G by 2^eG (its largest entry below 2^14, set at
// context creation) and V by 2^eV from a bound on |V|: |U_mn(t)| <=
// sum_p |A_p(t)|^2 <= sum_t sum_p |A_p(t)|^2 = (1/Nt) sum_w |psi0|^2 and
// |h_R * U| <= dt sum |h_R| max |U| < 2 max |U|, so 2^eV (2 x bound) < 2^14,
// the bound taken anew at the start of every long step (an energy that a
// gain raises along the fiber raises it too).  The epilogue undoes both
// exactly (a power of two).
// Points are the MMA's M dimension, so after tcgen05.ld each epilogue thread
// holds R_r(t) for its own point t and forms the l-sum in registers, with the
// row -> (p, l) map resolved at compile time.
//
// The same kernel with OUT 1 stores the accumulator rows (times the inverse
// FP16 scales) as Z = W U, the first GEMM of the low-rank coupling.
//
// Roles (192 threads): warp 0 issues TMA copies of K chunks (32 wide) of V
// and G into a ring of stages; warp 1 issues tcgen05.mma from the ring into
// one of two TMEM accumulators; warps 2-5 drain an accumulator (tcgen05.ld)
// while the MMAs of the next work item run.  A work item is (point tile, row
// block); NL of a tile is written after its last row block.
//
// Row blocks of NB >= 32 rows run on CTA pairs (2-CTA clusters, cta_group::2):
// one MMA of M = 256 points (a 128-point tile in each CTA) by NB rows, the
// first NB/2 coupling rows of each K chunk in the shared memory of CTA 0 and
// the other NB/2 in CTA 1, so each CTA loads its own V tile and half of the
// coupling chunk (plain TMA loads, no multicast) and the MMA reads both
// halves.  Per SM and K chunk that is 16 KB of V and NB/2 rows of G instead of
// NB rows, and the tensor cores read half of B from each SM's shared memory.
// CTA 0 issues the MMAs; the copies of both CTAs count on CTA 0's stage
// barrier; CTA 0's MMA commits release the stage in both CTAs and announce a
// finished accumulator to both; each CTA's epilogue drains its own TMEM
// (its tile's 128 points) and reports to CTA 0 by a remote arrival.
// Row blocks below 32 rows, and the GEMM that forms U in the kernel, run on
// single CTAs (cta_group::1).
//
// Operand layout (both K-major, no swizzle): core matrices of 8 rows x 8
// elements (16 bytes).  V is stored [k/8][point][8]; in shared memory a K
// chunk of 128 points is [4][128][8], so core matrices adjacent along K are
// 128*16 bytes apart (LBO) and along the points 128 bytes (SBO).  The
// coupling operand is stored row-grouped, [row/8][k/8][8][8]; a K chunk of
// NB/CL rows is [NB/(8 CL)][4][8][8] in shared memory (LBO 128 bytes, SBO
// 512), one contiguous box of the row-grouped layout.  The tensor maps give
// both operands rows of 256 elements (512 contiguous bytes: 32 points of a
// K plane of V, or the K chunk of one 8-row group of the coupling), so the
// TMA moves each box in 512-byte pieces; with the 16-byte rows of the core
// matrices as map rows, the copies ran at about 14 bytes per clock and SM
// and held both GEMMs to about a third of the tensor-core rate.
//
// Every mbarrier wait is bounded in time (TcArgs::wait_ns); on a timeout the
// kernel records an error in *err and every role stops issuing work.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace gm {

constexpr int TC_PTS = 128;  // MMA M: points per tile
constexpr int TC_KC = 32;    // K chunk per pipeline stage

struct TcArgs {
  int KKp;           // K padded to a multiple of TC_KC
  int f16;           // operands FP16 (else BF16)
  int eG;            // FP16: G scaled by 2^eG
  int eVoff;         // FP16: V scaled by 2^(eV - eVoff), eV from the energy bound
  int n, M;          // samples, substeps (tiles cover j = 0..M)
  const float2* A;   // [M+1][N][n]
  float2* NL;        // [M+1][N][n]
  unsigned* err;     // set to 1 if a wait times out
  int nrb;           // OUT 1: row blocks
  float* Zout;       // OUT 1: D rows [M+1][zrows][n]
  int zrows;         // OUT 1: rows stored (the rest is padding)
  int nmodes, K;     // U formed in the kernel: modes of A, 4 x 4 blocks of U
  int B;             // slots of a packed launch (1: one propagation)
  const int2* pairs; // U formed in the kernel: first (m, n) of each 4 x 4 block
  unsigned long long wait_ns;  // limit of every mbarrier wait [ns]
  int stall;         // test hook: the MMA issuer waits on a barrier nothing completes,
                     // 1: in single-CTA GEMMs, 2: in every GEMM
};

__host__ __device__ constexpr int tc_row_block(int P) { return P <= 256 ? (P + 15) / 16 * 16 : 256; }

// CTAs per MMA of the GEMM with row blocks of NB rows (NB a multiple of 16):
// a CTA pair from 32 rows (each CTA holds NB/2 rows, whole 8-row groups),
// else one CTA.
__host__ __device__ constexpr int tc_cluster(int NB) { return NB >= 32 ? 2 : 1; }

// FP16 scale exponent of V: 2^eV (2 x the bound on |V|) < 2^14; the bound
// is (1/Nt) sum_w |psi0|^2 at the start of the current long step (summed by
// the previous long step's advance; at the first, by the input sums), so it
// follows an energy that grows along the fiber (gain); within one long step
// the 4x headroom below the FP16 maximum covers the growth.
__device__ __forceinline__ int f16_v_exp(const LoopState* ls, int n, int B = 1) {
  // a packed launch takes the largest bound over its occupied slots
  double b = 0.0;
  for (int k = 0; k < B; ++k)
    if (!ls[k].idle) b = fmax(b, (ls[k].spec_v > 0.0 ? ls[k].spec_v : ls[k].spec[0]) / (double)n);
  if (!(b > 0.0) || !isfinite(b)) b = 1.0;
  int e;
  frexp(2.0 * b, &e);  // 2 b < 2^e
  return 14 - e;
}

// Operand types of the hi/lo split: OP 0 BF16, 1 FP16, 2 TF32 (FP32 words
// with the low 13 mantissa bits cleared by rounding to nearest, ties away).
template <int OP> struct Split;
template <> struct Split<0> {
  using T = __nv_bfloat16;
  static constexpr int EPC = 8;
  __device__ static T rn(float x) { return __float2bfloat16_rn(x); }
  __device__ static float back(T h) { return __bfloat162float(h); }
};
template <> struct Split<1> {
  using T = __half;
  static constexpr int EPC = 8;
  __device__ static T rn(float x) { return __float2half_rn(x); }
  __device__ static float back(T h) { return __half2float(h); }
};
template <> struct Split<2> {
  using T = float;
  static constexpr int EPC = 4;
  __device__ static T rn(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
  __device__ static float back(T h) { return h; }
};

// ES: operand element bytes, 2 (BF16 / FP16) or 4 (TF32); a core-matrix row
// of 16 bytes holds EPC = 16 / ES elements.
// FU: the store epilogue (OUT 1) with 16-bit operands forms its V operand,
// the pair products U of A, in the kernel: eight more warps compute each K
// chunk of U for the CTA's tile from A staged in shared memory and write it
// to the stage as hi/lo (no packed U in HBM).  The columns of U come in 4 x 4
// blocks of (m, n) (m-block <= n-block; the entries that are not pairs
// m <= n < N have zero columns in W, which also carries the weights 1 and 2),
// so that a thread forms 16 columns from four A_m and four A_n: half the
// shared-memory reads per column of one column at a time, for 17% more K at
// N = 42 (1056 columns for 903 pairs).  U_FIT_N bounds the modes of A it
// stages (rows up to U_FIT_NP, the ones from N on zero).
// TPW: point tiles per work item and CTA, sharing each stage's coupling chunk
// (TPW MMAs into TPW accumulators): 2 for the store epilogue without FU when
// two stages still fit, else 1.  NBUF: accumulator buffers in TMEM (2 lets
// the epilogue drain one work item while the next one's MMAs run).
constexpr int U_FIT_N = 42, U_FIT_NP = (U_FIT_N + 3) / 4 * 4;
constexpr int U_FIT_BLK = (U_FIT_NP / 4) * (U_FIT_NP / 4 + 1) / 2;  // 4 x 4 blocks of U
constexpr int U_FIT_KKP = (16 * U_FIT_BLK + 31) / 32 * 32;         // 1056 columns
template <int N, int NB, int ES = 2, int OUT = 0>
struct TcShape {
  static constexpr int P = N * (N + 1) / 2;
  static constexpr int NRB = (P + NB - 1) / NB;        // row blocks
  static constexpr int EPC = 16 / ES;                  // elements per core-matrix row
  static constexpr int KSTEPS = TC_KC * ES / 32;       // MMAs of 32 bytes of K per chunk
  static constexpr int V_BYTES = TC_PTS * TC_KC * ES;  // one of hi / lo, one tile
  static constexpr int G_BYTES = NB * TC_KC * ES;      // one of hi / lo, all NB rows
  static constexpr bool FU = OUT == 1 && ES == 2;
  // CTAs per MMA (2: CTA pair); the GEMM that forms U in the kernel runs on
  // single CTAs (measured faster: on a pair every K chunk waits for both
  // CTAs' producers, whose stage hand-over to the MMA-issuing CTA is a
  // cluster-scope release per warp and chunk; 0.30 against 0.20 ms per
  // 42-mode iteration)
  static constexpr int CL = FU ? 1 : tc_cluster(NB);
  static constexpr int G_HALF = G_BYTES / CL;          // this CTA's rows of a chunk (hi or lo)
  static constexpr int UW = FU ? 8 : 0;                // U-producer warps
  // the l-sum epilogue of more than 24 modes runs on two warps per TMEM lane
  // quarter, each forming NL_p for half of the modes (the registers of one
  // point's 2N mode values and 2N accumulators would spill)
  static constexpr bool ESPLIT = OUT == 0 && N > 24;
  static constexpr int EW = ESPLIT ? 8 : 4;            // epilogue warps
  static constexpr int THREADS = 64 + 32 * EW + 32 * UW;
  // A tile ([U_FIT_NP][128] float2) and block table ([KKp/16] int2) of FU
  static constexpr int U_RESERVE = FU ? U_FIT_NP * TC_PTS * 8 + U_FIT_KKP / 16 * 8 : 0;
  static constexpr int TPW = (OUT == 1 && !FU && 2 * 2 * (2 * V_BYTES + G_HALF) <= 200 * 1024) ? 2 : 1;
  static constexpr int STAGE = 2 * (TPW * V_BYTES + G_HALF);
  static constexpr int FIT = (200 * 1024 - U_RESERVE) / STAGE;
  static constexpr int STAGES = FIT < 2 ? 2 : (FIT > 6 ? 6 : FIT);
  static constexpr int ACC_COLS = TPW * NB;            // one accumulator buffer
  static constexpr int NBUF = 2 * ACC_COLS <= 512 ? 2 : 1;
  static constexpr int COLS = NBUF * ACC_COLS;
  static constexpr int TMEM_COLS = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));
  static constexpr size_t SMEM = (size_t)STAGES * STAGE + 1024 + U_RESERVE;
  // TMEM never runs short: with 228 KB of shared memory per SM at most two
  // of these CTAs (of any shape) share an SM, and one that takes more than
  // 256 columns has the SM to itself
  static_assert(SMEM + 1024 > 233472 / 3 && (TMEM_COLS <= 256 || SMEM + 1024 > 233472 / 2),
                "tensor-core GEMM CTAs could share an SM's TMEM beyond its 512 columns");
  // bytes that complete a stage's barrier: both CTAs' copies (V tiles unless
  // FU, and every coupling row of the chunk, hi and lo)
  static constexpr int TX = FU ? 2 * G_BYTES : CL * STAGE;
};

// Row r of the reduced coupling matrix is the pair (p, l), p <= l, in the
// order (0,0), (0,1), ..., (0,N-1), (1,1), ...
template <int N>
struct RowPair {
  __host__ __device__ static constexpr int p_of(int r) {
    int p = 0;
    while (r >= N - p) {
      r -= N - p;
      ++p;
    }
    return p;
  }
  __host__ __device__ static constexpr int l_of(int r) {
    int p = 0;
    while (r >= N - p) {
      r -= N - p;
      ++p;
    }
    return p + r;
  }
};

// NL_p += A_l R_r (and NL_l += A_p R_r) for the rows R .. REND - 1 (compile
// time), into the accumulators of modes LO .. HI - 1 only (nl[p - LO]).
template <int N, int R, int REND, int LO, int HI>
struct LSumH {
  __device__ __forceinline__ static void run(const float* v, const float2* a, float2* nl) {
    if constexpr (R < REND && R < N * (N + 1) / 2) {
      constexpr int p = RowPair<N>::p_of(R), l = RowPair<N>::l_of(R);
      constexpr int i = R % 16;
      if constexpr (p >= LO && p < HI) {
        nl[p - LO].x += a[l].x * v[i];
        nl[p - LO].y += a[l].y * v[i];
      }
      if constexpr (p != l && l >= LO && l < HI) {
        nl[l - LO].x += a[p].x * v[i];
        nl[l - LO].y += a[p].y * v[i];
      }
      LSumH<N, R + 1, REND, LO, HI>::run(v, a, nl);
    }
  }
};

// Whether any of rows R0 .. R0 + 15 adds to a mode in LO .. HI - 1.
template <int N>
__host__ __device__ constexpr bool rows_touch(int R0, int LO, int HI) {
  for (int r = R0; r < R0 + 16 && r < N * (N + 1) / 2; ++r) {
    const int p = RowPair<N>::p_of(r), l = RowPair<N>::l_of(r);
    if ((p >= LO && p < HI) || (l >= LO && l < HI)) return true;
  }
  return false;
}

// The first 16-column chunk from C on of an accumulator holding row block
// RB whose rows add to a mode in LO .. HI - 1 (-1: none).
template <int N>
__host__ __device__ constexpr int next_chunk(int NB, int RB, int C, int LO, int HI) {
  for (int c = C; c < NB && RB * NB + c < N * (N + 1) / 2; c += 16)
    if (rows_touch<N>(RB * NB + c, LO, HI)) return c;
  return -1;
}

// The l-sum of chunk C (its 16 values in r, loaded and waited for) and of
// every later chunk that adds to the modes LO .. HI - 1 (column chunks that
// add to none of them are not read).  Up to 24 modes the next chunk's TMEM
// load is issued before this chunk's sums, so that its latency overlaps
// them; above, the 16 more live registers spill (measured slower at 42
// modes), and each chunk is loaded after the previous one's sums.
template <int N, int NB, int RB, int C, int LO, int HI>
struct DrainP {
  __device__ __forceinline__ static void run(uint32_t taddr, const float2* a, float2* nl, uint32_t (&r)[16]) {
    constexpr int R0 = RB * NB + C;
    constexpr int CN = next_chunk<N>(NB, RB, C + 16, LO, HI);
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
    if constexpr (CN >= 0) {
      uint32_t rn[16];
      if constexpr (N <= 24) {
        tc::tmem_ld16_issue(taddr + CN, rn);
        LSumH<N, R0, R0 + 16, LO, HI>::run(v, a, nl);
      } else {
        LSumH<N, R0, R0 + 16, LO, HI>::run(v, a, nl);
        tc::tmem_ld16_issue(taddr + CN, rn);
      }
      tc::tmem_wait16(rn);
      DrainP<N, NB, RB, CN, LO, HI>::run(taddr, a, nl, rn);
    } else {
      LSumH<N, R0, R0 + 16, LO, HI>::run(v, a, nl);
    }
  }
};

// The l-sum of an accumulator holding row block rb (a runtime value) for the
// modes LO .. HI - 1.
template <int N, int NB, int RB, int LO, int HI>
__device__ __forceinline__ void drain_rb_h(int rb, uint32_t taddr, const float2* a, float2* nl) {
  if constexpr (RB < TcShape<N, NB>::NRB) {
    if (rb == RB) {
      constexpr int C0 = next_chunk<N>(NB, RB, 0, LO, HI);
      if constexpr (C0 >= 0) {
        uint32_t r[16];
        tc::tmem_ld16_issue(taddr + C0, r);
        tc::tmem_wait16(r);
        DrainP<N, NB, RB, C0, LO, HI>::run(taddr, a, nl, r);
      }
    } else {
      drain_rb_h<N, NB, RB + 1, LO, HI>(rb, taddr, a, nl);
    }
  }
}

// The same for every mode.
template <int N, int NB, int RB>
__device__ __forceinline__ void drain_rb(int rb, uint32_t taddr, const float2* a, float2* nl) {
  drain_rb_h<N, NB, RB, 0, N>(rb, taddr, a, nl);
}

// OUT 0: the l-sum epilogue into NL (N modes, compile-time); OUT 1: the
// accumulator rows stored as Z (first GEMM of the low-rank coupling; N is 0).
template <int N, int NB, int OUT, int ES = 2>
__global__ void __launch_bounds__(TcShape<N, NB, ES, OUT>::THREADS, 1) k_tc_contract(const __grid_constant__ CUtensorMap mapVhi,
                                                         const __grid_constant__ CUtensorMap mapVlo,
                                                         const __grid_constant__ CUtensorMap mapGhi,
                                                         const __grid_constant__ CUtensorMap mapGlo, TcArgs a,
                                                         const LoopState* __restrict__ ls) {
  using S = TcShape<N, NB, ES, OUT>;
  constexpr int TPW = S::TPW, NBUF = S::NBUF, CL = S::CL;
  constexpr bool PAIR = CL == 2;
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  unsigned char* smem = tc_smem_raw + ((1024 - (tc::smem_addr(tc_smem_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t full[S::STAGES], empty[S::STAGES], acc_full[2], acc_empty[2], never;
  __shared__ uint32_t tmem_base;
  __shared__ int stop_flag;
  volatile int* stop = &stop_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint64_t wait_ns = a.wait_ns;

  // FU: A tile [nmodes][128] and the column table after the stages
  float2* As = reinterpret_cast<float2*>(smem + (size_t)S::STAGES * S::STAGE);
  int2* Ps = reinterpret_cast<int2*>(As + (S::FU ? U_FIT_NP * TC_PTS : 0));
  const unsigned rank = PAIR ? tc::cluster_ctarank() : 0u;
  const bool leader = rank == 0;
  if (tid == 0) {
    for (int s = 0; s < S::STAGES; ++s) {
      // (used in CTA 0) the TMA producer's arrival, plus one per U warp of each CTA
      tc::mbar_init(&full[s], 1 + CL * S::UW);
      tc::mbar_init(&empty[s], 1);  // one MMA commit releases the stage
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(&acc_full[b], 1);
      tc::mbar_init(&acc_empty[b], S::EW * CL);  // (used in CTA 0) one arrival per epilogue warp of each CTA
    }
    tc::mbar_init(&never, 1);  // nothing arrives on it (the stall test hook)
    tc::fence_mbar_init();
    stop_flag = 0;
  }
  if (warp == 1) tc::tmem_alloc<PAIR>(&tmem_base, S::TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  // the peer's barriers exist before any remote arrival or copy, and its
  // columns are allocated before either CTA gives up the allocation permit
  if (PAIR) tc::cluster_sync();
  tc::fence_after_sync();
  if (warp == 1) tc::tmem_relinquish<PAIR>();
  pdl_enter();
  if (S::FU) {
    // block b of U: the offsets of its first A_m and A_n in the A tile (16
    // bits each); blocks past the last (the K padding) read rows 0, times
    // zero columns of W.  The A rows from nmodes to U_FIT_NP stay zero.
    for (int b = tid; b < a.KKp / 16; b += S::THREADS) {
      int2 e = make_int2(0, 0);
      if (b < a.K) {
        const int2 mn = a.pairs[b];
        e.x = (mn.x * TC_PTS) | ((mn.y * TC_PTS) << 16);
      }
      Ps[b] = e;
    }
    for (int i = a.nmodes * TC_PTS + tid; i < U_FIT_NP * TC_PTS; i += S::THREADS) As[i] = make_float2(0.f, 0.f);
    __syncthreads();
  }
  // shared::cluster addresses of CTA 0's barriers (the MMA issuer's), and of
  // a barrier in CTA `r`
  auto at0 = [&](uint64_t* bar) { return PAIR ? tc::mapa(tc::smem_addr(bar), 0) : tc::smem_addr(bar); };
  auto at = [&](uint64_t* bar, unsigned r) { return PAIR ? tc::mapa(tc::smem_addr(bar), r) : tc::smem_addr(bar); };
  auto fail = [&]() {
    *stop = 1;
    atomicExch(a.err, 1u);
  };
  const uint32_t tmem = tmem_base;
  const int nrb = OUT == 0 ? S::NRB : a.nrb;
  const int n = a.n;
  const int cid = blockIdx.x / CL, ncl = gridDim.x / CL;
  const int ntiles = a.B * (a.M + 1) * (n / TC_PTS);
  const int nitems = (ntiles + TPW * CL - 1) / (TPW * CL);  // work items of CL x TPW tiles
  const int kchunks = a.KKp / TC_KC;
  // this CTA's tiles of work item wi: (wi CL + rank) TPW + h
  auto tile_of = [&](int wi, int h) { return (wi * CL + (int)rank) * TPW + h; };
  // a tile (in one slice: n is a multiple of 128) is skipped when its slice
  // does no work (z0 after the first iteration; empty or converged slots)
  auto live = [&](int tile) {
    if (tile >= ntiles) return false;
    const int slice = tile * TC_PTS / n, b = slice / (a.M + 1), j = slice - b * (a.M + 1);
    return !slice_skipped(ls + b, j);
  };
  // an item runs in both CTAs of a pair if any of its tiles is live
  auto live_item = [&](int wi) {
    bool any = false;
    for (int h = 0; h < TPW * CL; ++h) any = any || live(wi * TPW * CL + h);
    return any;
  };

  if (warp == 0) {
    // ---------------- TMA producer (each CTA loads its own shares) ----------------
    if (lane == 0) {
      int c = 0;
      for (int wi = cid; wi < nitems && !*stop; wi += ncl) {
        if (!live_item(wi)) continue;
        for (int rb = 0; rb < nrb && !*stop; ++rb)
          for (int kc = 0; kc < kchunks; ++kc, ++c) {
            const int s = c % S::STAGES, round = c / S::STAGES;
            if (round > 0 && !tc::mbar_wait(&empty[s], (round - 1) & 1, wait_ns)) {
              fail();
              break;
            }
            unsigned char* st = smem + (size_t)s * S::STAGE;
            if (leader) tc::mbar_arrive_expect_tx(&full[s], S::TX);
            const uint32_t fb = at0(&full[s]);
            const int kq = kc * (TC_KC / S::EPC);  // K coordinate in core-matrix rows
#pragma unroll
            for (int h = 0; h < (S::FU ? 0 : TPW); ++h) {
              // a tile past the end repeats the last one (its result is not stored)
              const int tile = min(tile_of(wi, h), ntiles - 1);
              unsigned char* sv = st + (size_t)h * 2 * S::V_BYTES;
              // the operand map's rows are 256 elements: TC_PTS EPC / 256 of them per tile
              const int vy = tile * (TC_PTS * S::EPC / 256);
              if (PAIR) {
                tc::tma_load_3d_pair(sv, &mapVhi, 0, vy, kq, fb);
                tc::tma_load_3d_pair(sv + S::V_BYTES, &mapVlo, 0, vy, kq, fb);
              } else {
                tc::tma_load_3d(sv, &mapVhi, 0, vy, kq, &full[s]);
                tc::tma_load_3d(sv + S::V_BYTES, &mapVlo, 0, vy, kq, &full[s]);
              }
            }
            // this CTA's rows of the coupling chunk: 8-row groups g0 .. g0 + NB/(8 CL) - 1
            unsigned char* sg = st + (size_t)TPW * 2 * S::V_BYTES;
            const int g0 = rb * (NB / 8) + (int)rank * (NB / 8 / CL);
            // (the coupling map's rows are whole K chunks of an 8-row group)
            if (PAIR) {
              tc::tma_load_3d_pair(sg, &mapGhi, 0, kc, g0, fb);
              tc::tma_load_3d_pair(sg + S::G_HALF, &mapGlo, 0, kc, g0, fb);
            } else {
              tc::tma_load_3d(sg, &mapGhi, 0, kc, g0, &full[s]);
              tc::tma_load_3d(sg + S::G_HALF, &mapGlo, 0, kc, g0, &full[s]);
            }
          }
      }
      // wait for the release of the last stages: after that the MMAs have
      // read this CTA's shared memory for the last time (and every copy
      // into it has landed).  After a failure, give copies in flight time
      // to land before the CTA exits.
      const int first = c > S::STAGES ? c - S::STAGES : 0;
      for (int i = first; i < c && !*stop; ++i)
        if (!tc::mbar_wait(&empty[i % S::STAGES], (i / S::STAGES) & 1, wait_ns)) fail();
      if (*stop) {
        const uint64_t t0 = tc::globaltimer_ns();
        while (tc::globaltimer_ns() - t0 < 200000) __nanosleep(1000);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (CTA 0 of a pair) ----------------
    if (lane == 0 && leader) {
      const uint32_t idesc =
          tc::idesc_mma(TC_PTS * CL, NB, ES == 4 ? tc::FMT_TF32 : (a.f16 ? tc::FMT_F16 : tc::FMT_BF16));
      const uint32_t lboV = TC_PTS * 16, sboV = 128;
      const uint32_t lboG = 128, sboG = (TC_KC / S::EPC) * 128;
      if ((a.stall == 2 || (a.stall == 1 && !PAIR)) && !tc::mbar_wait(&never, 0, wait_ns)) fail();
      int c = 0, w = 0;
      for (int wi = cid; wi < nitems && !*stop; wi += ncl) {
        if (!live_item(wi)) continue;
        for (int rb = 0; rb < nrb && !*stop; ++rb, ++w) {
          const int acc = w % NBUF, use = w / NBUF;
          if (use > 0 && !tc::mbar_wait(&acc_empty[acc], (use - 1) & 1, wait_ns)) {
            fail();
            break;
          }
          tc::fence_after_sync();
          const uint32_t d0 = tmem + (uint32_t)(acc * S::ACC_COLS);
          for (int kc = 0; kc < kchunks; ++kc, ++c) {
            const int s = c % S::STAGES, round = c / S::STAGES;
            if (!tc::mbar_wait(&full[s], round & 1, wait_ns)) {
              fail();
              break;
            }
            tc::fence_after_sync();
            const uint32_t base = tc::smem_addr(smem + (size_t)s * S::STAGE);
            const uint32_t gH = base + TPW * 2 * S::V_BYTES, gL = gH + S::G_HALF;
#pragma unroll
            for (int kk = 0; kk < S::KSTEPS; ++kk) {
              // 32 bytes of K per MMA: two core matrices along K
              const uint32_t oV = (uint32_t)kk * 2 * lboV, oG = (uint32_t)kk * 2 * lboG;
#pragma unroll
              for (int h = 0; h < TPW; ++h) {
                const uint32_t d = d0 + (uint32_t)(h * NB);
                const uint32_t vH = base + h * 2 * S::V_BYTES, vL = vH + S::V_BYTES;
                tc::mma<ES == 4, PAIR>(d, tc::smem_desc(vH + oV, lboV, sboV), tc::smem_desc(gH + oG, lboG, sboG),
                                       idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                tc::mma<ES == 4, PAIR>(d, tc::smem_desc(vL + oV, lboV, sboV), tc::smem_desc(gH + oG, lboG, sboG),
                                       idesc, 1u);
                tc::mma<ES == 4, PAIR>(d, tc::smem_desc(vH + oV, lboV, sboV), tc::smem_desc(gL + oG, lboG, sboG),
                                       idesc, 1u);
              }
            }
            // the stage is free in each CTA once these MMAs have read it
            tc::mma_commit<PAIR>(tc::smem_addr(&empty[s]));
            if (PAIR) tc::mma_commit<PAIR>(at(&empty[s], 1));
          }
          if (*stop) break;
          // accumulator complete (in both CTAs' TMEM)
          tc::mma_commit<PAIR>(tc::smem_addr(&acc_full[acc]));
          if (PAIR) tc::mma_commit<PAIR>(at(&acc_full[acc], 1));
        }
      }
    }
  } else if (S::FU && warp >= 6) {
    // ---------------- U producers: warps 6..13, two threads per point ----------------
    // thread (q, half) writes K columns [16 half, 16 half + 16) of each chunk
    // (the 4 x 4 block 2 kc + half of U) for point q of the tile, as hi + lo
    // in the stage's [4][128][8] layout.  The A tile of the next work item is
    // fetched into registers while the current one's chunks are formed.
    constexpr int UT = 32 * (S::FU ? S::UW : 1);          // U threads
    constexpr int AL = (U_FIT_N * TC_PTS + UT - 1) / UT;  // A values per thread and tile
    const int u = tid - 192, q = u & (TC_PTS - 1), half = u >> 7;
    const int nm = a.nmodes;
    float2 nxt[AL];
    auto fetch = [&](int wi) {
      const int tile = min(tile_of(wi, 0), ntiles - 1);
      const int pt0 = tile * TC_PTS, j = pt0 / n, t0 = pt0 - j * n;
#pragma unroll
      for (int r = 0; r < AL; ++r) {
        const int i = u + r * UT;
        if (i < nm * TC_PTS) {
          const int l = i / TC_PTS, qq = i - l * TC_PTS;
          nxt[r] = a.A[((size_t)j * nm + l) * n + t0 + qq];
        }
      }
    };
    auto next_live = [&](int wi) {
      for (wi += ncl; wi < nitems && !live_item(wi); wi += ncl) {
      }
      return wi;
    };
    // FP16: U scaled by 2^eV (BF16: 1); the weights are in W
    const float sc = a.f16 ? ldexpf(1.0f, f16_v_exp(ls, a.n, a.B)) : 1.0f;
    // the 16 values Re(A_m conj A_n) of block b for this point: x[4 i + j]
    // from A_{m0+i} and A_{n0+j}
    auto u16 = [&](int b, float* x) {
      const int2 e = Ps[b];
      const float2* am = As + (e.x & 0xffff) + q;
      const float2* an = As + (e.x >> 16) + q;
      float2 vm[4], vn[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        vm[i] = am[i * TC_PTS];
        vn[i] = an[i * TC_PTS];
      }
      if (sc != 1.0f) {  // FP16: a power of two, so scaling A_m equals scaling the product
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          vm[i].x *= sc;
          vm[i].y *= sc;
        }
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) x[4 * i + j] = vm[i].x * vn[j].x + vm[i].y * vn[j].y;
    };
    // hi + lo of eight values, two per conversion
    auto split8 = [&](const float* x, uint4& hw, uint4& lw) {
      uint32_t h[4], l[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (a.f16) {
          const __half2 hh = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
          const float2 hb = __half22float2(hh);
          const __half2 ll = __floats2half2_rn(x[2 * i] - hb.x, x[2 * i + 1] - hb.y);
          h[i] = *reinterpret_cast<const uint32_t*>(&hh);
          l[i] = *reinterpret_cast<const uint32_t*>(&ll);
        } else {
          const __nv_bfloat162 hh = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
          const float2 hb = __bfloat1622float2(hh);
          const __nv_bfloat162 ll = __floats2bfloat162_rn(x[2 * i] - hb.x, x[2 * i + 1] - hb.y);
          h[i] = *reinterpret_cast<const uint32_t*>(&hh);
          l[i] = *reinterpret_cast<const uint32_t*>(&ll);
        }
      }
      hw = make_uint4(h[0], h[1], h[2], h[3]);
      lw = make_uint4(l[0], l[1], l[2], l[3]);
    };
    int wi = cid;
    while (wi < nitems && !live_item(wi)) wi += ncl;
    if (wi < nitems) fetch(wi);
    int c = 0;
    // every U thread passes the same named barriers: the item loop does not
    // depend on the stop flag; after a stop the chunks are skipped unwaited
    while (wi < nitems) {
      const int wn = next_live(wi);
      tc::named_sync(1, UT);  // every chunk of the previous tile is written
#pragma unroll
      for (int r = 0; r < AL; ++r) {
        const int i = u + r * UT;
        if (i < nm * TC_PTS) As[i] = nxt[r];
      }
      tc::named_sync(1, UT);
      if (wn < nitems) fetch(wn);
      for (int rb = 0; rb < nrb; ++rb)
        for (int kc = 0; kc < kchunks; ++kc, ++c) {
          const int s = c % S::STAGES, round = c / S::STAGES;
          // lane 0 waits for the stage; the warp follows its result (uniform)
          int go = 1;
          if (lane == 0) {
            if (*stop) {
              go = 0;
            } else if (round > 0 && !tc::mbar_wait(&empty[s], (round - 1) & 1, wait_ns)) {
              fail();
              go = 0;
            }
          }
          if (!__shfl_sync(0xffffffffu, go, 0)) continue;
          unsigned char* st = smem + (size_t)s * S::STAGE;
          float x[16];
          u16(2 * kc + half, x);
#pragma unroll
          for (int kq2 = 0; kq2 < 2; ++kq2) {
            const int kq = 2 * half + kq2;
            uint4 hw, lw;
            split8(x + 8 * kq2, hw, lw);
            const size_t o = ((size_t)kq * TC_PTS + q) * 16;
            *reinterpret_cast<uint4*>(st + o) = hw;
            *reinterpret_cast<uint4*>(st + S::V_BYTES + o) = lw;
          }
          tc::fence_proxy_async();  // the stores are seen by the tensor cores' reads
          __syncwarp();
          if (lane == 0) {
            if (PAIR) tc::mbar_arrive_cluster(at0(&full[s]));  // CTA 0's barrier, released at cluster scope
            else tc::mbar_arrive(&full[s]);
          }
        }
      wi = wn;
    }
  } else if (warp < 2 + S::EW) {
    // ---------------- epilogue: warps 2..5 (with ESPLIT 2..9), one point per thread ----------------
    const int quarter = warp & 3;  // this warp may access TMEM lanes 32 quarter ..
    // ESPLIT: warps 6..9 form NL for the upper half of the modes
    constexpr int NH = S::ESPLIT ? (N + 1) / 2 : (N > 0 ? N : 1);
    const int half = S::ESPLIT && warp >= 6 ? 1 : 0;
    const int row_in_tile = quarter * 32 + lane;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    // FP16: D = 2^(eV + eG) R; folded into the mode values of the l-sum
    const float inv = a.f16 ? ldexpf(1.0f, -(f16_v_exp(ls, a.n, a.B) - a.eVoff + a.eG)) : 1.0f;
    int w = 0;
    constexpr int NA = N > 0 ? N : 1;
    for (int wi = cid; wi < nitems && !*stop; wi += ncl) {
      if (!live_item(wi)) continue;
      // the l-sum epilogue has one tile per CTA and work item
      const bool mine = live(tile_of(wi, 0));
      const int pt = tile_of(wi, 0) * TC_PTS + row_in_tile;
      const int j = pt / n, t = pt - j * n;
      float2 av[NA], nl[NH];
      if (OUT == 0 && mine) {
#pragma unroll
        for (int l = 0; l < N; ++l) {
          av[l] = a.A[((size_t)j * N + l) * n + t];
          av[l].x *= inv;
          av[l].y *= inv;
        }
#pragma unroll
        for (int p = 0; p < NH; ++p) nl[p] = make_float2(0.f, 0.f);
      }
      for (int rb = 0; rb < nrb; ++rb, ++w) {
        const int acc = w % NBUF, use = w / NBUF;
        int ok = 1;
        if (lane == 0) ok = tc::mbar_wait(&acc_full[acc], use & 1, wait_ns) ? 1 : 0;
        if (!__shfl_sync(0xffffffffu, ok, 0)) {
          if (lane == 0) fail();
          break;
        }
        tc::fence_after_sync();
        const uint32_t taddr = tmem + lane_off + (uint32_t)(acc * S::ACC_COLS);
        if (OUT == 1) {
#pragma unroll
          for (int h = 0; h < TPW; ++h) {
            const int tile = tile_of(wi, h);
            if (!live(tile)) continue;  // (every thread of the warp skips alike)
            const int pth = tile * TC_PTS + row_in_tile;
            const int jh = pth / n, th = pth - jh * n;
            float* z = a.Zout + (size_t)jh * a.zrows * n + th;
            const uint32_t tb = taddr + (uint32_t)(h * NB);
            auto put = [&](int c0, const uint32_t (&v)[16]) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const int r = rb * NB + c0 + i;
                if (r < a.zrows) z[(size_t)r * n] = __uint_as_float(v[i]) * inv;
              }
            };
            // each 16-column TMEM load is issued before the previous chunk's
            // stores (two register buffers in turn)
            uint32_t va[16], vb[16];
            tc::tmem_ld16_issue(tb, va);
            tc::tmem_wait16(va);
            for (int c0 = 0; c0 < NB; c0 += 32) {
              const bool more1 = c0 + 16 < NB;
              if (more1) tc::tmem_ld16_issue(tb + c0 + 16, vb);
              put(c0, va);
              if (!more1) break;
              tc::tmem_wait16(vb);
              const bool more2 = c0 + 32 < NB;
              if (more2) tc::tmem_ld16_issue(tb + c0 + 32, va);
              put(c0 + 16, vb);
              if (more2) tc::tmem_wait16(va);
            }
          }
        } else if (mine) {
          if constexpr (S::ESPLIT) {
            if (half == 0) drain_rb_h<N, NB, 0, 0, NH>(rb, taddr, av, nl);
            else drain_rb_h<N, NB, 0, NH, N>(rb, taddr, av, nl);
          } else {
            drain_rb<N, NB, 0>(rb, taddr, av, nl);
          }
        }
        // this warp's reads of the accumulator are done: one arrival on
        // CTA 0's barrier
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) {
          if (PAIR) tc::mbar_arrive_remote(at0(&acc_empty[acc]));
          else tc::mbar_arrive(&acc_empty[acc]);
        }
      }
      if (*stop) break;
      if (OUT == 0 && mine) {
        float2* out = a.NL + (size_t)j * N * n + t;
        const int p0 = half * NH;
#pragma unroll
        for (int p = 0; p < NH; ++p)
          if (p0 + p < N) out[(size_t)(p0 + p) * n] = nl[p];
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (PAIR) tc::cluster_sync();  // no CTA leaves while its peer may still signal it or read its memory
  if (warp == 1) tc::tmem_dealloc<PAIR>(tmem, S::TMEM_COLS);
}

// V to the blocked 16-bit hi/lo operand layout [KKp/8][npts][8] read by the
// TMA of k_tc_contract (BF16, or FP16 scaled by 2^eV), V formed from the
// pair products U of A and from Y = h_R * U ([M+1][K][n]) as for K3:
// MODE (= raman_mode) 0: V = U; 1: V = (1 - fR) U + fR Y; 2: V = [U; Y].
// A block takes 32 points (the lanes of each warp) and stages their N mode
// values in shared memory ([N][32]); warp w packs the 8-wide chunks
// kc = w, w + 8, ...  Y loads and the 16-byte stores are coalesced across
// the lanes.
constexpr int PACK_PTS = 32, PACK_WARPS = 8;

// Eight consecutive K values of one point to the blocked layout
// [K/EPC][npts][EPC]: one or two 16-byte pieces.
template <int OP>
__device__ __forceinline__ void store_chunk8(typename Split<OP>::T* V, int kc, int npts_total, int pt,
                                             const typename Split<OP>::T* v8) {
  constexpr int EPC = Split<OP>::EPC;
#pragma unroll
  for (int q = 0; q < 8 / EPC; ++q) {
    const size_t o = ((size_t)(kc * (8 / EPC) + q) * npts_total + pt) * EPC;
    *reinterpret_cast<uint4*>(V + o) = *reinterpret_cast<const uint4*>(v8 + q * EPC);
  }
}

template <int MODE, int OP>
__global__ void __launch_bounds__(PACK_PTS * PACK_WARPS) k_pack_hilo(
    Geo g, const float2* __restrict__ A, const float* __restrict__ Y, const int2* __restrict__ pairs, int KKp,
    int npts_total, void* __restrict__ Vhi_, void* __restrict__ Vlo_, const LoopState* __restrict__ ls) {
  using H = Split<OP>;
  constexpr bool F16 = OP == 1;
  using T = typename H::T;
  T* Vhi = reinterpret_cast<T*>(Vhi_);
  T* Vlo = reinterpret_cast<T*>(Vlo_);
  extern __shared__ float2 pack_as[];  // [N][PACK_PTS]
  pdl_enter();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = g.n, npts = g.B * (g.M + 1) * n;
  const int pt0 = blockIdx.x * PACK_PTS;  // n is a multiple of 128: a block lies in one slice
  const int j = pt0 / n;                  // the slice
  {
    int b, jl;
    slot_of(g, j, b, jl);
    if (slice_skipped(ls + b, jl)) return;
  }
  const int pt = pt0 + lane, t = pt - j * n;
  const bool ok = pt < npts;
  const float scale = F16 ? ldexpf(1.0f, f16_v_exp(ls, n, g.B)) : 1.0f;
  for (int i = threadIdx.x; i < g.N * PACK_PTS; i += blockDim.x) {
    const int l = i / PACK_PTS, q = i - l * PACK_PTS;
    pack_as[i] = (pt0 + q < npts) ? A[((size_t)j * g.N + l) * n + (pt0 + q - j * n)] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (!ok) return;
  const float* y = Y + (size_t)j * g.K * n + t;
  const float fR = (float)g.fR, fK = (float)(1.0 - g.fR);
  auto U = [&](int k) {
    const int2 mn = pairs[k];
    const float2 am = pack_as[mn.x * PACK_PTS + lane];
    if (mn.x == mn.y) return am.x * am.x + am.y * am.y;
    const float2 an = pack_as[mn.y * PACK_PTS + lane];
    return 2.0f * (am.x * an.x + am.y * an.y);
  };
  for (int kc = w; kc < KKp / 8; kc += PACK_WARPS) {
    __align__(16) T hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kc * 8 + i;
      float x = 0.f;
      if (k < g.KK) {
        if (MODE == 0) x = U(k);
        else if (MODE == 1) x = fK * U(k) + fR * y[(size_t)k * n];
        else x = k < g.K ? U(k) : y[(size_t)(k - g.K) * n];
      }
      x *= scale;
      hi[i] = H::rn(x);
      lo[i] = H::rn(x - H::back(hi[i]));
    }
    store_chunk8<OP>(Vhi, kc, npts_total, pt, hi);
    store_chunk8<OP>(Vlo, kc, npts_total, pt, lo);
  }
}

// Low-rank coupling, second GEMM: V' = (1 - fR) Z + fR Y' (MODE 1) or Z
// (MODE 0) from the rows of Z = W U and Y' = h_R * Z ([M+1][r][n]) to the
// blocked hi/lo layout [KKp/EPC][npts][EPC] (r padded with zeros to KKp);
// FP16 scaled by 2^(eV - eVoff), since |Z| <= 2^eVoff max |U|.  A block
// takes 32 points (the lanes of each warp); warp w packs the 8-wide chunks
// kc = w, w + 8, ...: Z / Y' loads coalesced across the lanes, eight warps
// of loads in flight per 32 points.
template <int MODE, int OP>
__global__ void __launch_bounds__(PACK_PTS * PACK_WARPS) k_pack_rows(
    Geo g, const float* __restrict__ Zs, const float* __restrict__ Ys, int r, int KKp, int npts_total,
    void* __restrict__ Vhi_, void* __restrict__ Vlo_, int eVoff, const LoopState* __restrict__ ls) {
  using H = Split<OP>;
  using T = typename H::T;
  constexpr bool F16 = OP == 1;
  T* Vhi = reinterpret_cast<T*>(Vhi_);
  T* Vlo = reinterpret_cast<T*>(Vlo_);
  pdl_enter();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = g.n;
  const int pt = blockIdx.x * PACK_PTS + lane;
  if (pt >= g.B * (g.M + 1) * n) return;
  const int j = pt / n, t = pt - j * n;  // j: the slice
  {
    int b, jl;
    slot_of(g, j, b, jl);
    if (slice_skipped(ls + b, jl)) return;
  }
  const float* z = Zs + (size_t)j * r * n + t;
  const float* y = Ys + (size_t)j * r * n + t;
  const float fR = (float)g.fR, fK = (float)(1.0 - g.fR);
  const float scale = F16 ? ldexpf(1.0f, f16_v_exp(ls, n, g.B) - eVoff) : 1.0f;
  for (int kc = w; kc < KKp / 8; kc += PACK_WARPS) {
    __align__(16) T hi[8], lo[8];
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kc * 8 + i;
      x[i] = 0.f;
      if (k < r) x[i] = MODE == 1 ? fK * __ldcg(z + (size_t)k * n) + fR * __ldcg(y + (size_t)k * n)
                                  : __ldcg(z + (size_t)k * n);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float v = x[i] * scale;
      hi[i] = H::rn(v);
      lo[i] = H::rn(v - H::back(hi[i]));
    }
    store_chunk8<OP>(Vhi, kc, npts_total, pt, hi);
    store_chunk8<OP>(Vlo, kc, npts_total, pt, lo);
  }
}

// Low-rank coupling with 16-bit operands (OP 0 BF16, 1 FP16) and Raman: K2
// on the rows of Z, writing the operand of GEMM 2 directly:
// V' = (1 - fR) Z + fR h_R * Z = F^-1{F{Z} Hv} with the transfer function
// Hv = (1 - fR)/n + fR H.  A cluster of four blocks takes the eight rows
// 8 grp .. 8 grp + 7 of Z (one 16-byte core-matrix row of the blocked
// layout [KKp/8][npts][8] per point): block `rank` transforms rows
// 8 grp + 2 rank and + 1 as one complex transform pair (the forward
// transform's first pass reads them straight from global memory) and keeps
// the result in time order in its shared memory; then block `rank` writes
// the points [rank n/4, (rank + 1) n/4) of all eight rows, reading the
// other blocks' results through distributed shared memory, as whole 16-byte
// hi and lo rows (coalesced across the lanes), so that neither Y' nor a
// separate pack pass goes through HBM.  Rows r .. 8 ceil(r/8) - 1 are
// written as zeros; the padding columns beyond are zero from the
// workspace's creation.  FP16 values are scaled by 2^(eV - eVoff) as in
// k_pack_rows.  grid (4 ceil(r/8), M+1) in clusters of 4 along x.
template <int EPT, int OP>
__global__ void __launch_bounds__(512) k_raman_vpack(Geo g, const float* __restrict__ Zs, int r,
                                                      const float2* __restrict__ Hv, const float2* __restrict__ tw,
                                                      int npts_total, void* __restrict__ Vhi_,
                                                      void* __restrict__ Vlo_, int eVoff,
                                                      const LoopState* __restrict__ ls) {
  namespace cg = cooperative_groups;
  using Hs = Split<OP>;
  using T = typename Hs::T;
  static_assert(sizeof(T) == 2, "16-bit operands");
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  pdl_enter();
  const int j = blockIdx.y;  // the slice (the same for every block of a cluster)
  {
    int b, jl;
    slot_of(g, j, b, jl);
    if (slice_skipped(ls + b, jl)) return;
  }
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int n = g.n, grp = blockIdx.x / 4, k1 = 8 * grp + 2 * rank;
  if (k1 < r) {
    const bool has2 = k1 + 1 < r;
    const float* z1 = Zs + ((size_t)j * r + k1) * n;
    auto load = [&](int t) { return make_float2(__ldcg(z1 + t), has2 ? __ldcg(z1 + n + t) : 0.f); };
    auto to_smem = [&](int q, float2 x) { sm[pad16(q)] = cmul<float>(x, Hv[q]); };
    fft_block<float, -1, EPT>(sm, n, tw, load, to_smem);
    auto from_smem = [&](int q) { return sm[pad16(q)]; };
    auto keep = [&](int t, float2 y) { sm[pad16(t)] = y; };
    fft_block<float, +1, EPT>(sm, n, tw, from_smem, keep);
  }
  cluster.sync();  // the four row pairs of the group, in time order
  const float2* ys[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) ys[u] = cluster.map_shared_rank(sm, u);
  const float scale = OP == 1 ? ldexpf(1.0f, f16_v_exp(ls, n, g.B) - eVoff) : 1.0f;
  uint4* Vhi = reinterpret_cast<uint4*>(Vhi_) + (size_t)grp * npts_total + (size_t)j * n;
  uint4* Vlo = reinterpret_cast<uint4*>(Vlo_) + (size_t)grp * npts_total + (size_t)j * n;
  const int q4 = n / 4;
  // (unrolled: the partners' values of several points in flight at once)
#pragma unroll 4
  for (int i = threadIdx.x; i < q4; i += blockDim.x) {
    const int t = rank * q4 + i;
    __align__(16) T hi[8], lo[8];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int ku = 8 * grp + 2 * u;
      const float2 y = ku < r ? ys[u][pad16(t)] : make_float2(0.f, 0.f);
      const float v0 = y.x * scale, v1 = ku + 1 < r ? y.y * scale : 0.f;
      hi[2 * u] = Hs::rn(v0);
      hi[2 * u + 1] = Hs::rn(v1);
      lo[2 * u] = Hs::rn(v0 - Hs::back(hi[2 * u]));
      lo[2 * u + 1] = Hs::rn(v1 - Hs::back(hi[2 * u + 1]));
    }
    Vhi[t] = *reinterpret_cast<const uint4*>(hi);
    Vlo[t] = *reinterpret_cast<const uint4*>(lo);
  }
  cluster.sync();  // no block leaves while the others read its shared memory
}

}  // namespace gm
