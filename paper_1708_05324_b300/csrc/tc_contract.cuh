// Coupling contraction on the 5th-generation tensor cores (mixed precision).
//
// Per point (j, t) of the MPA iteration (Eq. 1 bracket after the symmetry
// rewrite):  R_r = sum_k G[r][k] V_k   (r = (p <= l), k over the pair terms),
//            NL_p = sum_l A_l R_pl.
// Over a tile of BN points this is the GEMM  D[128 x BN] = G[128 x KKp] .
// V[BN x KKp]^T  with G (<= 128 rows) and V split into BF16 hi + lo parts;
// D accumulates hi.hi + hi.lo + lo.hi in FP32 in TMEM (the lo.lo product is
// below FP32 rounding of the result).  V tiles arrive by TMA; one thread
// issues tcgen05.mma; the epilogue reads D with tcgen05.ld and forms the
// l-sum, writing NL in FP32.
//
// Operand layout (both K-major, no swizzle): core matrices of 8 rows x 8
// elements (16 bytes), stored [k/8][row][8], so that along K neighbouring
// core matrices are rows*16 bytes apart (LBO) and along M/N 128 bytes (SBO).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace gm {

constexpr int TC_M = 128;   // MMA M: rows of G (P padded)
constexpr int TC_BN = 128;  // MMA N: points per tile
constexpr int TC_KMAX = 160;

struct TcArgs {
  const __nv_bfloat16* Ghi;  // [KKp/8][128][8]
  const __nv_bfloat16* Glo;
  int KKp;                   // padded K (multiple of 16, <= TC_KMAX)
  int P;                     // live rows of G
  int N, n, M;               // modes, samples, substeps (tiles cover j = 0..M)
  const float2* A;           // [M+1][N][n] fields (for the l-sum)
  float2* NL;                // [M+1][N][n] output
  const int2* rows;          // [P] (p, l) of each row
  float* Rout;               // probe mode: [128][npts] raw D
  int npts;                  // total points (probe mode)
  unsigned* err;             // set to 1 if a wait times out
};

// B tiles, reused as the D staging area (128 x BN floats) after the MMAs
__host__ __device__ __forceinline__ size_t tc_bregion_bytes(int KKp) {
  const size_t b = (size_t)2 * TC_BN * KKp * 2, r = (size_t)TC_M * TC_BN * 4;
  return b > r ? b : r;
}
__host__ __device__ __forceinline__ size_t tc_smem_bytes(int KKp, int N) {
  return (size_t)2 * TC_M * KKp * 2            // Ghi, Glo
         + tc_bregion_bytes(KKp)               // Bhi, Blo / D staging
         + (size_t)4 * N * TC_BN * 4           // A values and NL accumulators
         + (size_t)TC_M * 8                    // rows table
         + 1024;                               // alignment of the base
}

template <bool PROBE>
__global__ void __launch_bounds__(128, 1) k_tc_contract(const __grid_constant__ CUtensorMap mapHi,
                                                         const __grid_constant__ CUtensorMap mapLo, TcArgs a,
                                                         const LoopState* __restrict__ ls) {
  extern __shared__ __align__(16) unsigned char tc_smem_raw[];
  // TMA destinations and MMA operands start on a 1024-byte boundary
  unsigned char* smraw = tc_smem_raw + ((1024 - (tc::smem_addr(tc_smem_raw) & 1023)) & 1023);
  __shared__ __align__(8) uint64_t bar_load, bar_mma;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KKp = a.KKp;
  const size_t opnd = (size_t)TC_M * KKp;  // elements per operand tile
  __nv_bfloat16* sGhi = reinterpret_cast<__nv_bfloat16*>(smraw);
  __nv_bfloat16* sGlo = sGhi + opnd;
  __nv_bfloat16* sBhi = sGlo + opnd;
  __nv_bfloat16* sBlo = sBhi + opnd;
  float* sR = reinterpret_cast<float*>(sBhi);            // D staging after the MMAs (128 x BN floats)
  float* sA = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(sBhi) + tc_bregion_bytes(KKp));  // [2N][BN]
  float* sNL = sA + 2 * a.N * TC_BN;                      // [2N][BN]
  int2* sRows = reinterpret_cast<int2*>(sNL + 2 * a.N * TC_BN);

  // constant operand and tables (before waiting on the previous kernel)
  {
    const uint4* gh = reinterpret_cast<const uint4*>(a.Ghi);
    const uint4* gl = reinterpret_cast<const uint4*>(a.Glo);
    uint4* sh = reinterpret_cast<uint4*>(sGhi);
    uint4* sl = reinterpret_cast<uint4*>(sGlo);
    const int chunks = (int)(opnd / 8);
    for (int i = tid; i < chunks; i += blockDim.x) {
      sh[i] = gh[i];
      sl[i] = gl[i];
    }
    if (!PROBE)
      for (int i = tid; i < a.P; i += blockDim.x) sRows[i] = a.rows[i];
  }
  if (tid == 0) {
    tc::mbar_init(&bar_load, 1);
    tc::mbar_init(&bar_mma, 1);
    tc::fence_mbar_init();
    abort_flag = 0;
  }
  // generic-proxy writes of G become visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) tc::tmem_alloc(&tmem_base, TC_BN);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  pdl_enter();
  const uint32_t tmem = tmem_base;
  const int iter = PROBE ? 0 : ls->iter;
  const int tiles_per_j = a.n / TC_BN;
  const int ntiles = PROBE ? a.npts / TC_BN : (a.M + 1) * tiles_per_j;
  const uint32_t idesc = tc::idesc_f16(TC_M, TC_BN, true);
  const uint32_t lboA = TC_M * 16, lboB = TC_BN * 16, sbo = 128;
  const unsigned tx_bytes = (unsigned)(2 * opnd * sizeof(__nv_bfloat16));
  unsigned phase = 0;

  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int pt0 = tile * TC_BN;
    const int j = PROBE ? 0 : pt0 / a.n;
    if (!PROBE && iter > 0 && j == 0) continue;
    if (tid == 0) {
      tc::mbar_arrive_expect_tx(&bar_load, tx_bytes);
      tc::tma_load_3d(sBhi, &mapHi, 0, pt0, 0, &bar_load);
      tc::tma_load_3d(sBlo, &mapLo, 0, pt0, 0, &bar_load);
      if (!tc::mbar_wait(&bar_load, phase)) {
        abort_flag = 1;
      } else {
        tc::fence_after_sync();
        const uint32_t aH = tc::smem_addr(sGhi), aL = tc::smem_addr(sGlo);
        const uint32_t bH = tc::smem_addr(sBhi), bL = tc::smem_addr(sBlo);
        for (int kk = 0; kk < KKp / 16; ++kk) {
          const uint32_t offA = (uint32_t)kk * 2 * lboA, offB = (uint32_t)kk * 2 * lboB;
          tc::mma_f16(tmem, tc::smem_desc(aH + offA, lboA, sbo), tc::smem_desc(bH + offB, lboB, sbo), idesc,
                      kk > 0 ? 1u : 0u);
          tc::mma_f16(tmem, tc::smem_desc(aH + offA, lboA, sbo), tc::smem_desc(bL + offB, lboB, sbo), idesc, 1u);
          tc::mma_f16(tmem, tc::smem_desc(aL + offA, lboA, sbo), tc::smem_desc(bH + offB, lboB, sbo), idesc, 1u);
        }
        tc::mma_commit(&bar_mma);
      }
    }
    __syncthreads();
    if (abort_flag) break;
    if (!tc::mbar_wait(&bar_mma, phase)) {
      atomicExch(a.err, 1u);
      abort_flag = 1;
    }
    phase ^= 1;
    __syncthreads();
    if (abort_flag) break;
    tc::fence_after_sync();
    // D row r = 32 warp + lane lives in TMEM lane r
    const int r = warp * 32 + lane;
    for (int c = 0; c < TC_BN; c += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
      if (PROBE) {
#pragma unroll
        for (int i = 0; i < 16; ++i) a.Rout[(size_t)r * a.npts + pt0 + c + i] = v[i];
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) sR[r * TC_BN + c + i] = v[i];
      }
    }
    tc::fence_before_sync();
    if (!PROBE) {
      // l-sum: thread t owns point t of the tile
      const int t = tid;
      const int t0 = pt0 - j * a.n;
      const float2* Aj = a.A + (size_t)j * a.N * a.n;
      for (int l = 0; l < a.N; ++l) {
        const float2 x = Aj[(size_t)l * a.n + t0 + t];
        sA[(2 * l) * TC_BN + t] = x.x;
        sA[(2 * l + 1) * TC_BN + t] = x.y;
        sNL[(2 * l) * TC_BN + t] = 0.f;
        sNL[(2 * l + 1) * TC_BN + t] = 0.f;
      }
      __syncthreads();  // sR complete
      for (int rr = 0; rr < a.P; ++rr) {
        const float Rv = sR[rr * TC_BN + t];
        const int2 pl = sRows[rr];
        sNL[(2 * pl.x) * TC_BN + t] += sA[(2 * pl.y) * TC_BN + t] * Rv;
        sNL[(2 * pl.x + 1) * TC_BN + t] += sA[(2 * pl.y + 1) * TC_BN + t] * Rv;
        if (pl.x != pl.y) {
          sNL[(2 * pl.y) * TC_BN + t] += sA[(2 * pl.x) * TC_BN + t] * Rv;
          sNL[(2 * pl.y + 1) * TC_BN + t] += sA[(2 * pl.x + 1) * TC_BN + t] * Rv;
        }
      }
      float2* out = a.NL + (size_t)j * a.N * a.n + t0 + t;
      for (int p = 0; p < a.N; ++p)
        out[(size_t)p * a.n] = make_float2(sNL[(2 * p) * TC_BN + t], sNL[(2 * p + 1) * TC_BN + t]);
    }
    __syncthreads();  // sR / B buffers and TMEM free for the next tile
    tc::fence_after_sync();
  }
  if (abort_flag && tid == 0) atomicExch(a.err, 1u);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TC_BN);
}

// V (FP32: [M+1][KK][n], or the pair products of A when Kerr only) to the
// blocked BF16 hi/lo operand layout [KKp/8][npts][8] read by the TMA of
// k_tc_contract.  One thread per point; each writes whole 16-byte chunks.
template <int MODE>
__global__ void __launch_bounds__(256) k_pack_bf16(Geo g, const float2* __restrict__ A, const float* __restrict__ V,
                                                   const int2* __restrict__ pairs, int KKp, int npts_total,
                                                   __nv_bfloat16* __restrict__ Vhi, __nv_bfloat16* __restrict__ Vlo,
                                                   const LoopState* __restrict__ ls) {
  pdl_enter();
  const int pt = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n;
  if (pt >= (g.M + 1) * n) return;
  const int j = pt / n, t = pt - j * n;
  if (ls->iter > 0 && j == 0) return;
  const float2* a = A + (size_t)j * g.N * n;
  const float* v = V + (size_t)j * g.KK * n + t;
  for (int kc = 0; kc < KKp / 8; ++kc) {
    __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = kc * 8 + i;
      float x = 0.f;
      if (k < g.KK) x = MODE == 0 ? pair_product<float>(a, n, pairs[k], t) : v[(size_t)k * n];
      hi[i] = __float2bfloat16_rn(x);
      lo[i] = __float2bfloat16_rn(x - __bfloat162float(hi[i]));
    }
    const size_t o = ((size_t)kc * npts_total + pt) * 8;
    *reinterpret_cast<uint4*>(Vhi + o) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(Vlo + o) = *reinterpret_cast<const uint4*>(lo);
  }
}

}  // namespace gm
