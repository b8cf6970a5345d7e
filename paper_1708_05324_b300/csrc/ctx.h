// Layout of a context and of a propagation workspace, shared by the host-side
// translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <mutex>
#include <vector>

#include <cuda.h>
#include <cuda_bf16.h>

#include "../../include/gmmnlse.h"
#include "kernels.cuh"
#include "contract_tile.cuh"

// ---------------------------------------------------------------------------
// Workspace of one propagation in flight
// ---------------------------------------------------------------------------
struct gm_job {
  gmmnlse_ctx* ctx = nullptr;
  int Mcap = 0;
  int slots = 1;            // propagations the workspace holds (a packed launch's B; 1 otherwise)
  double2* psi0 = nullptr;  // [N][n]
  void* psiR = nullptr;     // [N][n] cplx<R> (aliases psi0 in FP64)
  void* dpsi = nullptr;     // [M][N][n]
  void* A = nullptr;        // [M+1][N][n]
  void* V = nullptr;        // Y = h_R * U: [M+1][K][n]
  void* NL = nullptr;       // [M+1][N][n]
  void* I = nullptr;        // [M+1][N][n]
  void* E = nullptr;        // [M+1][N][n]
  double2* EM64 = nullptr;  // [2][N][n]
  double2* io = nullptr;    // [2][N][n] staging / FP64 FFT scratch
  int* flag = nullptr;
  gm::LoopState* ls = nullptr;      // device
  double2* part = nullptr;          // [TRAPZ_MAX_BLOCKS] per-block sums of K5
  unsigned* bar = nullptr;          // grid-barrier counter of the long-step kernel
  int persist_grid = -1;            // blocks of the long-step kernel (0: not used; -1: not chosen yet)
  gm::LoopState* h_ls = nullptr;    // pinned host mirror
  double2* h_io = nullptr;      // pinned host staging [N][n]
  cudaStream_t cap = nullptr;   // private stream for graph capture
  // phase tables currently in E
  double tab_dz = -1.0;
  int tab_M = -1, tab_Mrem = -1;
  // cached graphs: for substep counts M and Mrem
  struct G {
    int Mj = -1;
    int which = 0;
    double dz = 0.0;  // the kernels' parameters (dz/2 of the trapezoid) are baked into the graph
    int qv = -1;      // the context's Q version the graph was built with
    int Mfull = -1;   // the propagation's full long step (z of every substep derives from it)
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
  } graphs[2];
  // packed launches: the graph of a long step over the first B slots, [B]
  std::vector<G> pack_graphs;
  size_t bytes = 0;
  // mixed precision: blocked BF16 hi/lo pair-term operand and its TMA maps
  __nv_bfloat16* Vhi = nullptr;  // [KKp/EPC][(M+1) n][EPC] (and rKKp columns for the low-rank GEMM 2)
  __nv_bfloat16* Vlo = nullptr;
  CUtensorMap mapHi, mapLo;
  CUtensorMap mapHi2, mapLo2;    // the same buffers with rKKp columns (low-rank GEMM 2)
  void* Z = nullptr;             // low-rank: Z = W U, [M+1][r][n] R
  double* Ubar = nullptr;        // saturation: [M+1][K] time integrals of the pair products (FP64)
  double* Rs = nullptr;          // saturation: [M+1][P] rows R_(p<=l) (FP64)
  int Mprop = 0;                 // substeps per full long step of the current propagation
};

struct gmmnlse_ctx {
  gmmnlse_params prm;
  int N, n, K, P, KK, raman_mode, ept;
  bool fp64;
  double fR, omega0, gamma0;
  double* beta = nullptr;       // [N][n]
  double* Q = nullptr;          // [N][N] linear mode coupling Q[n][p] (device), or none
  double* gain = nullptr;       // [N] small-signal field gain g_p (device), or none
  double* fprof = nullptr;      // [fcount] longitudinal profile f(z) of Q (device), or none (f = 1)
  int fcount = 0;
  double fdz = 0.0;             // spacing of the profile samples [m]
  double sat = 0.0;             // saturation coefficient of the gain (1/I_sat), 0: none
  double* GRt = nullptr;        // [K][P] reduced S^R transposed (FP64, device), while sat != 0
  std::vector<double> GR_host;  // [P][K] reduced S^R (host), kept from creation for the saturation
  std::vector<double> beta0;    // [N] beta_p(omega = 0) (host): the intermode beat lengths
  double s_max = 0.0;           // max_p S^K_pppp (host): the nonlinear length
  int qv = 0;                   // bumped at every change of Q, f, gain or sat (graphs record the one they hold)
  double2* tw64 = nullptr;      // [n] + radix-16 pass tables of n
  double2* tw64h = nullptr;     // [n/2] + pass tables of n/2
  float2* tw32 = nullptr;       // [n] + pass tables of n
  void* H = nullptr;            // [n] cplx<R>: (dt/n) DFT(h_R), the Raman transfer function with the inverse 1/n
  void* Hv = nullptr;           // [n] float2 (FP32 contexts): (1 - fR)/n + fR H, the transfer function of
                                // V' = (1 - fR) Z + fR h_R * Z (the low-rank operand of 16-bit GEMM 2)
  void* fac = nullptr;          // [n] R: gamma0 s(w_q)
  void* G = nullptr;            // [P][KK] R
  int2* rows = nullptr;         // [P]
  int2* pairs = nullptr;        // [K]
  // N <= 8 on the CUDA cores: the contraction kernel compiled for this
  // context's nonzero coupling entries (nzlist.cu; CUmodule / CUfunction),
  // null when k_contract_reg runs instead
  void* nz_mod = nullptr;
  void* nz_fn = nullptr;
  bool tc = false;               // contraction on tensor cores (mixed precision)
  int KKp = 0;                   // K padded to a multiple of TC_KC (32)
  int tc_rows = 0;               // rows of G padded to whole row blocks
  bool f16 = false;              // tensor-core operands FP16 (MIXED_FP16), else BF16
  bool tf32 = false;             // tensor-core operands TF32 (MIXED_TF32), 4-byte elements
  int eG = 0;                    // FP16: G scaled by 2^eG
  __nv_bfloat16* Ghi = nullptr;  // [tc_rows/8][KKp/EPC][8][EPC]: 16-bit (EPC 8) or TF32 words (EPC 4)
  __nv_bfloat16* Glo = nullptr;
  CUtensorMap mapGhi, mapGlo;
  void* Gt = nullptr;            // [KKt][Pt] R: G transposed, zero-padded (N > 8, CUDA cores)
  int KKt = 0, Pt = 0;
  int2* rows_t = nullptr;        // [P] (p, l) of the rows of Gt and Xt: by diagonals l - p, so that
                                 // neighbouring rows of a tile have distinct p and l (l-sum atomics)
  // low-rank coupling G = X W (N > 8, S^R = S^K): X [P][r] orthonormal
  // columns, W = X^T G [r][K]; Z = W U, Y' = h_R * Z, R = X V'
  bool lr = false;
  int r = 0;
  // general coupling (complex S^K, S^R with no symmetry; Eq. 1 without the
  // real S of Eq. 2): the N^2 real rows U_k of the pair products, Re(A_m
  // A_n^*) for m <= n then Im(A_m A_n^*) for m < n (gpairs: (m, n), n + N
  // for an imaginary row), rows of Gt the real and imaginary parts of R_pl
  // for every (p, l): row 2 (p N + l) + {0, 1}
  bool general = false;
  int gK = 0;                    // N^2
  int2* gpairs = nullptr;        // [N^2]
  int eW = 0;                    // max_s sum_k |W[s][k]| < 2^eW (|Z| < 2^eW max |U|)
  void* Wt = nullptr;            // [KKt][rP1] R: W^T, CUDA-core GEMM 1 (rows r padded to rP1)
  void* Xt = nullptr;            // [rK2][Pt] R: X^T, CUDA-core GEMM 2 (K = r padded to rK2)
  int rP1 = 0, rK2 = 0;
  int NB1 = 0, r_rows = 0;       // tensor cores: row block of GEMM 1, r padded to whole blocks
  int rKKp = 0;                  // tensor cores: r padded to TC_KC (K of GEMM 2)
  int eW16 = 0, eX16 = 0;        // FP16 exponents of W and X
  // 16-bit GEMM 1 (U formed in the kernel): the columns of U in 4 x 4 blocks
  // of (m, n), m-block <= n-block, m-major; ublk [nublk] holds each block's
  // first (m0, n0); W's columns follow that order (zero where m > n or a
  // mode is past N); KKpU = 16 nublk padded to TC_KC
  int2* ublk = nullptr;
  int nublk = 0, KKpU = 0;
  __nv_bfloat16 *Whi = nullptr, *Wlo = nullptr, *Xhi = nullptr, *Xlo = nullptr;
  CUtensorMap mapWhi, mapWlo, mapXhi, mapXlo;
  // limit of every mbarrier wait of the tensor-core GEMMs [ns] (1 s;
  // GMMNLSE_TC_WAIT_MS at create), and the test hook GMMNLSE_TC_STALL that
  // makes their MMA issuer wait on a barrier nothing completes (1: in the
  // single-CTA GEMMs, 2: in all of them)
  unsigned long long tc_wait_ns = 1000000000ull;
  int tc_stall = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  gm_job* job = nullptr;        // workspace of gmmnlse_propagate
  std::mutex mu;
};


// ---------------------------------------------------------------------------
// Launch as a programmatic dependent of the previous kernel in the stream
// (kernels start with pdl_enter), unless GMMNLSE_NO_PDL=1.
// ---------------------------------------------------------------------------
static inline bool pdl_disabled() {
  static const bool off = [] {
    const char* v = getenv("GMMNLSE_NO_PDL");
    return v && v[0] == '1';
  }();
  return off;
}

// cluster > 1 groups consecutive blocks along x into thread-block clusters.
template <typename... KArgs, typename... Args>
static inline void pdl_launch_cl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                 int cluster, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[2];
  int na = 0;
  if (!pdl_disabled()) {
    at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cluster > 1) {
    at[na].id = cudaLaunchAttributeClusterDimension;
    at[na].val.clusterDim.x = (unsigned)cluster;
    at[na].val.clusterDim.y = 1;
    at[na].val.clusterDim.z = 1;
    ++na;
  }
  cfg.attrs = at;
  cfg.numAttrs = na;
  cudaLaunchKernelEx(&cfg, kern, args...);
}

template <typename... KArgs, typename... Args>
static inline void pdl_launch(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  pdl_launch_cl(kern, grid, block, smem, s, 1, args...);
}

// ---------------------------------------------------------------------------
// Coupling contraction launch: registers for N <= 8, shared memory otherwise
// ---------------------------------------------------------------------------
template <typename R, int N, int MODE>
static inline void launch_contract_reg(const gm::Geo& g, const gmmnlse_ctx* c, const void* A, const void* V,
                                       void* NL, const gm::LoopState* ls, cudaStream_t s) {
  const size_t pts = (size_t)g.B * (g.M + 1) * g.n;
  pdl_launch(gm::k_contract_reg<R, N, MODE>, dim3((unsigned)((pts + 127) / 128)), dim3(128), 0, s, g,
             (const gm::cplx<R>*)A, (const R*)V, (const R*)c->G, (gm::cplx<R>*)NL, ls);
}

template <typename R, int N>
static inline void launch_contract_n(const gm::Geo& g, const gmmnlse_ctx* c, const void* A, const void* V, void* NL,
                                     const gm::LoopState* ls, cudaStream_t s) {
  if (c->raman_mode == 0) launch_contract_reg<R, N, 0>(g, c, A, V, NL, ls, s);
  else if (c->raman_mode == 1) launch_contract_reg<R, N, 1>(g, c, A, V, NL, ls, s);
  else launch_contract_reg<R, N, 2>(g, c, A, V, NL, ls, s);
}

// false if the launch was refused (the caller then launches k_contract_reg)
bool gm_nz_launch(const gmmnlse_ctx* c, const gm::Geo& g, const void* A, const void* V, void* NL,
                  const gm::LoopState* ls, cudaStream_t s);

template <typename R>
static inline void launch_contract(const gm::Geo& g, const gmmnlse_ctx* c, const void* A, const void* V, void* NL,
                                   const gm::LoopState* ls, cudaStream_t s) {
  // N <= 8: the kernel compiled for this context's nonzero coupling entries
  if (c->nz_fn && gm_nz_launch(c, g, A, V, NL, ls, s)) return;
  switch (c->N) {
    case 1: launch_contract_n<R, 1>(g, c, A, V, NL, ls, s); return;
    case 2: launch_contract_n<R, 2>(g, c, A, V, NL, ls, s); return;
    case 3: launch_contract_n<R, 3>(g, c, A, V, NL, ls, s); return;
    case 4: launch_contract_n<R, 4>(g, c, A, V, NL, ls, s); return;
    case 5: launch_contract_n<R, 5>(g, c, A, V, NL, ls, s); return;
    case 6: launch_contract_n<R, 6>(g, c, A, V, NL, ls, s); return;
    case 7: launch_contract_n<R, 7>(g, c, A, V, NL, ls, s); return;
    case 8: launch_contract_n<R, 8>(g, c, A, V, NL, ls, s); return;
    default: {
      gm::TileArgs<R> a = {};
      a.A = (const gm::cplx<R>*)A;
      a.Ys = (const R*)V;
      a.Gt = (const R*)c->Gt;
      a.KK = c->KK;
      a.KKp = c->KKt;
      a.Pp = c->Pt;
      a.rows = c->P;
      a.cnt = c->K;
      a.rowpl = (const int2*)c->rows_t;
      a.pairs = (const int2*)c->pairs;
      a.NL = (gm::cplx<R>*)NL;
      const size_t pts = (size_t)g.B * (g.M + 1) * g.n;
      const dim3 grid((unsigned)((pts + gm::TileCfg<R>::TP - 1) / gm::TileCfg<R>::TP));
      const size_t smem = gm::contract_tile_smem<R>(c->N);
      auto go = [&](auto kern) { pdl_launch(kern, grid, dim3(256), smem, s, g, a, ls); };
      if (c->raman_mode == 0) go(gm::k_contract_tile<R, 0, 0, 0>);
      else if (c->raman_mode == 1) go(gm::k_contract_tile<R, 1, 0, 0>);
      else go(gm::k_contract_tile<R, 2, 0, 0>);
    }
  }
}
