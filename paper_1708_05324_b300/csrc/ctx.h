// Layout of a context and of a propagation workspace, shared by the host-side
// translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <mutex>

#include "../../include/gmmnlse.h"
#include "kernels.cuh"

// ---------------------------------------------------------------------------
// Workspace of one propagation in flight
// ---------------------------------------------------------------------------
struct gm_job {
  gmmnlse_ctx* ctx = nullptr;
  int Mcap = 0;
  double2* psi0 = nullptr;  // [N][n]
  void* dpsi = nullptr;     // [M][N][n]
  void* A = nullptr;        // [M+1][N][n]
  void* V = nullptr;        // [M+1][KK][n]
  void* NL = nullptr;       // [M+1][N][n]
  void* I = nullptr;        // [M+1][N][n]
  void* E = nullptr;        // [M+1][N][n]
  double2* EM64 = nullptr;  // [2][N][n]
  double2* io = nullptr;    // [2][N][n] staging / FP64 FFT scratch
  int* flag = nullptr;
  gm::LoopState* ls = nullptr;      // device
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
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
  } graphs[2];
  size_t bytes = 0;
};

struct gmmnlse_ctx {
  gmmnlse_params prm;
  int N, n, K, P, KK, raman_mode, ept;
  bool fp64;
  double fR, omega0, gamma0;
  double* beta = nullptr;       // [N][n]
  double2* tw64 = nullptr;      // [n]
  double2* tw64h = nullptr;     // [n/2]
  float2* tw32 = nullptr;       // [n]
  void* H = nullptr;            // [n] cplx<R>
  void* G = nullptr;            // [P][KK] R
  int2* rows = nullptr;         // [P]
  int2* pairs = nullptr;        // [K]
  int contract_threads = 128;
  size_t contract_smem = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  gm_job* job = nullptr;        // workspace of gmmnlse_propagate
  std::mutex mu;
};

