// Host interface of the tensor-core GEMMs of the coupling contraction
// (tc_contract.cuh), whose instantiations live in their own translation
// units (tc_lsum_*.cu: the l-sum epilogue for N = 9..64 modes; tc_store.cu:
// the store epilogue for row blocks of 16..256 rows), each for 16-bit
// (BF16 / FP16) and TF32 operands.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "tc_contract.cuh"

struct TcLaunch {
  const CUtensorMap *vhi, *vlo, *ghi, *glo;  // V operand (hi, lo) and coupling operand (hi, lo)
  gm::TcArgs a;
  const gm::LoopState* ls;
  cudaStream_t s;
  int ntiles;  // 128-point tiles of the launch
  bool tf32;   // TF32 operands (else BF16 / FP16)
};

constexpr int TC_MIN_N = 9, TC_MAX_N = 64;

// The GEMM with the l-sum epilogue for N modes, TC_MIN_N <= N <= TC_MAX_N
// (false for any other N: nothing launched).
bool gm_tc_lsum(int N, const TcLaunch& L);
// The GEMM with the store epilogue and row blocks of NB rows, NB a multiple
// of 16 in 16..256 (false otherwise).
bool gm_tc_store(int NB, const TcLaunch& L);
// Raise the dynamic shared-memory limit of every tensor-core GEMM kernel to
// what the device allows beside its static shared memory (once per device).
int gm_tc_setup(int smax);
