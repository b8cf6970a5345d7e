// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 61..64 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_i(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(61)
    GM_TC_LSUM_CASE(62)
    GM_TC_LSUM_CASE(63)
    GM_TC_LSUM_CASE(64)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_i(int smax) {
  GM_TC_LSUM_SETUP(61)
  GM_TC_LSUM_SETUP(62)
  GM_TC_LSUM_SETUP(63)
  GM_TC_LSUM_SETUP(64)
  return 0;
}
