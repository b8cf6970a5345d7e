// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 57..60 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_h(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(57)
    GM_TC_LSUM_CASE(58)
    GM_TC_LSUM_CASE(59)
    GM_TC_LSUM_CASE(60)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_h(int smax) {
  GM_TC_LSUM_SETUP(57)
  GM_TC_LSUM_SETUP(58)
  GM_TC_LSUM_SETUP(59)
  GM_TC_LSUM_SETUP(60)
  return 0;
}
