// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 41..46 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_e(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(41)
    GM_TC_LSUM_CASE(42)
    GM_TC_LSUM_CASE(43)
    GM_TC_LSUM_CASE(44)
    GM_TC_LSUM_CASE(45)
    GM_TC_LSUM_CASE(46)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_e(int smax) {
  GM_TC_LSUM_SETUP(41)
  GM_TC_LSUM_SETUP(42)
  GM_TC_LSUM_SETUP(43)
  GM_TC_LSUM_SETUP(44)
  GM_TC_LSUM_SETUP(45)
  GM_TC_LSUM_SETUP(46)
  return 0;
}
