// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 35..40 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_d(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(35)
    GM_TC_LSUM_CASE(36)
    GM_TC_LSUM_CASE(37)
    GM_TC_LSUM_CASE(38)
    GM_TC_LSUM_CASE(39)
    GM_TC_LSUM_CASE(40)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_d(int smax) {
  GM_TC_LSUM_SETUP(35)
  GM_TC_LSUM_SETUP(36)
  GM_TC_LSUM_SETUP(37)
  GM_TC_LSUM_SETUP(38)
  GM_TC_LSUM_SETUP(39)
  GM_TC_LSUM_SETUP(40)
  return 0;
}
