// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 27..34 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_c(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(27)
    GM_TC_LSUM_CASE(28)
    GM_TC_LSUM_CASE(29)
    GM_TC_LSUM_CASE(30)
    GM_TC_LSUM_CASE(31)
    GM_TC_LSUM_CASE(32)
    GM_TC_LSUM_CASE(33)
    GM_TC_LSUM_CASE(34)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_c(int smax) {
  GM_TC_LSUM_SETUP(27)
  GM_TC_LSUM_SETUP(28)
  GM_TC_LSUM_SETUP(29)
  GM_TC_LSUM_SETUP(30)
  GM_TC_LSUM_SETUP(31)
  GM_TC_LSUM_SETUP(32)
  GM_TC_LSUM_SETUP(33)
  GM_TC_LSUM_SETUP(34)
  return 0;
}
