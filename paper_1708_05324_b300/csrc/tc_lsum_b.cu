// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 17..26 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_b(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(17)
    GM_TC_LSUM_CASE(18)
    GM_TC_LSUM_CASE(19)
    GM_TC_LSUM_CASE(20)
    GM_TC_LSUM_CASE(21)
    GM_TC_LSUM_CASE(22)
    GM_TC_LSUM_CASE(23)
    GM_TC_LSUM_CASE(24)
    GM_TC_LSUM_CASE(25)
    GM_TC_LSUM_CASE(26)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_b(int smax) {
  GM_TC_LSUM_SETUP(17)
  GM_TC_LSUM_SETUP(18)
  GM_TC_LSUM_SETUP(19)
  GM_TC_LSUM_SETUP(20)
  GM_TC_LSUM_SETUP(21)
  GM_TC_LSUM_SETUP(22)
  GM_TC_LSUM_SETUP(23)
  GM_TC_LSUM_SETUP(24)
  GM_TC_LSUM_SETUP(25)
  GM_TC_LSUM_SETUP(26)
  return 0;
}
