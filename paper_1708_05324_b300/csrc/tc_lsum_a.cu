// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 9..16 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_a(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(9)
    GM_TC_LSUM_CASE(10)
    GM_TC_LSUM_CASE(11)
    GM_TC_LSUM_CASE(12)
    GM_TC_LSUM_CASE(13)
    GM_TC_LSUM_CASE(14)
    GM_TC_LSUM_CASE(15)
    GM_TC_LSUM_CASE(16)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_a(int smax) {
  GM_TC_LSUM_SETUP(9)
  GM_TC_LSUM_SETUP(10)
  GM_TC_LSUM_SETUP(11)
  GM_TC_LSUM_SETUP(12)
  GM_TC_LSUM_SETUP(13)
  GM_TC_LSUM_SETUP(14)
  GM_TC_LSUM_SETUP(15)
  GM_TC_LSUM_SETUP(16)
  return 0;
}
