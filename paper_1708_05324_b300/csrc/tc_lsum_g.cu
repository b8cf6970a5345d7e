// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 52..56 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_g(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(52)
    GM_TC_LSUM_CASE(53)
    GM_TC_LSUM_CASE(54)
    GM_TC_LSUM_CASE(55)
    GM_TC_LSUM_CASE(56)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_g(int smax) {
  GM_TC_LSUM_SETUP(52)
  GM_TC_LSUM_SETUP(53)
  GM_TC_LSUM_SETUP(54)
  GM_TC_LSUM_SETUP(55)
  GM_TC_LSUM_SETUP(56)
  return 0;
}
