// Tensor-core GEMM with the l-sum epilogue (tc_contract.cuh) instantiated for
// N = 47..51 modes, 16-bit and TF32 operands.
#include "tc_launch.cuh"

bool gm_tc_lsum_f(int N, const TcLaunch& L) {
  switch (N) {
    GM_TC_LSUM_CASE(47)
    GM_TC_LSUM_CASE(48)
    GM_TC_LSUM_CASE(49)
    GM_TC_LSUM_CASE(50)
    GM_TC_LSUM_CASE(51)
    default:
      return false;
  }
}

int gm_tc_setup_lsum_f(int smax) {
  GM_TC_LSUM_SETUP(47)
  GM_TC_LSUM_SETUP(48)
  GM_TC_LSUM_SETUP(49)
  GM_TC_LSUM_SETUP(50)
  GM_TC_LSUM_SETUP(51)
  return 0;
}
