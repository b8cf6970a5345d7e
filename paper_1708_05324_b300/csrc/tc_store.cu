// Tensor-core GEMM with the store epilogue (the first GEMM of the low-rank
// coupling, tc_contract.cuh) instantiated for row blocks of 16..256 rows,
// 16-bit and TF32 operands; and the dispatch over every tensor-core GEMM
// translation unit.
#include "tc_launch.cuh"

#define GM_TC_STORE_CASE(NB)                                         \
  case NB:                                                           \
    if (L.tf32) gm_tc::launch_one<0, NB, 1, 4>(L);                    \
    else gm_tc::launch_one<0, NB, 1, 2>(L);                           \
    return true;
#define GM_TC_STORE_SETUP(NB)                                                                        \
  if (gm_tc::setup_one<0, NB, 1, 4>(smax) || gm_tc::setup_one<0, NB, 1, 2>(smax)) return -1;

bool gm_tc_store(int NB, const TcLaunch& L) {
  switch (NB) {
    GM_TC_STORE_CASE(16) GM_TC_STORE_CASE(32) GM_TC_STORE_CASE(48) GM_TC_STORE_CASE(64)
    GM_TC_STORE_CASE(80) GM_TC_STORE_CASE(96) GM_TC_STORE_CASE(112) GM_TC_STORE_CASE(128)
    GM_TC_STORE_CASE(144) GM_TC_STORE_CASE(160) GM_TC_STORE_CASE(176) GM_TC_STORE_CASE(192)
    GM_TC_STORE_CASE(208) GM_TC_STORE_CASE(224) GM_TC_STORE_CASE(240) GM_TC_STORE_CASE(256)
    default:
      return false;
  }
}

#define GM_TC_PARTS(X) X(a) X(b) X(c) X(d) X(e) X(f) X(g) X(h) X(i)
#define GM_TC_DECL(x)                                 \
  bool gm_tc_lsum_##x(int N, const TcLaunch& L);      \
  int gm_tc_setup_lsum_##x(int smax);
GM_TC_PARTS(GM_TC_DECL)

bool gm_tc_lsum(int N, const TcLaunch& L) {
#define GM_TC_TRY(x) \
  if (gm_tc_lsum_##x(N, L)) return true;
  GM_TC_PARTS(GM_TC_TRY)
  return false;
}

int gm_tc_setup(int smax) {
  GM_TC_STORE_SETUP(16) GM_TC_STORE_SETUP(32) GM_TC_STORE_SETUP(48) GM_TC_STORE_SETUP(64)
  GM_TC_STORE_SETUP(80) GM_TC_STORE_SETUP(96) GM_TC_STORE_SETUP(112) GM_TC_STORE_SETUP(128)
  GM_TC_STORE_SETUP(144) GM_TC_STORE_SETUP(160) GM_TC_STORE_SETUP(176) GM_TC_STORE_SETUP(192)
  GM_TC_STORE_SETUP(208) GM_TC_STORE_SETUP(224) GM_TC_STORE_SETUP(240) GM_TC_STORE_SETUP(256)
#define GM_TC_SET(x) \
  if (gm_tc_setup_lsum_##x(smax)) return -1;
  GM_TC_PARTS(GM_TC_SET)
  return 0;
}
