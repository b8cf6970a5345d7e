// Launch and set-up helpers of one tensor-core GEMM instantiation, used by
// the translation units that instantiate them (tc_lsum_*.cu, tc_store.cu).
#pragma once

#include <algorithm>
#include <map>
#include <mutex>

#include "ctx.h"
#include "tc_gemm.h"

namespace gm_tc {

using namespace gm;

// CTAs of a tensor-core GEMM launch: CL x the clusters resident at once
// (cudaOccupancyMaxActiveClusters, once per kernel), at most one cluster per
// work item of CL x TPW point tiles.  A grid of more clusters than fit would
// run the surplus as a second wave.
static int tc_grid(const void* kern, size_t smem, int cl, int tpw, int ntiles, int threads) {
  static std::mutex mu;
  static std::map<const void*, int> resident;
  int maxc = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = resident.find(kern);
    if (it != resident.end()) {
      maxc = it->second;
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(148 / cl * cl);
      cfg.blockDim = dim3(threads);
      cfg.dynamicSmemBytes = smem;
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = (unsigned)cl;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      if (cudaOccupancyMaxActiveClusters(&maxc, kern, &cfg) != cudaSuccess || maxc <= 0) {
        (void)cudaGetLastError();
        maxc = 148 / cl / 2;  // a safe guess: half the SMs
      }
      resident[kern] = maxc;
    }
  }
  const int items = (ntiles + cl * tpw - 1) / (cl * tpw);
  return cl * std::max(1, std::min(items, maxc));
}

template <int N, int NB, int OUT, int ES>
static void launch_one(const TcLaunch& L) {
  using Sh = TcShape<N, NB, ES, OUT>;
  auto kern = k_tc_contract<N, NB, OUT, ES>;
  const dim3 grid(tc_grid((const void*)kern, Sh::SMEM, Sh::CL, Sh::TPW, L.ntiles, Sh::THREADS));
  pdl_launch_cl(kern, grid, dim3(Sh::THREADS), Sh::SMEM, L.s, Sh::CL, *L.vhi, *L.vlo, *L.ghi, *L.glo, L.a, L.ls);
}

template <int N, int NB, int OUT, int ES>
static int setup_one(int smax) {
  auto kern = k_tc_contract<N, NB, OUT, ES>;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return -1;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smax - (int)fa.sharedSizeBytes) !=
      cudaSuccess)
    return -1;
  return 0;
}

}  // namespace gm_tc

// The l-sum GEMM of N modes, both operand widths: a case of a switch over N
// in launch functions, and a line of a set-up function.
#define GM_TC_LSUM_CASE(NN)                                                                  \
  case NN:                                                                                   \
    if (L.tf32) gm_tc::launch_one<NN, gm::tc_row_block(NN * (NN + 1) / 2), 0, 4>(L);         \
    else gm_tc::launch_one<NN, gm::tc_row_block(NN * (NN + 1) / 2), 0, 2>(L);                \
    return true;
#define GM_TC_LSUM_SETUP(NN)                                                                   \
  if (gm_tc::setup_one<NN, gm::tc_row_block(NN * (NN + 1) / 2), 0, 4>(smax) ||                 \
      gm_tc::setup_one<NN, gm::tc_row_block(NN * (NN + 1) / 2), 0, 2>(smax))                   \
    return -1;
