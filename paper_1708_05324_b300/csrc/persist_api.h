// Host interface of the opt-in cooperative long-step kernel (persist.cuh),
// instantiated in its own translation units (persist_fp32.cu,
// persist_fp64.cu) for N <= 8 modes.
#pragma once

#include <cuda_runtime.h>

#include "ctx.h"

struct gm_job;

// Shared-memory attributes of every instantiation (once per device).
template <typename R> int persist_setup(int smax);
// Blocks of the long-step kernel for this job (every block resident), or 0
// where it does not apply (the default: GMMNLSE_PERSIST=1 enables it).
template <typename R> int long_step_grid(gm_job* jb);
// Zero the barrier counter, then the cooperative long-step kernel.
template <typename R>
void launch_long_step(gm_job* jb, const gm::Geo& g, int which, cudaStream_t s, cudaGraphConditionalHandle hStep,
                      int use_cond);
