// The opt-in cooperative long-step kernel (persist.cuh) for double iterates.
#include "persist_impl.cuh"

GM_PERSIST_INSTANTIATE(double)
