// The opt-in cooperative long-step kernel (persist.cuh) for float iterates.
#include "persist_impl.cuh"

GM_PERSIST_INSTANTIATE(float)
