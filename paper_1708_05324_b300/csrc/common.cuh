// Shared device helpers: complex arithmetic on float2/double2, reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gm {

template <typename R> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <typename R> using cplx = typename C2<R>::type;

template <typename R> __host__ __device__ __forceinline__ cplx<R> mk(R x, R y) {
  cplx<R> c; c.x = x; c.y = y; return c;
}
template <typename R> __device__ __forceinline__ cplx<R> cadd(cplx<R> a, cplx<R> b) {
  return mk<R>(a.x + b.x, a.y + b.y);
}
template <typename R> __device__ __forceinline__ cplx<R> csub(cplx<R> a, cplx<R> b) {
  return mk<R>(a.x - b.x, a.y - b.y);
}
template <typename R> __device__ __forceinline__ cplx<R> cmul(cplx<R> a, cplx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename R> __device__ __forceinline__ cplx<R> cmulc(cplx<R> a, cplx<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename R> __device__ __forceinline__ cplx<R> cscale(cplx<R> a, R s) {
  return mk<R>(a.x * s, a.y * s);
}
// multiply by +i (DIR = +1) or -i (DIR = -1)
template <typename R, int DIR> __device__ __forceinline__ cplx<R> mul_i(cplx<R> a) {
  return DIR > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x);
}
template <typename R> __device__ __forceinline__ R cabs2(cplx<R> a) { return a.x * a.x + a.y * a.y; }
template <typename R, typename S> __device__ __forceinline__ cplx<R> ccast(S a) {
  return mk<R>((R)a.x, (R)a.y);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sum of v over the block; the result is valid in thread 0.  scratch: 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* scratch) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? scratch[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}

}  // namespace gm
