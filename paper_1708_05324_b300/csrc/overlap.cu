// gmmnlse_overlap_tensor: the mode overlap tensor S_plmn of Eq. 2 from mode
// profiles sampled on a grid, on the GPU.
//
// S_plmn = int F_p F_l F_m F_n dA / sqrt(int F_p^2 dA ... int F_n^2 dA).  The
// numerator is the Gram matrix of the pair products P_k = F_m F_n (k = (m <= n),
// K = N(N+1)/2 of them) over the G grid cells, Gram[k1][k2] = sum_g P_k1 P_k2,
// so one FP64 GEMM [K x G] x [G x K] gives every distinct value; the host
// spreads them over the N^4 entries with the norms.  For the 42-mode step-index
// fiber on a 400^2 grid this is 903^2 x 160000 multiply-adds, about 0.13 TFLOP
// of FP64 on the CUDA cores (the tensor cores' FP64 rate is no faster on this
// part, and 16-bit operands would not hold the 1e-12 the FP64 path needs).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/gmmnlse.h"
#include "engine.h"

namespace {

constexpr int kTile = 64;   // Gram tile: 64 x 64 pair rows
constexpr int kChunk = 16;  // grid cells staged per step

// Gram tiles on and above the diagonal (the matrix is symmetric); each of
// the 256 threads owns a 4 x 4 block of the tile.  The pair products are
// formed while a chunk of cells is staged in shared memory.
__global__ void __launch_bounds__(256) k_overlap_gram(const double* __restrict__ F, long long G,
                                                      const int2* __restrict__ pairs, int K,
                                                      double* __restrict__ gram) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double a[kChunk][kTile + 1], b[kChunk][kTile + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.x * kTile, c0 = blockIdx.y * kTile;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (long long g0 = 0; g0 < G; g0 += kChunk) {
    for (int idx = threadIdx.x; idx < kChunk * kTile; idx += blockDim.x) {
      const int r = idx >> 4, c = idx & 15;
      const long long g = g0 + c;
      double va = 0.0, vb = 0.0;
      if (g < G) {
        if (r0 + r < K) {
          const int2 mn = pairs[r0 + r];
          va = F[mn.x * G + g] * F[mn.y * G + g];
        }
        if (c0 + r < K) {
          const int2 mn = pairs[c0 + r];
          vb = F[mn.x * G + g] * F[mn.y * G + g];
        }
      }
      a[c][r] = va;
      b[c][r] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kChunk; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        av[i] = a[kk][ty * 4 + i];
        bv[i] = b[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = r0 + ty * 4 + i, c = c0 + tx * 4 + j;
      if (r < K && c < K) gram[(size_t)r * K + c] = acc[i][j];
    }
}

// sum_g F_p(g)^2 per profile (one block per p, fixed reduction order)
__global__ void __launch_bounds__(256) k_row_squares(const double* __restrict__ F, long long G,
                                                     double* __restrict__ out) {
  __shared__ double part[256];
  const double* row = F + (long long)blockIdx.x * G;
  double s = 0.0;
  for (long long g = threadIdx.x; g < G; g += blockDim.x) s = fma(row[g], row[g], s);
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = part[0];
}

}  // namespace

extern "C" int gmmnlse_overlap_tensor(int device, const double* F, int N, long long G, double dA, double* S) {
  if (!F || !S || N < 1 || N > 64 || G < 1 || !(dA > 0) || !std::isfinite(dA)) return GMMNLSE_E_INVALID;
  const size_t NG = (size_t)N * (size_t)G;
  for (size_t i = 0; i < NG; ++i)
    if (!std::isfinite(F[i])) return GMMNLSE_E_INVALID;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return GMMNLSE_E_INVALID;
  }
  auto gate = gm_gate_device(device);
  const int K = N * (N + 1) / 2;
  std::vector<int2> pairs;
  std::vector<int> kof((size_t)N * N);
  for (int m = 0; m < N; ++m)
    for (int n = m; n < N; ++n) {
      kof[(size_t)m * N + n] = kof[(size_t)n * N + m] = (int)pairs.size();
      pairs.push_back(make_int2(m, n));
    }
  double *dF = nullptr, *dGram = nullptr, *dSq = nullptr;
  int2* dPairs = nullptr;
  cudaStream_t s = nullptr;
  int rc = GMMNLSE_OK;
  auto fail = [&](int code) {
    cudaGetLastError();
    rc = code;
  };
  if (cudaMalloc(&dF, NG * sizeof(double)) != cudaSuccess || cudaMalloc(&dGram, (size_t)K * K * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&dSq, N * sizeof(double)) != cudaSuccess || cudaMalloc(&dPairs, K * sizeof(int2)) != cudaSuccess)
    fail(GMMNLSE_E_NOMEM);
  if (!rc && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) fail(GMMNLSE_E_CUDA);
  std::vector<double> gram, sq(N);
  if (!rc) {
    const int nb = (K + kTile - 1) / kTile;
    if (cudaMemcpyAsync(dF, F, NG * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dPairs, pairs.data(), K * sizeof(int2), cudaMemcpyHostToDevice, s) != cudaSuccess) {
      fail(GMMNLSE_E_CUDA);
    } else {
      k_overlap_gram<<<dim3(nb, nb), 256, 0, s>>>(dF, G, dPairs, K, dGram);
      k_row_squares<<<N, 256, 0, s>>>(dF, G, dSq);
      gram.resize((size_t)K * K);
      if (cudaGetLastError() != cudaSuccess ||
          cudaMemcpyAsync(gram.data(), dGram, gram.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaMemcpyAsync(sq.data(), dSq, N * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess)
        fail(GMMNLSE_E_CUDA);
    }
  }
  if (s) cudaStreamDestroy(s);
  cudaFree(dF);
  cudaFree(dGram);
  cudaFree(dSq);
  cudaFree(dPairs);
  if (rc) return rc;
  // spread: the kernel wrote the tiles with row block <= column block
  std::vector<double> inv(N);
  for (int p = 0; p < N; ++p) {
    if (!(sq[p] > 0)) return GMMNLSE_E_INVALID;  // a zero profile has no normalisation
    inv[p] = 1.0 / std::sqrt(sq[p] * dA);
  }
  auto g = [&](int k1, int k2) {
    return (k1 / kTile <= k2 / kTile) ? gram[(size_t)k1 * K + k2] : gram[(size_t)k2 * K + k1];
  };
  for (int p = 0; p < N; ++p)
    for (int l = 0; l < N; ++l)
      for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n)
          S[(((size_t)p * N + l) * N + m) * N + n] =
              g(kof[(size_t)p * N + l], kof[(size_t)m * N + n]) * dA * inv[p] * inv[l] * inv[m] * inv[n];
  return GMMNLSE_OK;
}
