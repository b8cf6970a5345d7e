// Host side of the MPA solver: contexts (fiber data on the device), per-
// propagation workspaces, and the long-step driver (Sec. III.D).
//
// One long step is the kernel chain K1 -> K2 -> K3 -> K4 -> K5 repeated until
// K5's last block decides that the iteration has converged, followed by K6.
// The repetition is a CUDA-graph while-node whose condition K5 sets on the
// device, and the long steps themselves are an outer while-node that K6
// re-arms, so a whole fiber is one graph launch with no host round trip per
// iteration.  A host-driven loop over the same kernels is kept for graphs
// that fail to build (and for debugging, GMMNLSE_NO_GRAPH=1).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <condition_variable>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/gmmnlse.h"
#include "engine.h"
#include "kernels.cuh"
#include "ctx.h"
#include "tc_contract.cuh"
#include "tc_gemm.h"

using namespace gm;

#define CK(call)                                                        \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                            \
      gm_set_last_cuda_error(e_, #call, __FILE__, __LINE__);            \
      return GMMNLSE_E_CUDA;                                            \
    }                                                                   \
  } while (0)

static thread_local char g_last_err[512];

void gm_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_err, sizeof g_last_err, "%s at %s:%d: %s", cudaGetErrorString(e), file, line, what);
  if (getenv("GMMNLSE_VERBOSE")) fprintf(stderr, "gmmnlse: %s\n", g_last_err);
}

extern "C" const char* gmmnlse_last_error(void) { return g_last_err; }

void gm_set_last_error_text(const char* msg) { snprintf(g_last_err, sizeof g_last_err, "%s", msg); }

namespace {

constexpr int kMaxN = 64;
constexpr int kMaxM = 64;

int ept_for(int n, bool fp64) {
  (void)fp64;
  return n > 8192 ? 32 : 16;
}

template <typename R> size_t fft_smem(int n) { return (size_t)fft_smem_elems(n) * sizeof(cplx<R>); }

}  // namespace

// ---------------------------------------------------------------------------
// Helpers
// ---------------------------------------------------------------------------
static int set_device(int dev) {
  CK(cudaSetDevice(dev));
  return GMMNLSE_OK;
}

// Forward (DIR +1, unscaled) or inverse (DIR -1, scale) FP64 transform of the
// N rows of a [N][n] field.  n = 16384 goes through two half-length
// transforms and a combination step (the full FP64 transform would not fit
// in one block's shared memory).
static int fft64(gmmnlse_ctx* c, double2* scratch, const double2* in, double2* out, int rows, int dir,
                 double scale, cudaStream_t s) {
  const int n = c->n;
  if (n <= 8192) {
    const int ept = 16;
    const size_t sm = fft_smem<double>(n);
    if (dir > 0) k_fft64_rows<+1, 16><<<rows, n / ept, sm, s>>>(in, out, n, scale, c->tw64);
    else k_fft64_rows<-1, 16><<<rows, n / ept, sm, s>>>(in, out, n, scale, c->tw64);
  } else {
    const int h = n / 2;
    const size_t sm = fft_smem<double>(h);
    dim3 grid(rows, 2);
    if (dir > 0) {
      k_fft64_halves<+1, 16><<<grid, h / 16, sm, s>>>(in, scratch, n, c->tw64h);
      k_fft64_combine<+1><<<(rows * n + 255) / 256, 256, 0, s>>>(scratch, out, rows, n, scale, c->tw64);
    } else {
      k_fft64_halves<-1, 16><<<grid, h / 16, sm, s>>>(in, scratch, n, c->tw64h);
      k_fft64_combine<-1><<<(rows * n + 255) / 256, 256, 0, s>>>(scratch, out, rows, n, scale, c->tw64);
    }
  }
  CK(cudaGetLastError());
  return GMMNLSE_OK;
}

// The dynamic shared-memory limit is a property of each kernel function on
// the device, shared by every context, so it is raised once to the device's
// opt-in maximum (this reserves nothing; each launch asks for what it uses).
// The iteration kernels are set up by their own translation units.
static int set_smem_attrs(gmmnlse_ctx* c) {
  int sm = 0;
  CK(cudaDeviceGetAttribute(&sm, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->prm.device));
  CK(cudaFuncSetAttribute(k_fft64_rows<+1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fft64_rows<-1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fft64_halves<+1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  CK(cudaFuncSetAttribute(k_fft64_halves<-1, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm));
  return c->fp64 ? gm_prop_setup_f64(c->prm.device) : gm_prop_setup_f32(c->prm.device);
}

// ---------------------------------------------------------------------------
// Context creation
// ---------------------------------------------------------------------------
static bool finite_all(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

// S real with S_plmn = S_plnm = S_lpmn (Eq. 2 gives full symmetry).
static bool symmetric_enough(const double* S, int N) {
  double mx = 0.0;
  const size_t tot = (size_t)N * N * N * N;
  for (size_t i = 0; i < tot; ++i) mx = std::max(mx, std::fabs(S[i]));
  const double tol = 1e-12 * (mx > 0 ? mx : 1.0);
  auto at = [&](int p, int l, int m, int n) { return S[(((size_t)p * N + l) * N + m) * N + n]; };
  for (int p = 0; p < N; ++p)
    for (int l = 0; l < N; ++l)
      for (int m = 0; m < N; ++m)
        for (int n = 0; n < N; ++n) {
          const double v = at(p, l, m, n);
          if (std::fabs(v - at(p, l, n, m)) > tol) return false;
          if (std::fabs(v - at(l, p, m, n)) > tol) return false;
        }
  return true;
}

static void free_job(gm_job* jb);

static void free_ctx(gmmnlse_ctx* c) {
  if (!c) return;
  if (c->job) free_job(c->job);
  cudaFree(c->beta);
  cudaFree(c->Q);
  cudaFree(c->gain);
  cudaFree(c->fprof);
  cudaFree(c->GRt);
  cudaFree(c->tw64);
  cudaFree(c->tw64h);
  cudaFree(c->tw32);
  cudaFree(c->H);
  cudaFree(c->Hv);
  cudaFree(c->fac);
  cudaFree(c->G);
  cudaFree(c->Gt);
  cudaFree(c->rows);
  cudaFree(c->rows_t);
  cudaFree(c->pairs);
  gm_nz_free(c);
  cudaFree(c->ublk);
  cudaFree(c->gpairs);
  cudaFree(c->Ghi);
  cudaFree(c->Wt);
  cudaFree(c->Xt);
  cudaFree(c->Whi);
  cudaFree(c->Wlo);
  cudaFree(c->Xhi);
  cudaFree(c->Xlo);
  cudaFree(c->Glo);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

// Rank-revealing factorisation G = X W of the reduced coupling matrix
// (P x K, row-major): Gram-Schmidt with column pivoting, each new direction
// orthogonalised twice.  X (P x r) has orthonormal columns and W = X^T G
// (r x K), so G - X W is the residual of the projection onto the span of X,
// whose columns are all below tol x the largest column of G.  (The pair
// matrix of S is a Gram matrix of mode products F_p F_l, which are linearly
// dependent for the fibres here, so r < K exactly.)
static int lowrank(const std::vector<double>& G, int P, int K, double tol, std::vector<double>& X,
                   std::vector<double>& W) {
  std::vector<double> Rm((size_t)P * K);  // residual, column-major
  for (int p = 0; p < P; ++p)
    for (int k = 0; k < K; ++k) Rm[(size_t)k * P + p] = G[(size_t)p * K + k];
  auto colnorm2 = [&](int k) {
    double a = 0.0;
    for (int p = 0; p < P; ++p) a += Rm[(size_t)k * P + p] * Rm[(size_t)k * P + p];
    return a;
  };
  double n0 = 0.0;
  for (int k = 0; k < K; ++k) n0 = std::max(n0, colnorm2(k));
  std::vector<double> Q;  // columns of X, column-major
  int r = 0;
  while (r < std::min(P, K) && n0 > 0.0) {
    int c = 0;
    double best = -1.0;
    for (int k = 0; k < K; ++k) {
      const double a = colnorm2(k);
      if (a > best) {
        best = a;
        c = k;
      }
    }
    if (!(best > tol * tol * n0)) break;
    std::vector<double> q(Rm.begin() + (size_t)c * P, Rm.begin() + (size_t)(c + 1) * P);
    for (int pass = 0; pass < 2; ++pass) {
      for (int s = 0; s < r; ++s) {
        double d = 0.0;
        for (int p = 0; p < P; ++p) d += Q[(size_t)s * P + p] * q[p];
        for (int p = 0; p < P; ++p) q[p] -= d * Q[(size_t)s * P + p];
      }
      double nq = 0.0;
      for (int p = 0; p < P; ++p) nq += q[p] * q[p];
      nq = std::sqrt(nq);
      if (!(nq > 0.0)) return r;
      for (int p = 0; p < P; ++p) q[p] /= nq;
    }
    for (int k = 0; k < K; ++k) {
      double* col = &Rm[(size_t)k * P];
      double d = 0.0;
      for (int p = 0; p < P; ++p) d += q[p] * col[p];
      for (int p = 0; p < P; ++p) col[p] -= d * q[p];
    }
    Q.insert(Q.end(), q.begin(), q.end());
    ++r;
  }
  X.assign((size_t)P * r, 0.0);
  W.assign((size_t)r * K, 0.0);
  for (int s = 0; s < r; ++s)
    for (int p = 0; p < P; ++p) X[(size_t)p * r + s] = Q[(size_t)s * P + p];
  for (int s = 0; s < r; ++s)
    for (int k = 0; k < K; ++k) {
      double a = 0.0;
      for (int p = 0; p < P; ++p) a += Q[(size_t)s * P + p] * G[(size_t)p * K + k];
      W[(size_t)s * K + k] = a;
    }
  return r;
}

// 14 - e for the largest |x| below 2^e: the FP16 scale exponent that puts
// the largest entry below 2^14.
static int f16_exp(const std::vector<double>& m) {
  double a = 0.0;
  for (double x : m) a = std::max(a, std::fabs(x));
  if (!(a > 0.0)) return 0;
  int e;
  std::frexp(a, &e);
  return 14 - e;
}

// TF32 rounding of x (nearest, ties away from zero: the low 13 bits of the
// FP32 significand cleared), as the device's cvt.rna.tf32.f32 does.
static float tf32_rna(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float y;
  std::memcpy(&y, &u, 4);
  return y;
}

// A row-major [rows][cols] matrix scaled by 2^e, split into hi + lo in the
// row-grouped layout [rows_pad/8][cols_pad/EPC][8][EPC] (K-major core
// matrices of 8 rows x 16 bytes, the K chunks of one 8-row group adjacent)
// read by the tensor-core GEMM as its coupling operand, zero padding: TF32
// words (EPC 4) when tf32, else 16-bit FP16 (f16) or BF16 (EPC 8).
static inline size_t row_grouped(int r, int k, int cols_pad, int epc) {
  return (((size_t)(r / 8) * (cols_pad / epc) + k / epc) * 8 + r % 8) * epc + k % epc;
}

static int upload_hilo_tf32(const std::vector<double>& m, int rows, int cols, int rows_pad, int cols_pad,
                            __nv_bfloat16** hi, __nv_bfloat16** lo) {
  std::vector<float> gh((size_t)rows_pad * cols_pad), gl((size_t)rows_pad * cols_pad);
  for (int r = 0; r < rows_pad; ++r)
    for (int k = 0; k < cols_pad; ++k) {
      const float x = (r < rows && k < cols) ? (float)m[(size_t)r * cols + k] : 0.f;
      const size_t o = row_grouped(r, k, cols_pad, 4);
      gh[o] = tf32_rna(x);
      gl[o] = tf32_rna(x - gh[o]);
    }
  CK(cudaMalloc(hi, gh.size() * 4));
  CK(cudaMalloc(lo, gl.size() * 4));
  CK(cudaMemcpy(*hi, gh.data(), gh.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(*lo, gl.data(), gl.size() * 4, cudaMemcpyHostToDevice));
  return GMMNLSE_OK;
}

static int upload_hilo(const std::vector<double>& m, int rows, int cols, int rows_pad, int cols_pad, bool f16,
                       int e, __nv_bfloat16** hi, __nv_bfloat16** lo, bool tf32 = false) {
  if (tf32) return upload_hilo_tf32(m, rows, cols, rows_pad, cols_pad, hi, lo);
  std::vector<__nv_bfloat16> gh((size_t)rows_pad * cols_pad), gl((size_t)rows_pad * cols_pad);
  for (int r = 0; r < rows_pad; ++r)
    for (int k = 0; k < cols_pad; ++k) {
      const float x = (r < rows && k < cols) ? (float)std::ldexp(m[(size_t)r * cols + k], e) : 0.f;
      const size_t o = row_grouped(r, k, cols_pad, 8);
      if (f16) {
        const __half h = __float2half_rn(x), l = __float2half_rn(x - __half2float(h));
        std::memcpy(&gh[o], &h, 2);
        std::memcpy(&gl[o], &l, 2);
      } else {
        gh[o] = __float2bfloat16_rn(x);
        gl[o] = __float2bfloat16_rn(x - __bfloat162float(gh[o]));
      }
    }
  CK(cudaMalloc(hi, gh.size() * 2));
  CK(cudaMalloc(lo, gl.size() * 2));
  CK(cudaMemcpy(*hi, gh.data(), gh.size() * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(*lo, gl.data(), gl.size() * 2, cudaMemcpyHostToDevice));
  return GMMNLSE_OK;
}

// A row-major [rows][cols] matrix transposed to [cols_pad][rows_pad] in R,
// zero padding (the G operand of the CUDA-core tiled GEMM).
template <typename R>
static int upload_transposed(const std::vector<double>& m, int rows, int cols, int rows_pad, int cols_pad,
                             void** out) {
  std::vector<R> t((size_t)cols_pad * rows_pad, (R)0);
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < cols; ++k) t[(size_t)k * rows_pad + r] = (R)m[(size_t)r * cols + k];
  CK(cudaMalloc(out, t.size() * sizeof(R)));
  CK(cudaMemcpy(*out, t.data(), t.size() * sizeof(R), cudaMemcpyHostToDevice));
  return GMMNLSE_OK;
}

// Gd: the reduced coupling matrix in the standard row order; Gdiag: the same
// rows by diagonals (for the CUDA-core tiles, N > 8).
template <typename R>
static int upload_tables(gmmnlse_ctx* c, const std::vector<double>& Gd, const std::vector<double>& Gdiag) {
  std::vector<R> Gr(Gd.size());
  for (size_t i = 0; i < Gd.size(); ++i) Gr[i] = (R)Gd[i];
  CK(cudaMalloc(&c->G, Gr.size() * sizeof(R) + 16));
  CK(cudaMemcpy(c->G, Gr.data(), Gr.size() * sizeof(R), cudaMemcpyHostToDevice));
  if (c->Pt > 0) {
    const int rc = upload_transposed<R>(Gdiag, c->P, c->KK, c->Pt, c->KKt, &c->Gt);
    if (rc) return rc;
  }
  CK(cudaMalloc(&c->H, (size_t)c->n * sizeof(cplx<R>)));
  // integrand prefactor gamma0 s(w_q), s = 1 + w_q/omega0 with self-steepening
  const int n = c->n;
  std::vector<R> fac(n);
  for (int q = 0; q < n; ++q) {
    const int sq = q < n / 2 ? q : q - n;
    const double w = 2.0 * M_PI * (double)sq / ((double)n * c->prm.dt);
    fac[q] = (R)(c->prm.self_steepening ? c->gamma0 * (1.0 + w / c->omega0) : c->gamma0);
  }
  CK(cudaMalloc(&c->fac, n * sizeof(R)));
  CK(cudaMemcpy(c->fac, fac.data(), n * sizeof(R), cudaMemcpyHostToDevice));
  return GMMNLSE_OK;
}

template <typename R>
static int compute_H(gmmnlse_ctx* c, const double* hR) {
  const int n = c->n;
  double2 *hin = nullptr, *hsp = nullptr, *scr = nullptr;
  std::vector<double2> h(n);
  for (int i = 0; i < n; ++i) h[i] = make_double2(hR ? hR[i] : 0.0, 0.0);
  CK(cudaMalloc(&hin, n * sizeof(double2)));
  CK(cudaMalloc(&hsp, n * sizeof(double2)));
  CK(cudaMalloc(&scr, n * sizeof(double2)));
  CK(cudaMemcpy(hin, h.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
  int rc = fft64(c, scr, hin, hsp, 1, -1, 1.0, 0);
  if (rc) return rc;
  if (std::is_same<R, float>::value) CK(cudaMalloc(&c->Hv, (size_t)n * sizeof(float2)));
  k_raman_H<R><<<(n + 255) / 256, 256>>>(hsp, (cplx<R>*)c->H, (float2*)c->Hv, n, c->prm.dt, c->fR);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  cudaFree(hin);
  cudaFree(hsp);
  cudaFree(scr);
  return GMMNLSE_OK;
}

// cplx: SK and SR are complex, interleaved (re, im) [N][N][N][N][2], with no
// symmetry assumed (the general coupling); else real and symmetric (Eq. 2).
static int create_ctx(const gmmnlse_params* prm, const double* beta, const double* SK, const double* SR, double fR,
                      const double* hR, bool cplx, gmmnlse_ctx** out) {
  if (!prm || !beta || !SK || !out) return GMMNLSE_E_INVALID;
  *out = nullptr;
  const int N = prm->N, n = prm->Nt;
  if (N < 1 || N > kMaxN) return GMMNLSE_E_INVALID;
  if (n < 16 || n > 16384 || (n & (n - 1))) return GMMNLSE_E_INVALID;
  if (!(prm->dt > 0) || !(prm->lambda0 > 0) || !std::isfinite(prm->n2)) return GMMNLSE_E_INVALID;
  if (!(fR >= 0.0 && fR < 1.0)) return GMMNLSE_E_INVALID;
  if (fR > 0 && !hR) return GMMNLSE_E_INVALID;
  if (prm->precision < GMMNLSE_FP64 || prm->precision > GMMNLSE_MIXED_TF32) return GMMNLSE_E_INVALID;
  if (prm->max_iter < 0 || prm->fixed_iters < 0) return GMMNLSE_E_INVALID;
  const size_t S4 = (size_t)N * N * N * N, SW = cplx ? 2 * S4 : S4;
  if (!finite_all(beta, (size_t)N * n) || !finite_all(SK, SW) || (SR && !finite_all(SR, SW)) ||
      (hR && !finite_all(hR, n)))
    return GMMNLSE_E_INVALID;
  if (cplx) {
    // the general coupling: FP64 or FP32 on the CUDA cores, up to 32 modes
    if (N > 32) return GMMNLSE_E_UNSUPPORTED;
    if (prm->precision != GMMNLSE_FP64 && prm->precision != GMMNLSE_FP32) return GMMNLSE_E_UNSUPPORTED;
  } else if (!symmetric_enough(SK, N) || (SR && !symmetric_enough(SR, N))) {
    return GMMNLSE_E_UNSUPPORTED;
  }
  const bool fp64 = prm->precision == GMMNLSE_FP64;
  int rc = set_device(prm->device);
  if (rc) return rc;
  auto gate = gm_gate_device(prm->device);

  gmmnlse_ctx* c = new (std::nothrow) gmmnlse_ctx();
  if (!c) return GMMNLSE_E_NOMEM;
  c->prm = *prm;
  c->N = N;
  c->n = n;
  c->fp64 = fp64;
  c->ept = ept_for(n, fp64);
  c->fR = fR;
  c->omega0 = 2.0 * M_PI * C_LIGHT / prm->lambda0;
  c->gamma0 = prm->n2 * c->omega0 / C_LIGHT;
  c->K = N * (N + 1) / 2;
  c->P = c->K;
  bool same = (SR == nullptr) || (SR == SK) || std::memcmp(SR, SK, SW * sizeof(double)) == 0;
  c->raman_mode = (fR == 0.0) ? 0 : (same ? 1 : 2);
  c->KK = (c->raman_mode == 2) ? 2 * c->K : c->K;
  if (cplx) {
    c->general = true;
    c->gK = N * N;
    c->KK = (c->raman_mode == 2) ? 2 * c->gK : c->gK;
    c->P = 2 * c->gK;
  }

  // pair / row enumeration (m <= n), reduced coupling matrix G [P][KK]
  std::vector<int2> pairs;
  for (int m = 0; m < N; ++m)
    for (int q = m; q < N; ++q) pairs.push_back(make_int2(m, q));
  std::vector<double> Gd((size_t)c->P * c->KK);
  auto S_at = [&](const double* S, int p, int l, int m, int q) {
    return S[(((size_t)p * N + l) * N + m) * N + q];
  };
  // general coupling: sum_mn S_plmn A_m A_n^* over the real rows U of the
  // pair products (Re A_m A_n^* for m <= n, then Im A_m A_n^* for m < n):
  //   m = n:  S_plmm |A_m|^2
  //   m < n:  (S_plmn + S_plnm) Re(A_m A_n^*) + i (S_plmn - S_plnm) Im(A_m A_n^*)
  // (A_n A_m^* is the conjugate of A_m A_n^*); the complex coefficient of
  // row k gives Gd rows 2 (p N + l) (real part of R_pl) and + 1 (imaginary)
  std::vector<int2> gpairs;
  if (cplx) {
    for (int m = 0; m < N; ++m)
      for (int q = m; q < N; ++q) gpairs.push_back(make_int2(m, q));
    for (int m = 0; m < N; ++m)
      for (int q = m + 1; q < N; ++q) gpairs.push_back(make_int2(m, q + N));
    auto Sc = [&](const double* S, int p, int l, int m, int q) {
      const size_t i = 2 * ((((size_t)p * N + l) * N + m) * N + q);
      return std::complex<double>(S[i], S[i + 1]);
    };
    auto fill = [&](const double* S, double w, int col0) {
      for (int p = 0; p < N; ++p)
        for (int l = 0; l < N; ++l) {
          const size_t r = 2 * ((size_t)p * N + l);
          for (int k = 0; k < c->gK; ++k) {
            const int m = gpairs[k].x, q = gpairs[k].y;
            std::complex<double> coef;
            if (q >= N) coef = std::complex<double>(0.0, 1.0) * (Sc(S, p, l, m, q - N) - Sc(S, p, l, q - N, m));
            else if (m == q) coef = Sc(S, p, l, m, m);
            else coef = Sc(S, p, l, m, q) + Sc(S, p, l, q, m);
            Gd[r * c->KK + col0 + k] = w * coef.real();
            Gd[(r + 1) * c->KK + col0 + k] = w * coef.imag();
          }
        }
    };
    if (c->raman_mode == 2) {
      fill(SK, 1.0 - fR, 0);
      fill(SR, fR, c->gK);
    } else {
      fill(SK, 1.0, 0);
    }
  }
  for (int r = 0; r < c->P && !cplx; ++r) {
    const int p = pairs[r].x, l = pairs[r].y;
    for (int k = 0; k < c->K; ++k) {
      const int m = pairs[k].x, q = pairs[k].y;
      if (c->raman_mode == 2) {
        Gd[(size_t)r * c->KK + k] = (1.0 - fR) * S_at(SK, p, l, m, q);
        Gd[(size_t)r * c->KK + c->K + k] = fR * S_at(SR, p, l, m, q);
      } else {
        Gd[(size_t)r * c->KK + k] = S_at(SK, p, l, m, q);
      }
    }
  }

  // length scales of the step sizes (gmmnlse_choose_step)
  c->beta0.resize(N);
  for (int p = 0; p < N; ++p) {
    c->beta0[p] = beta[(size_t)p * n];
    const size_t pp = (((size_t)p * N + p) * N + p) * N + p;
    c->s_max = std::max(c->s_max, cplx ? std::hypot(SK[2 * pp], SK[2 * pp + 1]) : SK[pp]);
  }
  // the reduced S^R [P][K] kept on the host for the gain's saturation term
  // (uploaded when gmmnlse_set_gain_saturation switches it on)
  if (!cplx) c->GR_host.resize((size_t)c->P * c->K);
  for (int r = 0; r < c->P && !cplx; ++r)
    for (int k = 0; k < c->K; ++k)
      c->GR_host[(size_t)r * c->K + k] =
          S_at(SR ? SR : SK, pairs[r].x, pairs[r].y, pairs[k].x, pairs[k].y);

  // mixed precision: the contraction runs on the tensor cores where it is a
  // dense GEMM, N >= 9 (with Nt a multiple of the 128-point tile); for N <= 8
  // the FP32 register contraction is faster than a GEMM that small and is
  // used instead
  const bool mixed = prm->precision == GMMNLSE_MIXED_BF16 || prm->precision == GMMNLSE_MIXED_FP16 ||
                     prm->precision == GMMNLSE_MIXED_TF32;
  if (mixed && N > 8) {
    if (N < TC_MIN_N || N > TC_MAX_N || n % TC_PTS != 0) {
      delete c;
      return GMMNLSE_E_UNSUPPORTED;
    }
    const int NB = tc_row_block(c->P);
    c->tc = true;
    c->f16 = prm->precision == GMMNLSE_MIXED_FP16;
    c->tf32 = prm->precision == GMMNLSE_MIXED_TF32;
    c->KKp = (c->KK + TC_KC - 1) / TC_KC * TC_KC;
    c->tc_rows = (c->P + NB - 1) / NB * NB;
    if (const char* w = getenv("GMMNLSE_TC_WAIT_MS")) {
      const double ms = atof(w);
      if (ms > 0 && ms <= 60000) c->tc_wait_ns = (unsigned long long)(ms * 1e6);
    }
    const char* stall = getenv("GMMNLSE_TC_STALL");
    c->tc_stall = stall ? std::max(0, std::min(2, atoi(stall))) : 0;
  }

  // CUDA-core tiled contraction (N > 8): G transposed, padded to whole tiles
  const int KC = TileCfg<float>::KC, TR = TileCfg<float>::TR;
  static_assert(TileCfg<float>::KC == TileCfg<double>::KC && TileCfg<float>::TR == TileCfg<double>::TR,
                "one padding for both precisions");
  if (N > 8 || c->general) {
    c->KKt = (c->KK + KC - 1) / KC * KC;
    c->Pt = (c->P + TR - 1) / TR * TR;
  }

  // low-rank coupling G = X W (N > 8 with S^R = S^K), used when the rank is
  // at most 3/4 of K; GMMNLSE_DENSE=1 keeps the dense contraction
  std::vector<double> Xd, Wd, Gt_rows, Xt_rows;
  const char* dense_env = getenv("GMMNLSE_DENSE");
  // (with 16-bit tensor-core operands the first GEMM forms U from A in the
  // kernel, which stages the A of at most U_FIT_N modes: more modes keep the
  // dense coupling)
  const bool lr_fits = !(c->tc && !c->tf32 && N > U_FIT_N);
  if (N > 8 && !c->general && c->raman_mode != 2 && lr_fits && !(dense_env && dense_env[0] == '1')) {
    // the dropped part of the coupling (columns below tol x the largest)
    // stays under the rounding of the working precision's contraction:
    // 1e-12 for FP64; 1e-9 for FP32 and the mixed precisions, whose FP32
    // products round at ~6e-8 (the 42-mode step-index coupling: rank 210
    // instead of 255 of 903)
    const double lr_tol = fp64 ? 1e-12 : 1e-9;
    const int r = lowrank(Gd, c->P, c->K, lr_tol, Xd, Wd);
    if (r > 0 && 4 * r <= 3 * c->K) {
      c->lr = true;
      c->r = r;
      double ws = 0.0;
      for (int s = 0; s < r; ++s) {
        double a = 0.0;
        for (int k = 0; k < c->K; ++k) a += std::fabs(Wd[(size_t)s * c->K + k]);
        ws = std::max(ws, a);
      }
      int e;
      std::frexp(ws, &e);  // ws < 2^e
      c->eW = e;
      c->rP1 = (r + TR - 1) / TR * TR;
      c->rK2 = (r + KC - 1) / KC * KC;
      if (c->tc) {
        const int nblk = (r + 255) / 256;
        c->NB1 = ((r + nblk - 1) / nblk + 15) / 16 * 16;
        c->r_rows = c->NB1 * nblk;
        c->rKKp = (r + TC_KC - 1) / TC_KC * TC_KC;
      }
    }
  }

  // device copies: twiddles exp(-2 pi i m / n) followed by the pass tables
  // of the transform length (fft_block reads them at tw + n; layout as
  // fft_pass_table_len)
  auto pass_tables = [](int len, std::vector<double2>& out) {
    int logn = 0;
    while ((1 << logn) < len) ++logn;
    for (int Ns = 1 << (logn & 3); Ns < len; Ns <<= 4) {
      if (Ns == 1) continue;
      for (int r = 1; r < 16; ++r)
        for (int k = 0; k < Ns; ++k) {
          const double a = 2.0 * M_PI * (double)k * r / (16.0 * Ns);
          out.push_back(make_double2(std::cos(a), -std::sin(a)));
        }
    }
    if (logn == 14)  // the radix-32 pass with Ns = 32 of the 32 x 32 x 16 schedule
      for (int r = 1; r < 32; ++r)
        for (int k = 0; k < 32; ++k) {
          const double a = 2.0 * M_PI * (double)k * r / (32.0 * 32.0);
          out.push_back(make_double2(std::cos(a), -std::sin(a)));
        }
  };
  std::vector<double2> tw(n), twh(n / 2);
  for (int m = 0; m < n; ++m) {
    const double a = 2.0 * M_PI * (double)m / (double)n;
    tw[m] = make_double2(std::cos(a), -std::sin(a));
  }
  for (int m = 0; m < n / 2; ++m) twh[m] = tw[2 * m];
  pass_tables(n, tw);
  pass_tables(n / 2, twh);
  std::vector<float2> tw32(tw.size());
  for (size_t m = 0; m < tw.size(); ++m) tw32[m] = make_float2((float)tw[m].x, (float)tw[m].y);
#define CKC(call)                     \
  do {                                \
    cudaError_t e_ = (call);          \
    if (e_ != cudaSuccess) {          \
      gm_set_last_cuda_error(e_, #call, __FILE__, __LINE__); \
      free_ctx(c);                    \
      return GMMNLSE_E_CUDA;          \
    }                                 \
  } while (0)
  CKC(cudaMalloc(&c->beta, (size_t)N * n * sizeof(double)));
  CKC(cudaMemcpy(c->beta, beta, (size_t)N * n * sizeof(double), cudaMemcpyHostToDevice));
  CKC(cudaMalloc(&c->tw64, tw.size() * sizeof(double2)));
  CKC(cudaMemcpy(c->tw64, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice));
  CKC(cudaMalloc(&c->tw64h, twh.size() * sizeof(double2)));
  CKC(cudaMemcpy(c->tw64h, twh.data(), twh.size() * sizeof(double2), cudaMemcpyHostToDevice));
  CKC(cudaMalloc(&c->tw32, tw32.size() * sizeof(float2)));
  CKC(cudaMemcpy(c->tw32, tw32.data(), tw32.size() * sizeof(float2), cudaMemcpyHostToDevice));
  if (!c->general) {
    CKC(cudaMalloc(&c->rows, c->P * sizeof(int2)));
    CKC(cudaMemcpy(c->rows, pairs.data(), c->P * sizeof(int2), cudaMemcpyHostToDevice));
  } else {
    CKC(cudaMalloc(&c->gpairs, c->gK * sizeof(int2)));
    CKC(cudaMemcpy(c->gpairs, gpairs.data(), c->gK * sizeof(int2), cudaMemcpyHostToDevice));
    Gt_rows = Gd;  // rows in their own order (the complex l-sum needs no diagonal order)
  }
  CKC(cudaMalloc(&c->pairs, c->K * sizeof(int2)));
  CKC(cudaMemcpy(c->pairs, pairs.data(), c->K * sizeof(int2), cudaMemcpyHostToDevice));
  // CUDA-core tiles take their rows by diagonals (p, p + d): G and X rows
  // permuted to that order, with the (p, l) table to match
  if (N > 8 && !c->general) {
    std::vector<int2> diag;
    for (int d = 0; d < N; ++d)
      for (int p = 0; p + d < N; ++p) diag.push_back(make_int2(p, p + d));
    auto std_row = [&](int2 pl) { return pl.x * N - pl.x * (pl.x - 1) / 2 + (pl.y - pl.x); };
    auto permute = [&](const std::vector<double>& m, int cols) {
      std::vector<double> out(m.size());
      for (int i = 0; i < c->P; ++i)
        std::memcpy(&out[(size_t)i * cols], &m[(size_t)std_row(diag[i]) * cols], cols * sizeof(double));
      return out;
    };
    Gt_rows = permute(Gd, c->KK);
    if (c->lr) Xt_rows = permute(Xd, c->r);
    CKC(cudaMalloc(&c->rows_t, c->P * sizeof(int2)));
    CKC(cudaMemcpy(c->rows_t, diag.data(), c->P * sizeof(int2), cudaMemcpyHostToDevice));
  }
  rc = fp64 ? upload_tables<double>(c, Gd, Gt_rows) : upload_tables<float>(c, Gd, Gt_rows);
  if (!rc) rc = gm_nz_build(c, Gd);
  if (!rc && c->lr) {
    rc = fp64 ? upload_transposed<double>(Wd, c->r, c->K, c->rP1, c->KKt, &c->Wt)
              : upload_transposed<float>(Wd, c->r, c->K, c->rP1, c->KKt, &c->Wt);
    if (!rc)
      rc = fp64 ? upload_transposed<double>(Xt_rows, c->P, c->r, c->Pt, c->rK2, &c->Xt)
                : upload_transposed<float>(Xt_rows, c->P, c->r, c->Pt, c->rK2, &c->Xt);
    if (!rc && c->tc) {
      // 16-bit operands: GEMM 1 forms U in the kernel in 4 x 4 blocks of
      // (m, n) (each block from four A_m and four A_n); W's columns are
      // reordered to match, with the weights (1 on the diagonal, 2 off it)
      // and zeros for the block entries that are not pairs m <= n < N
      std::vector<double> Wu;
      int KU = c->K;
      if (!c->tf32) {
        const int nmb = (N + 3) / 4;
        std::vector<int2> blk;
        for (int bm = 0; bm < nmb; ++bm)
          for (int bn = bm; bn < nmb; ++bn) blk.push_back(make_int2(4 * bm, 4 * bn));
        c->nublk = (int)blk.size();
        KU = 16 * c->nublk;
        c->KKpU = (KU + TC_KC - 1) / TC_KC * TC_KC;
        Wu.assign((size_t)c->r * KU, 0.0);
        for (int b = 0; b < c->nublk; ++b)
          for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) {
              const int m = blk[b].x + i, nn = blk[b].y + j, k = 16 * b + 4 * i + j;
              if (m > nn || nn >= N) continue;
              const int ks = m * N - m * (m - 1) / 2 + (nn - m);  // (m, nn) in the order of `pairs`
              const double w = m == nn ? 1.0 : 2.0;
              for (int s = 0; s < c->r; ++s) Wu[(size_t)s * KU + k] = w * Wd[(size_t)s * c->K + ks];
            }
        if (cudaMalloc(&c->ublk, blk.size() * sizeof(int2)) != cudaSuccess ||
            cudaMemcpy(c->ublk, blk.data(), blk.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
          rc = GMMNLSE_E_NOMEM;
      }
      const std::vector<double>& Wup = c->tf32 ? Wd : Wu;
      c->eW16 = c->f16 ? f16_exp(Wup) : 0;
      c->eX16 = c->f16 ? f16_exp(Xd) : 0;
      if (!rc)
        rc = upload_hilo(Wup, c->r, KU, c->r_rows, c->tf32 ? c->KKp : c->KKpU, c->f16, c->eW16, &c->Whi, &c->Wlo,
                         c->tf32);
      if (!rc)
        rc = upload_hilo(Xd, c->P, c->r, c->tc_rows, c->rKKp, c->f16, c->eX16, &c->Xhi, &c->Xlo, c->tf32);
    }
  }
  if (!rc && c->tc) {
    // G split into hi + lo in the blocked operand layout; FP16 scaled by 2^eG
    // so that its largest entry is below 2^14
    if (c->f16) c->eG = f16_exp(Gd);
    rc = upload_hilo(Gd, c->P, c->KK, c->tc_rows, c->KKp, c->f16, c->eG, &c->Ghi, &c->Glo, c->tf32);
    if (!rc) rc = gm_make_g_maps(c);
  }
  if (!rc) rc = set_smem_attrs(c);
  if (!rc) rc = fp64 ? compute_H<double>(c, hR) : compute_H<float>(c, hR);
  if (rc) {
    free_ctx(c);
    return rc;
  }
  if (prm->stream) {
    c->stream = (cudaStream_t)prm->stream;
  } else {
    CKC(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = true;
  }
#undef CKC
  *out = c;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_create(const gmmnlse_params* prm, const double* beta, const double* SK,
                              const double* SR, double fR, const double* hR, gmmnlse_ctx** out) {
  return create_ctx(prm, beta, SK, SR, fR, hR, false, out);
}

extern "C" int gmmnlse_create_general(const gmmnlse_params* prm, const double* beta, const double* SK,
                                      const double* SR, double fR, const double* hR, gmmnlse_ctx** out) {
  return create_ctx(prm, beta, SK, SR, fR, hR, true, out);
}

extern "C" int gmmnlse_destroy(gmmnlse_ctx* c) {
  if (!c) return GMMNLSE_OK;
  cudaSetDevice(c->prm.device);
  auto gate = gm_gate_device(c->prm.device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_ctx(c);
  return GMMNLSE_OK;
}

// ---------------------------------------------------------------------------
// Workspaces
// ---------------------------------------------------------------------------
static size_t job_bytes(const gmmnlse_ctx* c, int M) {
  const size_t rs = c->fp64 ? 8 : 4, cs = 2 * rs;
  const size_t Nn = (size_t)c->N * c->n;
  size_t b = 0;
  b += Nn * 16;                                  // psi0
  if (!c->fp64) b += Nn * cs;                    // psiR
  b += (size_t)M * Nn * cs;                      // dpsi
  b += 4 * (size_t)(M + 1) * Nn * cs;            // A, NL, I, E
  const size_t vrows = c->general ? c->gK : c->K;
  if (c->raman_mode) b += (size_t)(M + 1) * vrows * c->n * rs;  // Y = h_R * U
  if (c->lr) b += (size_t)(M + 1) * c->r * c->n * rs;          // Z = W U
  if (c->general) b += (size_t)(M + 1) * c->gK * c->n * rs;    // the pair-product rows U
  b += 2 * Nn * 16 * 2;                          // EM64, io
  b += sizeof(LoopState) + 64 + sizeof(double2) * TRAPZ_MAX_BLOCKS;
  b += (size_t)(M + 1) * (c->K + c->P) * sizeof(double);  // saturation: Ubar, Rs
  if (c->tc) b += (size_t)2 * c->KKp * (M + 1) * c->n * (c->tf32 ? 4 : 2);  // hi/lo operand
  return b;
}

extern "C" size_t gmmnlse_request_bytes(const gmmnlse_ctx* c, int M) { return c ? job_bytes(c, M) : 0; }

static void free_job(gm_job* jb) {
  if (!jb) return;
  for (auto& g : jb->graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  for (auto& g : jb->pack_graphs) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  if (jb->psiR != (void*)jb->psi0) cudaFree(jb->psiR);
  cudaFree(jb->psi0);
  cudaFree(jb->dpsi);
  cudaFree(jb->A);
  cudaFree(jb->V);
  cudaFree(jb->Z);
  cudaFree(jb->NL);
  cudaFree(jb->I);
  cudaFree(jb->E);
  cudaFree(jb->EM64);
  cudaFree(jb->io);
  cudaFree(jb->flag);
  cudaFree(jb->Vhi);
  cudaFree(jb->Vlo);
  cudaFree(jb->ls);
  cudaFree(jb->part);
  cudaFree(jb->bar);
  cudaFree(jb->Ubar);
  cudaFree(jb->Rs);
  cudaFreeHost(jb->h_ls);
  cudaFreeHost(jb->h_io);
  if (jb->cap) cudaStreamDestroy(jb->cap);
  delete jb;
}

// TMA maps of the blocked hi/lo operands (V: [K/EPC][points][EPC], see
// tc_map; coupling: row-grouped, see tc_map_rows), one K chunk per box; the
// encode function comes from the CUDA driver at run time (no link dependency
// on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int tc_encoder(EncodeTiledFn* out) {
  static EncodeTiledFn enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess) {
      gm_set_last_error_text("cuTensorMapEncodeTiled is not available from the driver");
      return GMMNLSE_E_CUDA;
    }
    enc = (EncodeTiledFn)fn;
  }
  *out = enc;
  return GMMNLSE_OK;
}

// Map of a blocked [KKp/EPC][rows][EPC] operand (16-byte core-matrix rows:
// EPC 8 for BF16 / FP16, 4 for TF32 words); box = one K chunk of box_rows
// rows.
static int tc_map(CUtensorMap* map, void* base, cuuint64_t rows, int KKp, int box_rows, bool f16,
                  bool tf32 = false) {
  EncodeTiledFn enc;
  const int rc = tc_encoder(&enc);
  if (rc) return rc;
  // A K plane [rows][epc] is contiguous: it is described as rows of 256
  // elements (32 points of 8 BF16/FP16 values, or 64 points of 4 TF32 ones),
  // so that each row of the box is one 512- or 1024-byte transfer instead of
  // a 16-byte one; the box lands in shared memory in the same [kq][point][epc]
  // order.  rows is a multiple of 128.
  const int epc = tf32 ? 4 : 8, esz = tf32 ? 4 : 2;
  const cuuint64_t dims[3] = {256, rows * epc / 256, (cuuint64_t)(KKp / epc)};
  const cuuint64_t strides[2] = {(cuuint64_t)(256 * esz), rows * 16};
  const cuuint32_t box[3] = {256, (cuuint32_t)(box_rows * epc / 256), (cuuint32_t)(TC_KC / epc)};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                      : (f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  const CUresult r = enc(map, dt, 3, base, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    gm_set_last_error_text("cuTensorMapEncodeTiled rejected the operand layout");
    return GMMNLSE_E_CUDA;
  }
  return GMMNLSE_OK;
}

// Map of a row-grouped [rows/8][KKp/EPC][8][EPC] coupling operand; box = one
// K chunk of NB / cl rows (one CTA's share of a row block of NB rows when
// cl = 2 CTAs share each MMA).
static int tc_map_rows(CUtensorMap* map, void* base, cuuint64_t rows, int KKp, int NB, bool f16, bool tf32, int cl) {
  EncodeTiledFn enc;
  const int rc = tc_encoder(&enc);
  if (rc) return rc;
  // The K chunk of an 8-row group ([TC_KC/epc][8][epc], 512 bytes for 16-bit
  // operands, 1024 for TF32) is contiguous: the map's rows are those chunks
  // (256 elements), so each 8-row group of the box is one transfer; the box
  // lands in shared memory as [group][kq][8][epc] as before.
  const int epc = tf32 ? 4 : 8, esz = tf32 ? 4 : 2;
  const cuuint64_t kq = (cuuint64_t)(KKp / epc);
  const cuuint64_t dims[3] = {256, (cuuint64_t)(KKp / TC_KC), rows / 8};
  const cuuint64_t strides[2] = {(cuuint64_t)(256 * esz), kq * 128};
  const cuuint32_t box[3] = {256, 1, (cuuint32_t)(NB / 8 / cl)};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                      : (f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
  const CUresult r = enc(map, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    gm_set_last_error_text("cuTensorMapEncodeTiled rejected the coupling operand layout");
    return GMMNLSE_E_CUDA;
  }
  return GMMNLSE_OK;
}

int gm_make_g_maps(gmmnlse_ctx* c) {
  const int NB = tc_row_block(c->P);
  // CTAs that share each MMA: as TcShape<..>::CL (the first low-rank GEMM
  // with 16-bit operands forms U in the kernel and runs on single CTAs)
  const int cl = tc_cluster(NB), cl1 = c->tf32 ? tc_cluster(c->NB1) : 1;
  int rc = tc_map_rows(&c->mapGhi, c->Ghi, (cuuint64_t)c->tc_rows, c->KKp, NB, c->f16, c->tf32, cl);
  if (!rc) rc = tc_map_rows(&c->mapGlo, c->Glo, (cuuint64_t)c->tc_rows, c->KKp, NB, c->f16, c->tf32, cl);
  if (!rc && c->lr) {
    const int kw = c->tf32 ? c->KKp : c->KKpU;  // K of GEMM 1 (16-bit: the blocked U columns)
    rc = tc_map_rows(&c->mapWhi, c->Whi, (cuuint64_t)c->r_rows, kw, c->NB1, c->f16, c->tf32, cl1);
    if (!rc) rc = tc_map_rows(&c->mapWlo, c->Wlo, (cuuint64_t)c->r_rows, kw, c->NB1, c->f16, c->tf32, cl1);
    if (!rc) rc = tc_map_rows(&c->mapXhi, c->Xhi, (cuuint64_t)c->tc_rows, c->rKKp, NB, c->f16, c->tf32, cl);
    if (!rc) rc = tc_map_rows(&c->mapXlo, c->Xlo, (cuuint64_t)c->tc_rows, c->rKKp, NB, c->f16, c->tf32, cl);
  }
  return rc;
}

int gm_make_tc_maps(gmmnlse_ctx* c, gm_job* jb, int M) {
  const cuuint64_t npts = (cuuint64_t)(M + 1) * c->n * jb->slots;
  int rc = tc_map(&jb->mapHi, jb->Vhi, npts, c->KKp, TC_PTS, c->f16, c->tf32);
  if (!rc) rc = tc_map(&jb->mapLo, jb->Vlo, npts, c->KKp, TC_PTS, c->f16, c->tf32);
  if (!rc && c->lr) {
    rc = tc_map(&jb->mapHi2, jb->Vhi, npts, c->rKKp, TC_PTS, c->f16, c->tf32);
    if (!rc) rc = tc_map(&jb->mapLo2, jb->Vlo, npts, c->rKKp, TC_PTS, c->f16, c->tf32);
  }
  return rc;
}

int gm_job_create(gmmnlse_ctx* c, int M, gm_job** out) { return gm_job_create_slots(c, M, 1, out); }

// A workspace of `slots` propagations with M substeps per long step: every
// array once per slot (the per-slice arrays by slice = slot (M + 1) + j).
int gm_job_create_slots(gmmnlse_ctx* c, int M, int slots, gm_job** out) {
  *out = nullptr;
  if (slots < 1 || slots > 64) return GMMNLSE_E_INVALID;
  auto gate = gm_gate_device(c->prm.device);
  gm_job* jb = new (std::nothrow) gm_job();
  if (!jb) return GMMNLSE_E_NOMEM;
  jb->ctx = c;
  jb->Mcap = M;
  jb->slots = slots;
  const size_t rs = c->fp64 ? 8 : 4, cs = 2 * rs;
  const size_t Nn = (size_t)c->N * c->n, B = (size_t)slots;
  const size_t S1 = (size_t)(M + 1) * B;  // slices
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b ? b : 16);
  };
  al((void**)&jb->psi0, B * Nn * 16);
  if (c->fp64) jb->psiR = jb->psi0;
  else al(&jb->psiR, B * Nn * cs);
  al(&jb->dpsi, B * (size_t)M * Nn * cs);
  al(&jb->A, S1 * Nn * cs);
  al(&jb->NL, S1 * Nn * cs);
  al(&jb->I, S1 * Nn * cs);
  al(&jb->E, S1 * Nn * cs);
  if (c->raman_mode) al(&jb->V, S1 * (c->general ? c->gK : c->K) * c->n * rs);
  if (c->lr) al(&jb->Z, S1 * c->r * c->n * rs);
  if (c->general) al(&jb->Z, S1 * c->gK * c->n * rs);
  al((void**)&jb->EM64, B * 2 * Nn * 16);
  al((void**)&jb->io, 2 * Nn * 16);
  al((void**)&jb->flag, sizeof(int));
  al((void**)&jb->ls, B * sizeof(LoopState));
  al((void**)&jb->part, B * sizeof(double2) * TRAPZ_MAX_BLOCKS);
  al((void**)&jb->bar, 64);
  al((void**)&jb->Ubar, S1 * c->K * sizeof(double));
  al((void**)&jb->Rs, S1 * c->P * sizeof(double));
  const size_t vb = (size_t)c->KKp * S1 * c->n * (c->tf32 ? 4 : 2);
  if (c->tc) {
    al((void**)&jb->Vhi, vb);
    al((void**)&jb->Vlo, vb);
  }
  // the hi/lo operand starts at zero: with the low-rank coupling its padding
  // columns from 8 ceil(r/8) on are never written again (k_raman_vpack
  // writes whole 8-column groups, the columns from r as zeros)
  if (c->tc && e == cudaSuccess) e = cudaMemset(jb->Vhi, 0, vb);
  if (c->tc && e == cudaSuccess) e = cudaMemset(jb->Vlo, 0, vb);
  // every slot starts empty (a packed launch skips it)
  if (e == cudaSuccess) e = cudaMemset(jb->ls, 0, B * sizeof(LoopState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&jb->h_ls, B * sizeof(LoopState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&jb->h_io, Nn * 16);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&jb->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess && slots > 1) {
    for (int k = 0; k < slots; ++k) {
      std::memset(&jb->h_ls[k], 0, sizeof(LoopState));
      jb->h_ls[k].idle = 1;
    }
    e = cudaMemcpy(jb->ls, jb->h_ls, B * sizeof(LoopState), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    gm_set_last_cuda_error(e, "workspace allocation", __FILE__, __LINE__);
    cudaGetLastError();
    free_job(jb);
    return e == cudaErrorMemoryAllocation ? GMMNLSE_E_NOMEM : GMMNLSE_E_CUDA;
  }
  if (c->tc) {
    const int rc = gm_make_tc_maps(c, jb, M);
    if (rc) {
      free_job(jb);
      return rc;
    }
  }
  jb->bytes = job_bytes(c, M) * B;
  *out = jb;
  return GMMNLSE_OK;
}

void gm_job_destroy(gm_job* jb) {
  if (!jb) return;
  auto gate = gm_gate_device(jb->ctx->prm.device);
  free_job(jb);
}

// ---------------------------------------------------------------------------
// Kernel chain of one iteration and the long-step driver
// ---------------------------------------------------------------------------
// Substep schedule: round(L/dz) substeps of dz, long steps of M, remainder last.
int gm_schedule(double L, double dz, int M, long* nfull, int* Mrem) {
  if (!(L > 0) || !(dz > 0) || M < 1 || M > kMaxM || !std::isfinite(L) || !std::isfinite(dz))
    return GMMNLSE_E_INVALID;
  const double r = L / dz;
  if (r > 1e12) return GMMNLSE_E_INVALID;
  const long total = (long)std::llround(r);
  if (total < 1 || std::fabs((double)total * dz - L) > 1e-9 * std::max(L, dz)) return GMMNLSE_E_INVALID;
  *nfull = total / M;
  *Mrem = (int)(total % M);
  return GMMNLSE_OK;
}

// The device work gate.  Tensor-core propagations running at the same time
// as other propagations on other streams of one device were seen to stall
// for good: a CTA of a pair waiting in its TMEM allocation while its peer
// waited at the cluster barrier, although no other kernel held TMEM on that
// SM (the same kernels on one stream never stalled).  The gate keeps the
// tensor-core work of this library alone on its device.
namespace {
struct DeviceGate {
  std::mutex m;
  std::condition_variable cv;
  int readers = 0, writers_waiting = 0;
  bool writer = false;
};
DeviceGate g_gate[64];
}  // namespace

GmGateHold::GmGateHold(int d, bool e) : dev(d), excl(e) {
  if (dev < 0 || dev >= 64) {
    dev = -1;
    return;
  }
  DeviceGate& g = g_gate[dev];
  std::unique_lock<std::mutex> lk(g.m);
  if (excl) {
    ++g.writers_waiting;
    g.cv.wait(lk, [&] { return !g.writer && g.readers == 0; });
    --g.writers_waiting;
    g.writer = true;
  } else {
    g.cv.wait(lk, [&] { return !g.writer && g.writers_waiting == 0; });
    ++g.readers;
  }
}

GmGateHold::~GmGateHold() {
  if (dev < 0) return;
  DeviceGate& g = g_gate[dev];
  std::lock_guard<std::mutex> lk(g.m);
  if (excl) g.writer = false;
  else g.readers -= 1;
  g.cv.notify_all();
}

GmGateHold gm_gate(const gmmnlse_ctx* c) { return GmGateHold(c->prm.device, c->tc); }
GmGateHold gm_gate_device(int device) { return GmGateHold(device, false); }

int gm_job_propagate(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                     double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  gmmnlse_ctx* c = jb->ctx;
  if (M > jb->Mcap) return GMMNLSE_E_INVALID;
  auto gate = gm_gate(c);
  return c->fp64 ? gm_propagate_f64(jb, A0, dev_io, L, dz, M, tol, Aout, st, s)
                 : gm_propagate_f32(jb, A0, dev_io, L, dz, M, tol, Aout, st, s);
}

size_t gm_job_bytes(const gm_job* jb) { return jb->bytes; }

bool gm_packable(const gmmnlse_ctx* c, double L, double dz, int M) {
  long nfull = 0;
  int Mrem = 0;
  if (gm_schedule(L, dz, M, &nfull, &Mrem) != GMMNLSE_OK || Mrem != 0 || nfull < 1) return false;
  // the Sec. IV terms, the opt-in cooperative long step and FP64 at 2^14
  // (cluster transforms) run unpacked
  const char* persist = getenv("GMMNLSE_PERSIST");
  if (persist && persist[0] == '1') return false;
  if (c->fp64 && c->n > 8192) return false;
  const char* cl = getenv("GMMNLSE_CLUSTER_FFT");
  if (cl && cl[0] == '1') return false;
  return !(c->Q || c->gain || c->sat != 0.0);
}

int gm_pack_admit(gm_job* jb, int slot, const double* A0, double L, double dz, double tol, cudaStream_t s) {
  if (cudaSetDevice(jb->ctx->prm.device) != cudaSuccess) return GMMNLSE_E_CUDA;
  auto gate = gm_gate_device(jb->ctx->prm.device);
  return jb->ctx->fp64 ? gm_pack_admit_f64(jb, slot, A0, L, dz, tol, s) : gm_pack_admit_f32(jb, slot, A0, L, dz, tol, s);
}

int gm_pack_step(gm_job* jb, cudaStream_t s, int* finished) {
  if (cudaSetDevice(jb->ctx->prm.device) != cudaSuccess) return GMMNLSE_E_CUDA;
  auto gate = gm_gate(jb->ctx);
  return jb->ctx->fp64 ? gm_pack_step_f64(jb, s, finished) : gm_pack_step_f32(jb, s, finished);
}

int gm_pack_retire(gm_job* jb, int slot, double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  if (cudaSetDevice(jb->ctx->prm.device) != cudaSuccess) return GMMNLSE_E_CUDA;
  auto gate = gm_gate_device(jb->ctx->prm.device);
  return jb->ctx->fp64 ? gm_pack_retire_f64(jb, slot, Aout, st, s) : gm_pack_retire_f32(jb, slot, Aout, st, s);
}

extern "C" int gmmnlse_profile(gmmnlse_ctx* c, int M, int reps, double* ms, double* bytes) {
  if (!c || !ms || !bytes || reps < 1 || M < 1 || M > kMaxM) return GMMNLSE_E_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  if (!c->job || c->job->Mcap < M || c->job->tab_M < M) return GMMNLSE_E_INVALID;
  auto gate = gm_gate(c);
  return c->fp64 ? gm_profile_f64(c, c->job, M, reps, ms, bytes) : gm_profile_f32(c, c->job, M, reps, ms, bytes);
}

int gm_ctx_device(const gmmnlse_ctx* c) { return c->prm.device; }
int gm_ctx_modes(const gmmnlse_ctx* c) { return c->N; }
int gm_ctx_samples(const gmmnlse_ctx* c) { return c->n; }

extern "C" int gmmnlse_propagate(gmmnlse_ctx* c, const double* A0, double L, double dz, int M, double tol,
                                 double* Aout, gmmnlse_stats* st) {
  if (!c || !A0 || !Aout) return GMMNLSE_E_INVALID;
  long nf;
  int mr;
  int rc = gm_schedule(L, dz, M, &nf, &mr);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  rc = set_device(c->prm.device);
  if (rc) return rc;
  if (c->job && c->job->Mcap < M) {
    cudaStreamSynchronize(c->stream);
    gm_job_destroy(c->job);
    c->job = nullptr;
  }
  if (!c->job) {
    rc = gm_job_create(c, M, &c->job);
    if (rc) return rc;
  }
  return gm_job_propagate(c->job, A0, c->prm.io_device != 0, L, dz, M, tol, Aout, st, c->stream);
}

extern "C" int gmmnlse_propagate_rk4ip(gmmnlse_ctx* c, const double* A0, double L, double h, double* Aout,
                                       gmmnlse_stats* st) {
  if (!c || !A0 || !Aout) return GMMNLSE_E_INVALID;
  long nf;
  int mr;
  int rc = gm_schedule(L, h, 1, &nf, &mr);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(c->mu);
  rc = set_device(c->prm.device);
  if (rc) return rc;
  if (!c->job) {
    rc = gm_job_create(c, 1, &c->job);
    if (rc) return rc;
  }
  auto gate = gm_gate(c);
  return c->fp64 ? gm_rk4ip_f64(c->job, A0, c->prm.io_device != 0, L, h, Aout, st, c->stream)
                 : gm_rk4ip_f32(c->job, A0, c->prm.io_device != 0, L, h, Aout, st, c->stream);
}

extern "C" int gmmnlse_set_linear_coupling(gmmnlse_ctx* c, const double* Q) {
  if (!c) return GMMNLSE_E_INVALID;
  const size_t NN = (size_t)c->N * c->N;
  if (Q)
    for (size_t i = 0; i < NN; ++i)
      if (!std::isfinite(Q[i])) return GMMNLSE_E_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto gate = gm_gate_device(c->prm.device);
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->qv += 1;  // graphs built before this call no longer apply
  if (!Q) {
    cudaFree(c->Q);
    c->Q = nullptr;
    return GMMNLSE_OK;
  }
  if (!c->Q && cudaMalloc(&c->Q, NN * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->Q = nullptr;
    return GMMNLSE_E_NOMEM;
  }
  if (cudaMemcpy(c->Q, Q, NN * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return GMMNLSE_E_CUDA;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_set_gain(gmmnlse_ctx* c, const double* g) {
  if (!c) return GMMNLSE_E_INVALID;
  const size_t N = (size_t)c->N;
  if (g)
    for (size_t i = 0; i < N; ++i)
      if (!std::isfinite(g[i])) return GMMNLSE_E_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  auto gate = gm_gate_device(c->prm.device);
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->qv += 1;  // graphs built before this call no longer apply
  if (!g) {
    cudaFree(c->gain);
    c->gain = nullptr;
    return GMMNLSE_OK;
  }
  if (!c->gain && cudaMalloc(&c->gain, N * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->gain = nullptr;
    return GMMNLSE_E_NOMEM;
  }
  if (cudaMemcpy(c->gain, g, N * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) return GMMNLSE_E_CUDA;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_set_gain_saturation(gmmnlse_ctx* c, double sat) {
  if (!c || !std::isfinite(sat) || sat < 0.0) return GMMNLSE_E_INVALID;
  if (c->general && sat != 0.0) return GMMNLSE_E_UNSUPPORTED;  // its rows use the real reduced S^R
  std::lock_guard<std::mutex> lk(c->mu);
  auto gate = gm_gate_device(c->prm.device);
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->qv += 1;  // graphs built before this call no longer apply
  if (sat == 0.0) {
    c->sat = 0.0;
    return GMMNLSE_OK;
  }
  if (!c->GRt) {
    std::vector<double> t((size_t)c->K * c->P);
    for (int r = 0; r < c->P; ++r)
      for (int k = 0; k < c->K; ++k) t[(size_t)k * c->P + r] = c->GR_host[(size_t)r * c->K + k];
    if (cudaMalloc(&c->GRt, t.size() * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      c->GRt = nullptr;
      return GMMNLSE_E_NOMEM;
    }
    if (cudaMemcpy(c->GRt, t.data(), t.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
      return GMMNLSE_E_CUDA;
  }
  c->sat = sat;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_set_coupling_profile(gmmnlse_ctx* c, const double* f, int count, double fdz) {
  if (!c) return GMMNLSE_E_INVALID;
  if (f) {
    if (count < 1 || !(fdz > 0.0) || !std::isfinite(fdz)) return GMMNLSE_E_INVALID;
    for (int i = 0; i < count; ++i)
      if (!std::isfinite(f[i])) return GMMNLSE_E_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  auto gate = gm_gate_device(c->prm.device);
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  if (c->stream) cudaStreamSynchronize(c->stream);
  c->qv += 1;  // graphs built before this call no longer apply
  cudaFree(c->fprof);
  c->fprof = nullptr;
  c->fcount = 0;
  if (!f) return GMMNLSE_OK;
  if (cudaMalloc(&c->fprof, (size_t)count * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    c->fprof = nullptr;
    return GMMNLSE_E_NOMEM;
  }
  if (cudaMemcpy(c->fprof, f, (size_t)count * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return GMMNLSE_E_CUDA;
  c->fcount = count;
  c->fdz = fdz;
  return GMMNLSE_OK;
}

extern "C" int gmmnlse_choose_m(gmmnlse_ctx* c, const double* A0, double dz, double tol,
                                const int* candidates, int count, int trial_substeps, double* scratch,
                                double* sec_per_substep, int* M_best) {
  if (!c || !A0 || !candidates || count < 1 || count > kMaxM || trial_substeps < 1 || !scratch || scratch == A0 ||
      !M_best || !(dz > 0) || !std::isfinite(dz) || !(tol > 0))
    return GMMNLSE_E_INVALID;
  int order[kMaxM];
  for (int i = 0; i < count; ++i) {
    if (candidates[i] < 1 || candidates[i] > kMaxM) return GMMNLSE_E_INVALID;
    order[i] = i;
  }
  // Largest M first: the first trial sizes the workspace for all the others.
  std::sort(order, order + count, [&](int a, int b) { return candidates[a] > candidates[b]; });
  const double L = trial_substeps * dz;
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return GMMNLSE_E_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return GMMNLSE_E_CUDA;
  }
  int best = -1, last = GMMNLSE_OK;
  double best_t = 0;
  for (int k = 0; k < count; ++k) {
    const int i = order[k], M = candidates[i];
    double t = std::numeric_limits<double>::infinity();
    rc = gmmnlse_propagate(c, A0, L, dz, M, tol, scratch, nullptr);  // untimed: tables and graph for M
    if (rc == GMMNLSE_OK) {
      cudaEventRecord(e0, c->stream);
      rc = gmmnlse_propagate(c, A0, L, dz, M, tol, scratch, nullptr);
      cudaEventRecord(e1, c->stream);
      float ms = 0;
      if (rc == GMMNLSE_OK && cudaEventSynchronize(e1) == cudaSuccess &&
          cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        t = 1e-3 * ms / trial_substeps;
      else if (rc == GMMNLSE_OK)
        rc = GMMNLSE_E_CUDA;
    }
    if (rc == GMMNLSE_E_INVALID || rc == GMMNLSE_E_CUDA || rc == GMMNLSE_E_NOMEM) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return rc;  // the field or the device, not the candidate, is at fault
    }
    last = rc;
    if (sec_per_substep) sec_per_substep[i] = t;
    if (rc == GMMNLSE_OK && (best < 0 || t < best_t)) {
      best = i;
      best_t = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return last;
  *M_best = candidates[best];
  return GMMNLSE_OK;
}

// ---------------------------------------------------------------------------
// Step sizes from the length scales and a step-doubling error estimate
// ---------------------------------------------------------------------------
extern "C" int gmmnlse_choose_step(gmmnlse_ctx* c, const double* A0, double L, double rtol, double tol,
                                   double* scratch, gmmnlse_step* out) {
  if (!c || !A0 || !scratch || !out || scratch == A0 || !(L > 0) || !std::isfinite(L) || !(tol > 0) ||
      !(rtol >= 0) || !std::isfinite(rtol))
    return GMMNLSE_E_INVALID;
  int rc = set_device(c->prm.device);
  if (rc) return rc;
  const size_t Nn = (size_t)c->N * c->n;
  const bool dev = c->prm.io_device != 0;
  // the field on the host (its peak power; the trial results are compared there)
  std::vector<double> a0(2 * Nn), a1(2 * Nn), a2(2 * Nn);
  auto fetch = [&](const double* src, std::vector<double>& dst) -> int {
    if (dev) {
      if (cudaMemcpy(dst.data(), src, Nn * 16, cudaMemcpyDeviceToHost) != cudaSuccess) {
        gm_set_last_cuda_error(cudaGetLastError(), "cudaMemcpy", __FILE__, __LINE__);
        return GMMNLSE_E_CUDA;
      }
    } else {
      std::memcpy(dst.data(), src, Nn * 16);
    }
    return GMMNLSE_OK;
  };
  rc = fetch(A0, a0);
  if (rc) return rc;
  double P0 = 0.0;
  for (int k = 0; k < c->n; ++k) {
    double pk = 0.0;
    for (int p = 0; p < c->N; ++p) {
      const double* z = &a0[2 * ((size_t)p * c->n + k)];
      pk += z[0] * z[0] + z[1] * z[1];
    }
    if (!std::isfinite(pk)) return GMMNLSE_E_INVALID;
    P0 = std::max(P0, pk);
  }
  if (!(P0 > 0.0) || !(c->gamma0 > 0.0) || !(c->s_max > 0.0)) return GMMNLSE_E_INVALID;
  // Sec. III.D: L_long = M dz << z_NL (about z_NL / 10) and dz << z_IM; the
  // paper's usual z_NL / dz is about 200
  const double z_nl = 1.0 / (c->gamma0 * c->s_max * P0);
  double db = 0.0;
  for (int p = 0; p < c->N; ++p) db = std::max(db, std::fabs(c->beta0[p] - c->beta0[0]));
  const double z_im = db > 0.0 ? 1.0 / db : std::numeric_limits<double>::infinity();
  double dz = std::min(z_nl / 200.0, z_im / 10.0);
  const double dz_cap = dz;
  auto pick_M = [&](double d, long nsub) {
    long m = (long)std::floor(z_nl / (10.0 * d));
    return (int)std::max(1L, std::min({m, (long)kMaxM, nsub}));
  };
  double err = 0.0;
  int trials = 0;
  if (rtol > 0.0) {
    // step doubling on a trial piece of one nonlinear length (or the whole
    // fiber if shorter): the trapezoid is second order, so A(dz) - A_exact
    // ~ (4/3) (A(dz) - A(dz/2)); the error grows about linearly along z
    const double ell = std::min(L, z_nl);
    for (int it = 0; it < 4; ++it) {
      long ns = std::max(2L, 2 * (long)std::ceil(ell / (2.0 * dz)));
      const double d = ell / (double)ns;
      const int M = pick_M(d, ns);
      double* s1 = scratch;
      double* s2 = scratch + 2 * Nn;
      rc = gmmnlse_propagate(c, A0, ell, d, M, tol, s1, nullptr);
      if (!rc) rc = gmmnlse_propagate(c, A0, ell, 0.5 * d, M, tol, s2, nullptr);
      trials += 2;
      if (rc) return rc;
      rc = fetch(s1, a1);
      if (!rc) rc = fetch(s2, a2);
      if (rc) return rc;
      double dd = 0.0, nn = 0.0;
      for (size_t i = 0; i < 2 * Nn; ++i) {
        dd += (a1[i] - a2[i]) * (a1[i] - a2[i]);
        nn += a2[i] * a2[i];
      }
      err = (4.0 / 3.0) * std::sqrt(dd / nn) * (L / ell);
      dz = d;
      if (err <= rtol) break;
      dz = d * std::sqrt(rtol / err) * 0.9;  // second order: err ~ dz^2
      err = err * (dz / d) * (dz / d);        // (the estimate at the new dz)
    }
  }
  dz = std::min(dz, dz_cap);
  const long nsub = std::max(1L, (long)std::ceil(L / dz - 1e-9));
  out->dz = L / (double)nsub;
  out->M = pick_M(out->dz, nsub);
  out->z_nl = z_nl;
  out->z_im = z_im;
  out->err_est = err;
  out->trials = trials;
  return GMMNLSE_OK;
}

extern "C" const char* gmmnlse_strerror(int s) {
  switch (s) {
    case GMMNLSE_OK: return "ok";
    case GMMNLSE_PENDING: return "pending";
    case GMMNLSE_E_INVALID: return "invalid argument";
    case GMMNLSE_E_NOMEM: return "out of device memory or over the memory budget";
    case GMMNLSE_E_UNSUPPORTED: return "unsupported configuration";
    case GMMNLSE_E_NOT_CONVERGED: return "MPA iteration did not converge within max_iter";
    case GMMNLSE_E_NONFINITE: return "non-finite value in the field";
    case GMMNLSE_E_CUDA: return "CUDA error";
    case GMMNLSE_E_BUSY: return "server queue full";
    case GMMNLSE_E_CANCELLED: return "request cancelled";
    default: return "unknown status";
  }
}
