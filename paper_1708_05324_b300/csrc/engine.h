// Internal interface between the solver engine and the request server.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/gmmnlse.h"

struct gm_job;

// Device work gate.  Every library call that puts work on a device holds its
// gate until that work has finished (each such call synchronizes before it
// returns): calls that launch the tensor-core contraction hold it alone,
// every other call shares it.  So tensor-core work never runs beside other
// work of this library on the device, as on a single stream; the rest
// overlaps freely.  Writers (tensor-core calls) waiting keep new readers
// out.  Not re-entrant: a call holding it runs no other gated call.
struct GmGateHold {
  int dev = -1;
  bool excl = false;
  GmGateHold() = default;
  GmGateHold(int d, bool e);
  GmGateHold(GmGateHold&& o) noexcept : dev(o.dev), excl(o.excl) { o.dev = -1; }
  GmGateHold(const GmGateHold&) = delete;
  GmGateHold& operator=(const GmGateHold&) = delete;
  GmGateHold& operator=(GmGateHold&&) = delete;
  ~GmGateHold();
};
// The hold a call on context c takes (exclusive when c's contraction runs on
// the tensor cores).
GmGateHold gm_gate(const gmmnlse_ctx* c);
GmGateHold gm_gate_device(int device);  // shared

void gm_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void gm_set_last_error_text(const char* msg);
int gm_job_create(gmmnlse_ctx* c, int M, gm_job** out);
int gm_job_create_slots(gmmnlse_ctx* c, int M, int slots, gm_job** out);
size_t gm_job_bytes(const gm_job* jb);
// Packed propagations (serving): slots of one workspace that share the
// context and M, each with its own field, dz and tolerance.
bool gm_packable(const gmmnlse_ctx* c, double L, double dz, int M);
int gm_pack_admit(gm_job* jb, int slot, const double* A0_host, double L, double dz, double tol, cudaStream_t s);
int gm_pack_step(gm_job* jb, cudaStream_t s, int* finished);  // finished[slot]: 1 when that slot has ended
int gm_pack_retire(gm_job* jb, int slot, double* Aout_host, gmmnlse_stats* st, cudaStream_t s);
int gm_make_tc_maps(gmmnlse_ctx* c, gm_job* jb, int M);
int gm_make_g_maps(gmmnlse_ctx* c);
// N <= 8 on the CUDA cores: build (at context creation) and free the
// contraction kernel compiled for the context's nonzero coupling entries
// (nzlist.cu); Gd is the reduced coupling [P][KK] in the standard row order
int gm_nz_build(gmmnlse_ctx* c, const std::vector<double>& Gd);
void gm_nz_free(gmmnlse_ctx* c);
void gm_job_destroy(gm_job* jb);
int gm_job_propagate(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                     double* Aout, gmmnlse_stats* st, cudaStream_t s);
int gm_schedule(double L, double dz, int M, long* nfull, int* Mrem);
int gm_propagate_f32(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                     double* Aout, gmmnlse_stats* st, cudaStream_t s);
int gm_propagate_f64(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                     double* Aout, gmmnlse_stats* st, cudaStream_t s);
int gm_rk4ip_f32(gm_job* jb, const double* A0, bool dev_io, double L, double h, double* Aout, gmmnlse_stats* st,
                 cudaStream_t s);
int gm_rk4ip_f64(gm_job* jb, const double* A0, bool dev_io, double L, double h, double* Aout, gmmnlse_stats* st,
                 cudaStream_t s);
int gm_profile_f32(gmmnlse_ctx* c, gm_job* jb, int M, int reps, double* ms, double* bytes);
int gm_profile_f64(gmmnlse_ctx* c, gm_job* jb, int M, int reps, double* ms, double* bytes);
int gm_pack_admit_f32(gm_job* jb, int slot, const double* A0, double L, double dz, double tol, cudaStream_t s);
int gm_pack_admit_f64(gm_job* jb, int slot, const double* A0, double L, double dz, double tol, cudaStream_t s);
int gm_pack_step_f32(gm_job* jb, cudaStream_t s, int* finished);
int gm_pack_step_f64(gm_job* jb, cudaStream_t s, int* finished);
int gm_pack_retire_f32(gm_job* jb, int slot, double* Aout, gmmnlse_stats* st, cudaStream_t s);
int gm_pack_retire_f64(gm_job* jb, int slot, double* Aout, gmmnlse_stats* st, cudaStream_t s);
int gm_prop_setup_f32(int device);
int gm_prop_setup_f64(int device);
int gm_ctx_device(const gmmnlse_ctx* c);
int gm_ctx_modes(const gmmnlse_ctx* c);
int gm_ctx_samples(const gmmnlse_ctx* c);
