// Internal interface between the solver engine and the request server.
#pragma once

#include <cuda_runtime.h>

#include "../../include/gmmnlse.h"

struct gm_job;

void gm_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void gm_set_last_error_text(const char* msg);
int gm_job_create(gmmnlse_ctx* c, int M, gm_job** out);
int gm_make_tc_maps(gmmnlse_ctx* c, gm_job* jb, int M);
int gm_make_g_maps(gmmnlse_ctx* c);
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
int gm_prop_setup_f32(int device);
int gm_prop_setup_f64(int device);
int gm_ctx_device(const gmmnlse_ctx* c);
int gm_ctx_modes(const gmmnlse_ctx* c);
int gm_ctx_samples(const gmmnlse_ctx* c);
