// MPA long-step driver instantiated for float iterates.
#include "prop_impl.cuh"

int gm_propagate_f32(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                     double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  return gm_prop::propagate_impl<float>(jb, A0, dev_io, L, dz, M, tol, Aout, st, s);
}

int gm_profile_f32(gmmnlse_ctx* c, gm_job* jb, int M, int reps, double* ms, double* bytes) {
  return gm_prop::profile_impl<float>(c, jb, M, reps, ms, bytes);
}

int gm_prop_setup_f32(int device) { return gm_prop::setup_device<float>(device); }

int gm_rk4ip_f32(gm_job* jb, const double* A0, bool dev_io, double L, double h, double* Aout, gmmnlse_stats* st,
                 cudaStream_t s) {
  return gm_prop::rk4ip_impl<float>(jb, A0, dev_io, L, h, Aout, st, s);
}

int gm_pack_admit_f32(gm_job* jb, int slot, const double* A0, double L, double dz, double tol, cudaStream_t s) {
  return gm_prop::pack_admit<float>(jb, slot, A0, L, dz, tol, s);
}

int gm_pack_step_f32(gm_job* jb, cudaStream_t s, int* finished) { return gm_prop::pack_step<float>(jb, s, finished); }

int gm_pack_retire_f32(gm_job* jb, int slot, double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  return gm_prop::pack_retire<float>(jb, slot, Aout, st, s);
}
