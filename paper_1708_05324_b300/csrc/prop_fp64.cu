// MPA long-step driver instantiated for double iterates.
#include "prop_impl.cuh"

int gm_propagate_f64(gm_job* jb, const double* A0, bool dev_io, double L, double dz, int M, double tol,
                     double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  return gm_prop::propagate_impl<double>(jb, A0, dev_io, L, dz, M, tol, Aout, st, s);
}

int gm_profile_f64(gmmnlse_ctx* c, gm_job* jb, int M, int reps, double* ms, double* bytes) {
  return gm_prop::profile_impl<double>(c, jb, M, reps, ms, bytes);
}

int gm_prop_setup_f64(int device) { return gm_prop::setup_device<double>(device); }

int gm_rk4ip_f64(gm_job* jb, const double* A0, bool dev_io, double L, double h, double* Aout, gmmnlse_stats* st,
                 cudaStream_t s) {
  return gm_prop::rk4ip_impl<double>(jb, A0, dev_io, L, h, Aout, st, s);
}

int gm_pack_admit_f64(gm_job* jb, int slot, const double* A0, double L, double dz, double tol, cudaStream_t s) {
  return gm_prop::pack_admit<double>(jb, slot, A0, L, dz, tol, s);
}

int gm_pack_step_f64(gm_job* jb, cudaStream_t s, int* finished) { return gm_prop::pack_step<double>(jb, s, finished); }

int gm_pack_retire_f64(gm_job* jb, int slot, double* Aout, gmmnlse_stats* st, cudaStream_t s) {
  return gm_prop::pack_retire<double>(jb, slot, Aout, st, s);
}
