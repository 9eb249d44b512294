// Host-side interface between the C ABI and the templated solvers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "spfc_state.h"

namespace spfc {

struct KernelTimes {
  std::vector<std::string> names;
  std::vector<int64_t> launches;
  std::vector<double> ms;
};

class SolverBase {
 public:
  virtual ~SolverBase() {}
  virtual int init(const double* phi0, bool on_device, int mode) = 0;
  virtual int set_state(const double* phi, const double* phi_prev, double r, double r_prev, bool on_device) = 0;
  virtual int step(long long n) = 0;
  virtual int energy(double* E_orig, double* E_mod, double* E_breve) = 0;
  virtual int mass(double* mass, double* mean) = 0;
  virtual int scalars(SavScal* out) = 0;
  virtual int get_field(double* out, bool on_device, int which) = 0;
  virtual int dt_change(double dt) = 0;
  virtual int set_stab(double A) = 0;  // stabiliser of Sec. 5.2 for the following steps
  // optional phi^4 term (gamma3 >= 0) for the following steps; a solver
  // without such kernels accepts gamma3 = 0 only
  virtual int set_gamma3(double g3) {
    if (g3 == 0.0) return 0;
    err = "this solver has no kernels for the phi^4 term";
    return 1;
  }
  // the PFC model of Sec. 1 (phi^4 coefficient g3 > 0) or the SPFC model (0);
  // a solver without its kernels accepts 0 only
  virtual int set_pfc(double g3) {
    if (g3 == 0.0) return 0;
    err = "this solver has no kernels for the PFC model (2D single runs only)";
    return 1;
  }
  virtual int sync() = 0;
  virtual int set_timing(bool on) = 0;
  virtual int kernel_times(KernelTimes* kt) = 0;
  virtual int64_t device_bytes() const = 0;
  // raw state (scalar record + both spectral levels, newest first) for exact checkpoints
  virtual int dump(std::string* blob) = 0;
  virtual int restore(const std::string& blob) = 0;

  // per-step record ring (device-visible pointer into pinned host memory)
  virtual int set_ring(double* dev, long long cap) = 0;
  void apply_ring(SavScal* h) const {
    h->ring = ring_dev;
    h->ring_cap = ring_cap;
  }
  double* ring_dev = nullptr;
  long long ring_cap = 0;

  Params P{};
  int precision = 0;
  int schedule = 0;
  bool inited = false;
  std::string err;
};

// Fill the float32 copies of the per-run constants (call after any change).
inline void fill_float_params(Params* P) {
  P->invP = 1.0 / P->P;
  for (int i = 0; i < 3; ++i) P->kf_f[i] = (float)P->kf[i];
  P->dt_f = (float)P->dt;
  P->a_f = (float)P->a;
  P->beta_f = (float)P->beta;
  P->invP_f = (float)P->invP;
  P->sdt = P->stab * P->dt;
  P->sdt_f = (float)P->sdt;
  P->g3b = (P->beta > 0.0) ? P->g3 / P->beta : 0.0;
  P->g3_f = (float)P->g3;
  P->g3b_f = (float)P->g3b;
  P->e1c4 = P->pfc ? 0.25 * P->g3 : 0.25 * P->beta;
  P->e1c2 = P->pfc ? -0.5 : -1.0;
}

// Factories (one translation unit per precision); return nullptr and set err on failure.
SolverBase* make_solver_f64(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err);
SolverBase* make_solver_f32(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err);
int num_schedules(int d, int N);
SolverBase* make_solver_3d_f64(const Params& P, cudaStream_t st, int* status, std::string* err);
SolverBase* make_solver_3d_f32(const Params& P, cudaStream_t st, int* status, std::string* err);

}  // namespace spfc

// The single-run handle behind spfc_t.
struct spfc_s {
  spfc::SolverBase* s = nullptr;
  std::string err;
};

// Internal view of a network handle (spfc_fno_t) for the surrogate loop:
// its grid size, largest batch and stream.
struct spfc_fno_s;
namespace spfc {
void fno_shape(const spfc_fno_s* f, int* n, int* max_batch, cudaStream_t* st);
}  // namespace spfc
