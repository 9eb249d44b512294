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
  virtual int sync() = 0;
  virtual int set_timing(bool on) = 0;
  virtual int kernel_times(KernelTimes* kt) = 0;
  virtual int64_t device_bytes() const = 0;
  // raw state (scalar record + both spectral levels, newest first) for exact checkpoints
  virtual int dump(std::string* blob) = 0;
  virtual int restore(const std::string& blob) = 0;

  Params P{};
  int precision = 0;
  bool inited = false;
  std::string err;
};

// Factories (one translation unit per precision); return nullptr and set err on failure.
SolverBase* make_solver_f64(const Params& P, cudaStream_t st, int* status, std::string* err);
SolverBase* make_solver_f32(const Params& P, cudaStream_t st, int* status, std::string* err);

}  // namespace spfc
