// float64 instantiation of the solvers.
#include "spfc_solver2d.cuh"

namespace spfc {
SolverBase* make_solver_f64(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err) {
  if (P.d == 2) return make_solver_2d<double>(P, st, schedule, status, err);
  if (schedule != 0) {
    *status = 1;
    *err = "3D grids have one schedule";
    return nullptr;
  }
  return make_solver_3d_f64(P, st, status, err);
}
int num_schedules(int d, int N) { return d == 2 ? num_schedules_2d(N) : 1; }
}  // namespace spfc
