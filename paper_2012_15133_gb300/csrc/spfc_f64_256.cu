// float64 solvers for 256 x 256 grids (all launch schedules).
#include "spfc_solver2d.cuh"

namespace spfc {
SolverBase* make_solver_2d_f64_256(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err) {
  return make_solver_2d_n<double, 256>(P, st, schedule, status, err);
}
}  // namespace spfc
