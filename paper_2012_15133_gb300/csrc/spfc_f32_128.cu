// float32-bulk solvers for 128 x 128 grids (all launch schedules).
#include "spfc_solver2d.cuh"

namespace spfc {
SolverBase* make_solver_2d_f32_128(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err) {
  return make_solver_2d_n<float, 128>(P, st, schedule, status, err);
}
}  // namespace spfc
