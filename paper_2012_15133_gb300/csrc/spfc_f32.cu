// float32-bulk instantiation of the solvers (FP64 reductions and scalars).
#include "spfc_solver2d.cuh"

namespace spfc {
SolverBase* make_solver_f32(const Params& P, cudaStream_t st, int schedule, int* status, std::string* err) {
  if (P.d == 2) return make_solver_2d<float>(P, st, schedule, status, err);
  if (schedule != 0) {
    *status = 1;
    *err = "3D grids have one schedule";
    return nullptr;
  }
  return make_solver_3d_f32(P, st, status, err);
}
}  // namespace spfc
