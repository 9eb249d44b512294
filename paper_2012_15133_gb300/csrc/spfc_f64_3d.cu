// float64 3D solvers (N = 16, 32, 64, 128).
#include "spfc_solver3d.cuh"

namespace spfc {
SolverBase* make_solver_3d_f64(const Params& P, cudaStream_t st, int* status, std::string* err) {
  switch (P.N) {
    case 16: return new_solver_3d<double, 16>(P, st, status, err);
    case 32: return new_solver_3d<double, 32>(P, st, status, err);
    case 64: return new_solver_3d<double, 64>(P, st, status, err);
    case 128: return new_solver_3d<double, 128>(P, st, status, err);
    default:
      *status = 1;
      *err = "3D grid size must be one of 16, 32, 64, 128";
      return nullptr;
  }
}
}  // namespace spfc
