// float64 instantiation of the solvers.
#include "spfc_solver2d.cuh"

namespace spfc {
SolverBase* make_solver_f64(const Params& P, cudaStream_t st, int* status, std::string* err) {
  if (P.d == 2) return make_solver_2d<double>(P, st, status, err);
  *status = 1;
  *err = "3D is not available in this build";
  return nullptr;
}
}  // namespace spfc
