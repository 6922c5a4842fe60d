// Mixed-precision instantiation (FP32 bulk, FP64 depth / hydrostatic term /
// positivity / mass update) of the solver, all three models.
#include "sgn_solver.cuh"

namespace sgn {
SolverBase* make_solver_mixed(int model) {
  switch (model) {
    case 0: return new Solver<0, float>();
    case 1: return new Solver<1, float>();
    case 2: return new Solver<2, float>();
  }
  return nullptr;
}
}  // namespace sgn
