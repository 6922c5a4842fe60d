// FP64 instantiation of the solver (all three models).
#include "sgn_solver.cuh"

namespace sgn {
SolverBase* make_solver_f64(int model) {
  switch (model) {
    case 0: return new Solver<0, double>();
    case 1: return new Solver<1, double>();
    case 2: return new Solver<2, double>();
  }
  return nullptr;
}
}  // namespace sgn
