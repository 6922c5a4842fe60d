// FP64 instantiation of the refined hierarchy (all three models).
#include "sgn_amr.cuh"

namespace sgn {
AmrBase* make_amr_f64(int model) {
  switch (model) {
    case 0: return new Amr<0, double>();
    case 1: return new Amr<1, double>();
    case 2: return new Amr<2, double>();
  }
  return nullptr;
}
}  // namespace sgn
