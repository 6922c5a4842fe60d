// Mixed-precision instantiation of the refined hierarchy (all three models).
#include "sgn_amr.cuh"

namespace sgn {
AmrBase* make_amr_mixed(int model) {
  switch (model) {
    case 0: return new Amr<0, float>();
    case 1: return new Amr<1, float>();
    case 2: return new Amr<2, float>();
  }
  return nullptr;
}
}  // namespace sgn
