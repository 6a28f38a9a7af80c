// Compiled 3D kernel families: (p, q1) = (1,2), (2,4), (3,6), (4,6), (4,8).
#include "lh_ops.cuh"

namespace lh {
const Ops *find_ops_3d(int p, int q1) {
  if (p == 1 && q1 == 2) return OpsBuilder<3, 1, 2>::get();
  if (p == 2 && q1 == 4) return OpsBuilder<3, 2, 4>::get();
  if (p == 3 && q1 == 6) return OpsBuilder<3, 3, 6>::get();
  if (p == 4 && q1 == 6) return OpsBuilder<3, 4, 6>::get();
  if (p == 4 && q1 == 8) return OpsBuilder<3, 4, 8>::get();
  return nullptr;
}
}  // namespace lh
