// Instantiations of the plane passes (float) for the plane shapes listed below.
#include "plane_chain.cuh"

namespace ace {
bool plane_ops_f32_small(int n2, int n3, PlaneOps<float> *out) {
#define X(A, B)                                                   \
  if (n2 == A && n3 == B && PlaneLaunch<float, A, B>::fits(false)) { \
    out->fwd = &PlaneLaunch<float, A, B>::fwd;                       \
    out->inv = &PlaneLaunch<float, A, B>::inv;                       \
    out->acc_fits = PlaneLaunch<float, A, B>::fits(true);            \
    return true;                                                  \
  }
  X(12,24) X(16,16) X(32,32) X(48,48) X(64,64) X(72,72)
#undef X
  return false;
}
}  // namespace ace
