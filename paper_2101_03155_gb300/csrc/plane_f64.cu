// Instantiations of the plane passes (double) for the plane shapes listed below.
#include "plane_chain.cuh"

namespace ace {
bool plane_ops_f64(int n2, int n3, PlaneOps<double> *out) {
#define X(A, B)                                                   \
  if (n2 == A && n3 == B && PlaneLaunch<double, A, B>::fits(false)) { \
    out->fwd = &PlaneLaunch<double, A, B>::fwd;                       \
    out->inv = &PlaneLaunch<double, A, B>::inv;                       \
    out->acc_fits = PlaneLaunch<double, A, B>::fits(true);            \
    return true;                                                  \
  }
  X(12,24) X(16,16) X(32,32) X(48,48) X(64,64) X(72,72) X(96,96) X(108,108)
#undef X
  return false;
}
}  // namespace ace
