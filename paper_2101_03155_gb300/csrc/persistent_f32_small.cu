// Instantiations of the persistent pair chain (float) for the grids listed below.
#include "persistent_chain.cuh"

namespace ace {
bool persist_ops_f32_small(int n1, int n2, int n3, PersistOps<float> *out) {
#define X(A, B, C)                                                     \
  if (n1 == A && n2 == B && n3 == C) {                                \
    using Ln = PersistLaunch<float, A, B, C>;                          \
    out->blocks_per_sm = &Ln::blocks_per_sm;                           \
    out->launch = &Ln::launch;                                         \
    out->tasks_per_pack = 2 * A + Ln::NC;                              \
    return true;                                                       \
  }
  X(32, 32, 32) X(48, 48, 48) X(64, 64, 64) X(72, 72, 72)
#undef X
  return false;
}
}  // namespace ace
