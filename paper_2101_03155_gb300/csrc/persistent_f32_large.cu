// Instantiations of the persistent pair chain (float) for the grids listed below.
#include "persistent_chain.cuh"

namespace ace {
bool persist_ops_f32_large(int n1, int n2, int n3, PersistOps<float> *out) {
#define X(A, B, C)                                                     \
  if (n1 == A && n2 == B && n3 == C) {                                \
    using Ln = PersistLaunch<float, A, B, C>;                          \
    out->blocks_per_sm = &Ln::blocks_per_sm;                           \
    out->launch = &Ln::launch;                                         \
    out->tasks_per_pack = 2 * A + Ln::NC;                              \
    return true;                                                       \
  }
  X(96, 96, 96) X(108, 108, 108) X(128, 128, 128) X(144, 144, 144) X(160, 144, 128)
#undef X
  return false;
}
}  // namespace ace
