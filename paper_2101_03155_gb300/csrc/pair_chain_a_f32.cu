// Pencil-pass and axis-1 kernels (float) for the axis lengths of group A (pair_chain.cuh).
#include "pair_chain.cuh"

namespace ace {
ACE_DEFINE_GROUP(a_f32, float, ACE_LENGTHS_A, ACE_LENGTHS_A)
}  // namespace ace
