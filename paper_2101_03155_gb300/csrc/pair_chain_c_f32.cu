// Pencil-pass and axis-1 kernels (float) for the axis lengths of group C (pair_chain.cuh).
#include "pair_chain.cuh"

namespace ace {
ACE_DEFINE_GROUP(c_f32, float, ACE_LENGTHS_C, ACE_CONV_LENGTHS_C)
}  // namespace ace
