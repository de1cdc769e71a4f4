// Pencil-pass and axis-1 kernels (double) for the axis lengths of group C (pair_chain.cuh).
#include "pair_chain.cuh"

namespace ace {
ACE_DEFINE_GROUP(c_f64, double, ACE_LENGTHS_C, ACE_CONV_LENGTHS_C)
}  // namespace ace
