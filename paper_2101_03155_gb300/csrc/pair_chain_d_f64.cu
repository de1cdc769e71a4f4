// Pencil-pass and axis-1 kernels (double) for the axis lengths of group D (pair_chain.cuh).
#include "pair_chain.cuh"

namespace ace {
ACE_DEFINE_GROUP(d_f64, double, ACE_LENGTHS_D, ACE_NO_LENGTHS)
}  // namespace ace
