// Pencil-pass and axis-1 kernels (double) for the axis lengths of group A (pair_chain.cuh).
#include "pair_chain.cuh"

namespace ace {
ACE_DEFINE_GROUP(a_f64, double, ACE_LENGTHS_A, ACE_LENGTHS_A)
}  // namespace ace
