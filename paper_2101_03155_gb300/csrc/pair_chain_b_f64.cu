// Pencil-pass and axis-1 kernels (double) for the axis lengths of group B (pair_chain.cuh).
#include "pair_chain.cuh"

namespace ace {
ACE_DEFINE_GROUP(b_f64, double, ACE_LENGTHS_B, ACE_LENGTHS_B)
}  // namespace ace
