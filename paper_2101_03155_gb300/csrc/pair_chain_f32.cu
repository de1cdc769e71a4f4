// FP32 instantiation of the pair-potential chain (mixed form).
#include "pair_chain.cuh"

namespace ace {
template <>
cudaError_t launch_pair_pass<float>(int mode, const PairPassArgs<float> &a, int npacks, cudaStream_t st) {
  return launch_pair_pass_impl<float>(mode, a, npacks, st);
}
template <>
cudaError_t launch_conv_pass<float>(const PairPassArgs<float> &a, int npacks, cudaStream_t st) {
  return launch_conv_impl<float>(a, npacks, st);
}

bool axis_factors(int L, int *r1, int *r2) {
  switch (L) {
#define ACE_CASE(L_)        \
  case L_:                  \
    *r1 = Factor<L_>::R1;   \
    *r2 = Factor<L_>::R2;   \
    return true;
    ACE_PASS_LENGTHS(ACE_CASE)
#undef ACE_CASE
    default:
      return false;
  }
}

bool pass_length_supported(int L) {
  switch (L) {
#define ACE_CASE(L_) case L_:
    ACE_PASS_LENGTHS(ACE_CASE)
#undef ACE_CASE
    return true;
    default:
      return false;
  }
}
}  // namespace ace
