// FP64 instantiation of the pair-potential chain (plain form).
#include "pair_chain.cuh"

namespace ace {
template <>
cudaError_t launch_pair_pass<double>(int mode, const PairPassArgs<double> &a, int npacks, cudaStream_t st) {
  return launch_pair_pass_impl<double>(mode, a, npacks, st);
}
template <>
cudaError_t launch_conv_pass<double>(const PairPassArgs<double> &a, int npacks, cudaStream_t st) {
  return launch_conv_impl<double>(a, npacks, st);
}
}  // namespace ace
