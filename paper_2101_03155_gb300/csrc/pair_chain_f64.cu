// Dispatch of the pair-potential chain's pencil kernels (double, plain form) over the length groups.
#include "pair_chain.cuh"

namespace ace {
#define ACE_DECLARE_GROUP(G)                                                                             \
  bool pass_##G##_f64(int L, int mode, const PairPassArgs<double> &a, int npacks, cudaStream_t st, cudaError_t *e); \
  bool conv_##G##_f64(int L, const PairPassArgs<double> &a, int npacks, cudaStream_t st, cudaError_t *e);
ACE_DECLARE_GROUP(a)
ACE_DECLARE_GROUP(b)
ACE_DECLARE_GROUP(c)
ACE_DECLARE_GROUP(d)
#undef ACE_DECLARE_GROUP

template <>
cudaError_t launch_pair_pass<double>(int mode, const PairPassArgs<double> &a, int npacks, cudaStream_t st) {
  const int L = (mode == PASS_FWD3_PAIR || mode == PASS_INV3_ACC) ? a.n3 : (mode == PASS_CONV1 ? a.n1 : a.n2);
  cudaError_t e = cudaErrorInvalidValue;
  if (pass_a_f64(L, mode, a, npacks, st, &e) || pass_b_f64(L, mode, a, npacks, st, &e) ||
      pass_c_f64(L, mode, a, npacks, st, &e) || pass_d_f64(L, mode, a, npacks, st, &e))
    return e;
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_conv_pass<double>(const PairPassArgs<double> &a, int npacks, cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
  if (conv_a_f64(a.n1, a, npacks, st, &e) || conv_b_f64(a.n1, a, npacks, st, &e) ||
      conv_c_f64(a.n1, a, npacks, st, &e) || conv_d_f64(a.n1, a, npacks, st, &e))
    return e;
  return cudaErrorInvalidValue;
}
}  // namespace ace
