// Dispatch of the pair-potential chain's pencil kernels (float, mixed form) over the length groups.
#include "pair_chain.cuh"

namespace ace {
#define ACE_DECLARE_GROUP(G)                                                                             \
  bool pass_##G##_f32(int L, int mode, const PairPassArgs<float> &a, int npacks, cudaStream_t st, cudaError_t *e); \
  bool conv_##G##_f32(int L, const PairPassArgs<float> &a, int npacks, cudaStream_t st, cudaError_t *e);
ACE_DECLARE_GROUP(a)
ACE_DECLARE_GROUP(b)
ACE_DECLARE_GROUP(c)
ACE_DECLARE_GROUP(d)
#undef ACE_DECLARE_GROUP

template <>
cudaError_t launch_pair_pass<float>(int mode, const PairPassArgs<float> &a, int npacks, cudaStream_t st) {
  const int L = (mode == PASS_FWD3_PAIR || mode == PASS_INV3_ACC) ? a.n3 : (mode == PASS_CONV1 ? a.n1 : a.n2);
  cudaError_t e = cudaErrorInvalidValue;
  if (pass_a_f32(L, mode, a, npacks, st, &e) || pass_b_f32(L, mode, a, npacks, st, &e) ||
      pass_c_f32(L, mode, a, npacks, st, &e) || pass_d_f32(L, mode, a, npacks, st, &e))
    return e;
  return cudaErrorInvalidValue;
}

template <>
cudaError_t launch_conv_pass<float>(const PairPassArgs<float> &a, int npacks, cudaStream_t st) {
  cudaError_t e = cudaErrorInvalidValue;
  if (conv_a_f32(a.n1, a, npacks, st, &e) || conv_b_f32(a.n1, a, npacks, st, &e) ||
      conv_c_f32(a.n1, a, npacks, st, &e) || conv_d_f32(a.n1, a, npacks, st, &e))
    return e;
  return cudaErrorInvalidValue;
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

bool conv_length_supported(int L) {
  switch (L) {
#define ACE_CASE(L_) case L_:
    ACE_LENGTHS_A(ACE_CASE) ACE_LENGTHS_B(ACE_CASE) ACE_CONV_LENGTHS_C(ACE_CASE)
#undef ACE_CASE
    return true;
    default:
      return false;
  }
}
}  // namespace ace
