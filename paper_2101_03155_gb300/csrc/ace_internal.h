// ace_internal.h -- declarations shared by the translation units of the library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ace {

template <typename T>
struct alignas(2 * sizeof(T)) cpx;

// Passes of the pair-potential chain (Eq. e:vij by FFT, accumulated as in Eq. vx).
enum PassMode : int {
  PASS_FWD3_PAIR = 0,  // axis 3 forward; prologue forms z = phi_a phi_b + i phi_c phi_d
  PASS_FWD2 = 1,       // axis 2 forward
  PASS_CONV1 = 2,      // axis 1 forward, multiply by 4 pi/(N |G|^2), axis 1 inverse
  PASS_INV2 = 3,       // axis 2 inverse
  PASS_INV3_ACC = 4    // axis 3 inverse; epilogue W_a += v_ab phi_b, W_b += v_ab phi_a, ...
};

// A pack holds two pairs (a,b) and (c,d) transformed together as z = rho_ab + i rho_cd; the
// Coulomb kernel is real and even, so the inverse transform returns v_ab + i v_cd.
// c = d = -1 marks an empty second slot.
template <typename T>
struct PairPassArgs {
  const T *phi;             // [norb][N]
  T *W;                     // [norb][N]
  cpx<T> *scratch;          // [batch][N] complex workspace
  const int4 *packs;        // [npacks]
  int pack0;                // first pack of this launch
  const T *kernel;          // [N] 4 pi / (N |G_m|^2), natural order, 0 at G = 0
  const cpx<T> *tw;         // [L] e^{-2 pi i e / L} for the axis of this pass
  long long N;              // N1 N2 N3
  int n1, n2, n3;
};

// Launch one pass over `npacks` packs (grid.y); returns cudaErrorInvalidValue if the axis
// length has no compiled plan.
template <typename T>
cudaError_t launch_pair_pass(int mode, const PairPassArgs<T> &a, int npacks, cudaStream_t st);

bool pass_length_supported(int L);

// Dense steps.
template <typename T>
cudaError_t launch_gram(const T *X, int nx, const T *Y, int ny, long long K, double scale, bool abs_values,
                        bool upper_only, double *G, cudaStream_t st);
template <typename T>
cudaError_t launch_left_mul(const T *A, int m, int n, const T *Y, long long K, T *Z, cudaStream_t st);

cudaError_t launch_cholesky(const double *M_raw, int n, double spin_factor, double *M, double *L, double *Linv,
                            double *energy, int *status, cudaStream_t st);
cudaError_t launch_screen_compact(const double *O, int n, double rho_cut, int2 *pairs, int4 *packs,
                                  int *count, double *O_sym, cudaStream_t st);

template <typename T>
cudaError_t launch_transpose_scale(const double *C, int n, int m, double scale, T *A, cudaStream_t st);

// Sets the message returned by ace_last_error() on this thread.
void set_last_error(const char *msg);

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *in, Tout *out, long long count, double scale, cudaStream_t st);

}  // namespace ace
