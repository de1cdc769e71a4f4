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
  int conv_tile;            // axis-1 pencil pass of the plane chain, FP32: 0 (32 columns, default
                            // threads), 1 (32 columns, the other thread count), 2 (16 columns, 128)
};

// Arguments of the three-pass (plane, pencil, plane) chain.
template <typename T>
struct PlaneArgs {
  const T *phi;        // [norb][N]
  T *W;                // [norb][N]
  cpx<T> *scratch;     // [batch][N], pack p of the launch at p - batch0
  const int4 *packs;   // all packs of the build
  const int4 *groups;  // (first pack, pack count, shared first orbital or -1, 0)
  int pack0;           // forward pass: first pack of this launch
  int group0;          // inverse pass: first group of this launch
  int batch0;          // first pack of the batch held in the scratch
  const cpx<T> *tw2;   // [N2] e^{-2 pi i e / N2}
  const cpx<T> *tw3;   // [N3] e^{-2 pi i e / N3}
  long long N;
  int n1;
  int hints;           // bit 0: drop each consumed scratch plane from L2 without writing it back
  const float *pmax;   // plane maxima [norb][n1] and orbital maxima [norb] for the plane skip
  const float *gmax;
  float skip_rel;      // > 0: planes below this fraction of the orbitals' maxima are skipped
};

// Plane passes for one (N2, N3) plane shape; absent shapes fall back to the five pencil passes.
template <typename T>
struct PlaneOps {
  cudaError_t (*fwd)(const PlaneArgs<T> &, int npacks, cudaStream_t);
  cudaError_t (*inv)(const PlaneArgs<T> &, int ngroups, bool acc, cudaStream_t);
  bool acc_fits;  // the inverse pass can keep a plane of W_i partial sums in shared memory
};
bool plane_ops_f32_small(int n2, int n3, PlaneOps<float> *out);
bool plane_ops_f32_large(int n2, int n3, PlaneOps<float> *out);
bool plane_ops_f64(int n2, int n3, PlaneOps<double> *out);

// Persistent pair chain (persistent_chain.cuh): one launch walks every pack of one or more builds
// on one grid through a device-side task queue.
template <typename T>
struct ChainBuild {
  const T *phi;      // [norb][N]
  T *W;              // [norb][N], accumulated into
  const T *Kperm;    // Coulomb table in the plane passes' permuted layout
  const float *pmax; // [norb][N1] max |phi| over each plane i1 of each orbital (plane skip), or null
  const float *gmax; // [norb] max |phi| of each orbital
};
template <typename T>
struct PersistArgs {
  const ChainBuild<T> *builds;  // [builds]
  const int *pack_build;        // [npacks] build of each pack; null: every pack belongs to build 0
  const int4 *packs;            // [npacks] (a, b, c, d), c = d = -1 for a single pair
  int npacks;
  const int *npacks_d;          // non-null: the pack count, read on the device (npacks bounds it)
  cpx<T> *scratch;              // [nslots][N] complex
  int nslots;                   // >= 2 lag + 2
  int lag;                      // rounds between the stages of one pack in the queue
  const cpx<T> *tw1, *tw2, *tw3;
  int *counters;                // [3][npacks] finished F, C and I tasks per pack, zeroed
  int *ticket;                  // next task number, zeroed
  int *err;                     // set to 1 when a wait gives up
  long long N;
  unsigned long long wait_ns;   // time limit of one wait for a pack's earlier tasks
  const int *stall;             // null; else the pencil tasks wait for this word to reach 1 (a test)
  int hints;                    // as PlaneArgs::hints
  float skip_rel;               // as PlaneArgs::skip_rel (plane maxima in each ChainBuild)
};
template <typename T>
struct PersistOps {
  int (*blocks_per_sm)();
  cudaError_t (*launch)(const PersistArgs<T> &, int grid, cudaStream_t);
  int tasks_per_pack;  // F + C + I tasks
};
bool persist_ops_f32_small(int n1, int n2, int n3, PersistOps<float> *out);

// One build's device pack list for a concatenated queue: the packs of the screen's compaction
// (consecutive pairs two at a time) and the pair count it wrote.
struct QueueSrc {
  const int4 *packs;
  const int *count;
};
constexpr int kQueueMaxBuilds = 1024;
// Concatenates the pack lists of nb <= kQueueMaxBuilds builds, in build order, into packs_out,
// with the build of each pack in pack_build and the total pack count in *np_out (all on the device;
// the pair counts are read there).
// Plane maxima of the orbitals for the plane skip: pmax[a][i1] = max |phi_a| over plane i1 (npl
// points) and gmax[a] = max over all planes (gmax zeroed by the caller); n1 planes, norb orbitals.
cudaError_t launch_plane_max(const float *phi, int norb, int n1, long long npl, float *pmax, float *gmax,
                             cudaStream_t st);
// *dst[i] = 1 for every i < n if *src is non-zero (a give-up flag passed on to several builds).
cudaError_t launch_flag_fanout(const int *src, int *const *dst, int n, cudaStream_t st);
cudaError_t launch_queue_assemble(const QueueSrc *src, int nb, int4 *packs_out, int *pack_build, int *np_out,
                                  cudaStream_t st);
bool persist_ops_f32_large(int n1, int n2, int n3, PersistOps<float> *out);

// Launch one pass over `npacks` packs (grid.y); returns cudaErrorInvalidValue if the axis
// length has no compiled plan.
template <typename T>
cudaError_t launch_pair_pass(int mode, const PairPassArgs<T> &a, int npacks, cudaStream_t st);

// Axis-1 pass of the plane chain (32-column tiles, direct global stage-1 loads and stores).
template <typename T>
cudaError_t launch_conv_pass(const PairPassArgs<T> &a, int npacks, cudaStream_t st);

bool pass_length_supported(int L);
// Axis-1 pass of the plane chain compiled for this length (lengths up to 160)
bool conv_length_supported(int L);
// Two-stage factorisation L = r1 * r2 of a compiled axis length (output index k sits at
// position (k % r1) * r2 + k / r1 after a forward transform).
bool axis_factors(int L, int *r1, int *r2);

// Dense steps.
// partial (gram_chunks_bytes, or null): the CUDA-core Gram of the FP64 form writes chunk sums
// there and adds them in a fixed order (deterministic), instead of FP64 atomics across chunks.
template <typename T>
cudaError_t launch_gram(const T *X, int nx, const T *Y, int ny, long long K, double scale, bool abs_values,
                        bool upper_only, double *G, cudaStream_t st, double *partial = nullptr);
size_t gram_chunks_bytes(int nx, int ny, long long K);
template <typename T>
cudaError_t launch_left_mul(const T *A, int m, int n, const T *Y, long long K, T *Z, cudaStream_t st);

// gwork: n*n + n doubles of device workspace, needed when n > 128 (else may be NULL)
cudaError_t launch_cholesky(const double *M_raw, int n, double spin_factor, double *M, double *L, double *Linv,
                            double *energy, int *status, double *gwork, cudaStream_t st);
cudaError_t launch_screen_compact(const double *O, int n, double rho_cut, int2 *pairs, int4 *packs,
                                  int *count, double *O_sym, cudaStream_t st);

template <typename T>
cudaError_t launch_transpose_scale(const double *C, int n, int m, double scale, T *A, cudaStream_t st);

// Tensor-core (tcgen05) BF16x3 contractions for FP32 operands.  *err is set to 1 when a bounded
// wait inside the kernel gave up.  tc_shapes_ok: K a multiple of 128 (every tensor-core kernel);
// tc_gram_shape_ok: K a multiple of 32 (the Gram, whose last chunk may be short).
bool tc_shapes_ok(long long K);
bool tc_gram_shape_ok(long long K);
// Screen contribution of columns [0, K) of X (row stride ld): G += scale |X||X|^T, upper triangle.
cudaError_t launch_screen_cols(const float *X, int n, long long ld, long long K, double scale, double *G,
                               cudaStream_t st);
// Recompute the screen values within band * rho_cut of rho_cut from phi (n rows of N points) with
// FP32 products and compensated sums (upper triangle, off-diagonal).
cudaError_t launch_screen_refine(const float *phi, int n, long long N, double dV, double rho_cut, double band,
                                 double *O, cudaStream_t st);
// Screen contribution of the columns [c0, c0 + K) of phi (n rows of ld points) by the TMA-fed
// kernel; false (nothing launched) when TMA cannot be used for these operands.
bool launch_screen_tma(const float *X, int n, long long ld, long long c0, long long K, double scale, double *G,
                       int *err, cudaStream_t st);
// workspace of launch_tc_gram for these operands (the path it takes depends on them)
size_t tc_gram_workspace_bytes(const float *X, int nx, const float *Y, int ny, long long K);
cudaError_t launch_tc_gram(const float *X, int nx, const float *Y, int ny, long long K, double scale, double *G,
                           void *ws, int *err, cudaStream_t st, long *launches);
// Z = A Y (A m x n, Y n x K, Z m x K, FP32 row-major): the TMA kernel for any K % 4 == 0 (a
// short last column tile), else the register-staged kernel for K % 128 == 0; cudaErrorNotSupported
// (nothing launched) for other shapes.
cudaError_t launch_tc_left_mul(const float *A, int m, int n, const float *Y, long long K, float *Z, int *err,
                               cudaStream_t st);
// Screen contribution of the columns [c0, c0 + K) of phi (n rows of ld points) on the tensor cores:
// G += scale |X| |X|^T (the whole n x n matrix), BF16x3 products as in the Gram.  ws holds
// tc_screen_workspace_bytes (0: the plan does not apply).  false: nothing launched (no TMA map for
// these operands); true: launched, *e the launch status.
size_t tc_screen_workspace_bytes(const float *X, int n, long long K);
// Screen contribution of the columns [c0, c0 + K) of phi on the CUDA cores (FP32 products, FP64
// across K-splits): G += scale |X| |X|^T on the upper triangle.  ws holds
// screen_syrk_workspace_bytes(n, N) for any K <= N.  false: nothing launched (TMA cannot map phi);
// true: launched, *e the launch status.
// With pm (pmax of n x n1 floats and gmax of n floats, both zeroed before the first call), the
// kernel also takes atomic maxima of |phi| per (orbital, plane of npl points) and per orbital, the
// table of launch_plane_max, when c0 and npl are multiples of 32; *pm->done is cleared otherwise.
struct PlaneMaxOut {
  float *pmax, *gmax;
  long long npl;
  int n1;
  bool *done;
};
size_t screen_syrk_workspace_bytes(int n, long long K);
bool launch_screen_syrk(const float *X, int n, long long ld, long long c0, long long K, double scale, double *G,
                        void *ws, int *err, cudaStream_t st, long *launches, cudaError_t *e,
                        const PlaneMaxOut *pm = nullptr);
bool launch_tc_screen(const float *X, int n, long long ld, long long c0, long long K, double scale, double *G,
                      void *ws, int *err, cudaStream_t st, long *launches, cudaError_t *e);

// SCDM localisation (scdm.cu).  launch_scdm selects the n grid columns and computes the Loewdin
// factor; every output lives in the workspace `ws` (scdm_workspace_bytes, 256-byte aligned).
struct ScdmResult {
  int *piv;     // [n] selected grid indices, in selection order
  double *U;    // [n][n] FP64, phi_k = sum_i psi_i U[i][k]
  void *Ut;     // [n][n] U^T in the working type: the left factor of Phi = U^T Psi
  double *dev;  // [scdm_max_iterations()] max |T - I| of each Newton-Schulz iteration, 0 once skipped
  int *dependent;  // 1 if a chosen column lay in the span of the earlier ones (Psi of rank < n)
};
int scdm_max_iterations();
size_t scdm_workspace_bytes(int n, long long N, size_t elem);
template <typename T>
cudaError_t launch_scdm(const T *psi, int n, long long N, void *ws, cudaStream_t st, long *launches, ScdmResult *res);

// Sets the message returned by ace_last_error() on this thread.
void set_last_error(const char *msg);

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *in, Tout *out, long long count, double scale, cudaStream_t st);

}  // namespace ace
