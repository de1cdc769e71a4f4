// noalloc.cu -- ace_exchange_w_noalloc: the pair-potential chain (W_i = sum_j v_ij phi_j) with every
// byte of workspace taken from one fixed array compiled into the library, so that the call itself
// allocates nothing.
//
// Who needs this: code that must not call cudaMalloc or any allocator while it runs -- for example a
// host application that hands the library pre-allocated device buffers and forbids allocation after
// start-up (fixed memory budgets, allocator-free real-time loops, or a caller embedded in a framework
// that owns all device memory).  Such a caller passes the orbitals and the output W; the FFT
// workspace, the pack list, the Coulomb kernel table and the twiddles live in g_noalloc_scratch.
//
// Limits and sharing:
//   * the array holds ACE_NOALLOC_SCRATCH_BYTES (32 MiB).  Every GPU that loads the library holds
//     one copy of it until the process exits;
//   * one grid needs sizeof(T) * N (kernel table) + 2 sizeof(T) * N (one pack of FFT workspace)
//     + a few KB; larger grids are rejected with ACE_ERR_ARG before any work is queued;
//   * every call on a device uses the same array, and the array keeps the previous call's contents:
//     each call rewrites the tables and the pack list it reads and zeroes W before accumulating.
//     Calls whose work overlaps on the GPU (two streams, or two host threads) race on the array;
//     serialise them;
//   * the first call on a device looks up the array's device address with cudaGetSymbolAddress
//     (with that device current) and caches it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/ace.h"
#include "ace_internal.h"
#include "fft.cuh"

using ace::cpx;

namespace {

constexpr size_t kScratchBytes = ACE_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;
constexpr int kPackChunk = 4096;          // packs staged per upload
constexpr size_t kPackBytes = sizeof(int4) * kPackChunk;
constexpr size_t kTwBytes = 3 * 16 * 256;  // three axes, up to 256 complex doubles each

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_dev[kMaxDevices] = {};

ace_status nf_fail(ace_status st, const char *fmt, ...);

// Device address of g_noalloc_scratch on the current device (looked up once per device).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_dev[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// e^{-2 pi i e / L} from sincospi in double, rounded once to T
template <typename T>
__global__ void noalloc_twiddle_kernel(cpx<T> *tw, int L) {
  for (int e = threadIdx.x; e < L; e += blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)e / (double)L, &s, &c);
    tw[e] = cpx<T>{(T)c, (T)(-s)};
  }
}

// Kernel / N with |G|^2 = m^T g m (g = Gram matrix of the reciprocal basis), averaged over the
// +-N_k/2 choices at Nyquist indices: periodic 4 pi / |G|^2 with G = 0 -> 0, or (trunc) the
// isolated-cell kernel 4 pi (1 - cos(|G| rc)) / |G|^2 with its G = 0 limit 2 pi rc^2.
struct RecipGram {
  double g[3][3];
  int trunc;
  double rc;
};

template <typename T>
__global__ void noalloc_kernel_table(T *K, int n1, int n2, int n3, RecipGram rg) {
  const long long N = (long long)n1 * n2 * n3;
  const double fourpi_over_N = 4.0 * ace::kPi / (double)N;
  for (long long lin = blockIdx.x * (long long)blockDim.x + threadIdx.x; lin < N;
       lin += (long long)gridDim.x * blockDim.x) {
    const int i3 = (int)(lin % n3);
    const int i2 = (int)((lin / n3) % n2);
    const int i1 = (int)(lin / ((long long)n2 * n3));
    const int idx[3] = {i1, i2, i3}, nn[3] = {n1, n2, n3};
    int m[3];
    bool nyq[3];
    for (int k = 0; k < 3; ++k) {
      m[k] = (2 * idx[k] < nn[k]) ? idx[k] : idx[k] - nn[k];
      nyq[k] = (nn[k] % 2 == 0) && (2 * idx[k] == nn[k]);
    }
    if (m[0] == 0 && m[1] == 0 && m[2] == 0) {
      K[lin] = rg.trunc ? (T)(fourpi_over_N * 0.5 * rg.rc * rg.rc) : (T)0;
      continue;
    }
    double acc = 0.0;
    int cnt = 0;
    for (int s = 0; s < 8; ++s) {
      bool ok = true;
      double mm[3];
      for (int k = 0; k < 3; ++k) {
        const bool flip = (s >> k) & 1;
        if (flip && !nyq[k]) ok = false;
        mm[k] = flip ? -m[k] : m[k];
      }
      if (!ok) continue;
      double q = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) q += mm[k] * mm[l] * rg.g[k][l];
      acc += rg.trunc ? (1.0 - cos(sqrt(q) * rg.rc)) / q : 1.0 / q;
      ++cnt;
    }
    K[lin] = (T)(fourpi_over_N * acc / cnt);
  }
}

template <typename T>
ace_status run_noalloc(const ace_desc &d, const T *phi, const int *pairs, long npairs, T *W, cudaStream_t st) {
  const int n = d.norb;
  const long long N = (long long)d.n[0] * d.n[1] * d.n[2];
  const size_t k_bytes = align256(sizeof(T) * (size_t)N);
  const size_t pack_ws = sizeof(cpx<T>) * (size_t)N;
  const size_t fixed = kPackBytes + kTwBytes + k_bytes;
  if (fixed + pack_ws > kScratchBytes)
    return nf_fail(ACE_ERR_ARG,
                   "grid %dx%dx%d needs %zu bytes of workspace in the no-allocation path; its fixed array holds "
                   "%zu bytes",
                   d.n[0], d.n[1], d.n[2], fixed + pack_ws, kScratchBytes);
  // pair indices are checked on the host before anything is queued
  for (long p = 0; p < npairs; ++p) {
    const int i = pairs[2 * p], j = pairs[2 * p + 1];
    if (i < 0 || j < i || j >= n) return nf_fail(ACE_ERR_ARG, "pair %ld = (%d, %d) is not 0 <= i <= j < norb", p, i, j);
  }
  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return nf_fail(ACE_ERR_CUDA, "scratch address: %s", cudaGetErrorString(e));
  unsigned char *b = static_cast<unsigned char *>(base);
  int4 *packs_d = reinterpret_cast<int4 *>(b);
  cpx<T> *tw_d[3];
  for (int a = 0; a < 3; ++a) tw_d[a] = reinterpret_cast<cpx<T> *>(b + kPackBytes + a * 16 * 256);
  T *K_d = reinterpret_cast<T *>(b + kPackBytes + kTwBytes);
  cpx<T> *ws_d = reinterpret_cast<cpx<T> *>(b + fixed);
  const int batch_cap = (int)((kScratchBytes - fixed) / pack_ws);

  // tables (rewritten on every call: the array keeps whatever the previous call left)
  const double *A = &d.lattice[0][0];
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  double adj[9] = {A[4] * A[8] - A[5] * A[7], A[2] * A[7] - A[1] * A[8], A[1] * A[5] - A[2] * A[4],
                   A[5] * A[6] - A[3] * A[8], A[0] * A[8] - A[2] * A[6], A[2] * A[3] - A[0] * A[5],
                   A[3] * A[7] - A[4] * A[6], A[1] * A[6] - A[0] * A[7], A[0] * A[4] - A[1] * A[3]};
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return nf_fail(ACE_ERR_ARG, "lattice is singular");
  double B[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) B[k][c] = 2.0 * ace::kPi * adj[c * 3 + k] / det;
  RecipGram rg;
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) rg.g[k][l] = B[k][0] * B[l][0] + B[k][1] * B[l][1] + B[k][2] * B[l][2];
  rg.trunc = d.coulomb == ACE_COULOMB_TRUNCATED;
  rg.rc = d.r_cut;
  if (rg.trunc && !(rg.rc > 0.0)) {  // radius of the largest sphere inside the cell
    rg.rc = HUGE_VAL;
    for (int k = 0; k < 3; ++k) rg.rc = std::min(rg.rc, ace::kPi / std::sqrt(rg.g[k][k]));
  }
  for (int a = 0; a < 3; ++a) noalloc_twiddle_kernel<T><<<1, 256, 0, st>>>(tw_d[a], d.n[a]);
  noalloc_kernel_table<T><<<(unsigned)std::min<long long>((N + 255) / 256, 4096), 256, 0, st>>>(K_d, d.n[0], d.n[1],
                                                                                              d.n[2], rg);
  e = cudaMemsetAsync(W, 0, sizeof(T) * (size_t)n * N, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return nf_fail(ACE_ERR_CUDA, "tables: %s", cudaGetErrorString(e));

  ace::PairPassArgs<T> a;
  a.phi = phi;
  a.W = W;
  a.scratch = ws_d;
  a.packs = packs_d;
  a.kernel = K_d;
  a.N = N;
  a.n1 = d.n[0];
  a.n2 = d.n[1];
  a.n3 = d.n[2];
  const long npacks = (npairs + 1) / 2;
  int4 host_packs[256];  // staged through a small stack buffer, 256 packs per upload
  for (long c0 = 0; c0 < npacks; c0 += kPackChunk) {
    const long cn = std::min<long>(kPackChunk, npacks - c0);
    for (long s0 = 0; s0 < cn; s0 += 256) {
      const long sn = std::min<long>(256, cn - s0);
      for (long q = 0; q < sn; ++q) {
        const long p = 2 * (c0 + s0 + q);
        const bool two = p + 1 < npairs;
        host_packs[q] = make_int4(pairs[2 * p], pairs[2 * p + 1], two ? pairs[2 * p + 2] : -1,
                                  two ? pairs[2 * p + 3] : -1);
      }
      // pageable source: the call returns once host_packs has been consumed
      e = cudaMemcpyAsync(packs_d + s0, host_packs, sizeof(int4) * sn, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return nf_fail(ACE_ERR_CUDA, "pack upload: %s", cudaGetErrorString(e));
    }
    for (long p0 = 0; p0 < cn; p0 += batch_cap) {
      const int nb = (int)std::min<long>(batch_cap, cn - p0);
      a.pack0 = (int)p0;
      const int modes[5] = {ace::PASS_FWD3_PAIR, ace::PASS_FWD2, ace::PASS_CONV1, ace::PASS_INV2, ace::PASS_INV3_ACC};
      const int axis[5] = {2, 1, 0, 1, 2};
      for (int k = 0; k < 5; ++k) {
        a.tw = tw_d[axis[k]];
        e = ace::launch_pair_pass<T>(modes[k], a, nb, st);
        if (e != cudaSuccess) return nf_fail(ACE_ERR_CUDA, "pair pass: %s", cudaGetErrorString(e));
      }
    }
  }
  return ACE_OK;
}

ace_status nf_fail(ace_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  ace::set_last_error(buf);  // readable through ace_last_error()
  return st;
}

}  // namespace

extern "C" {

ace_status ace_exchange_w_noalloc(const ace_desc *desc, const void *phi_dev, ace_dtype dtype, const int *pairs_host,
                                  long npairs, void *W_dev, void *cuda_stream) {
  if (!desc || !phi_dev || !W_dev || (npairs > 0 && !pairs_host) || npairs < 0)
    return nf_fail(ACE_ERR_ARG, "NULL argument or negative pair count");
  if (desc->norb < 1) return nf_fail(ACE_ERR_ARG, "norb = %d < 1", desc->norb);
  if ((reinterpret_cast<uintptr_t>(phi_dev) | reinterpret_cast<uintptr_t>(W_dev)) & 15)
    return nf_fail(ACE_ERR_ARG, "phi_dev and W_dev must be 16-byte aligned");
  for (int k = 0; k < 3; ++k)
    if (!ace::pass_length_supported(desc->n[k]))
      return nf_fail(ACE_ERR_UNSUPPORTED_GRID, "grid axis %d length %d has no compiled FFT plan", k, desc->n[k]);
  if (desc->coulomb != ACE_COULOMB_PERIODIC && desc->coulomb != ACE_COULOMB_TRUNCATED)
    return nf_fail(ACE_ERR_ARG, "unknown Coulomb kernel %d", (int)desc->coulomb);
  if (desc->coulomb == ACE_COULOMB_TRUNCATED && !std::isfinite(desc->r_cut))
    return nf_fail(ACE_ERR_ARG, "non-finite r_cut");
  const bool fp64 = desc->prec == ACE_FP64;
  if ((fp64 && dtype != ACE_F64) || (!fp64 && dtype != ACE_F32))
    return nf_fail(ACE_ERR_ARG, "dtype must be the working type of the precision (F64 for ACE_FP64, F32 for ACE_MIXED)");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (fp64)
    return run_noalloc<double>(*desc, static_cast<const double *>(phi_dev), pairs_host, npairs,
                               static_cast<double *>(W_dev), st);
  return run_noalloc<float>(*desc, static_cast<const float *>(phi_dev), pairs_host, npairs, static_cast<float *>(W_dev),
                            st);
}

}  // extern "C"
