// scdm.cu -- SCDM localisation (selected columns of the density matrix), the unitary change of
// basis of section II (Eq. unit) that turns canonical orbitals into the localized orbitals the pair
// screen needs:
//   1. greedy column-pivoted QR of Psi^T (norb x N, column r = psi(r)): step k takes the grid point
//      of largest residual norm d(r) = |psi(r)|^2 - sum_{j<k} (u_j . psi(r))^2 (first index on
//      ties) and extends the orthonormal basis u_j of the chosen columns;
//   2. M[i][j] = psi_i(c_j), the selected columns of the density matrix P = Psi Psi^T;
//   3. symmetric orthonormalisation: U = M (M^T M)^{-1/2}, phi_k = sum_i psi_i U[i][k].
// The inverse square root is the coupled Newton-Schulz iteration (Higham, "Functions of Matrices",
// 2008, section 6.3) on A = S / |S|_F: Y0 = A, Z0 = I, T = (3 I - Z Y) / 2, Y <- Y T, Z <- T Z, with
// Z -> A^{-1/2} quadratically once |I - Z Y| < 1.  Only FP64 and FP32 ALU arithmetic is used: the
// contractions are n x n, far too small for the tensor cores to matter.
#include <cuda_runtime.h>

#include <algorithm>

#include "ace_internal.h"

namespace ace {
namespace {

constexpr int kSelNT = 256;  // threads of the one-CTA selection kernel
constexpr int kUpdNT = 256;  // threads of the streaming update kernel
constexpr int kUpdBlocks = 152 * 4;
constexpr int kNsMax = 64;          // Newton-Schulz iterations at most
constexpr double kNsStop = 1e-12;   // max |T - I| below which the following iterations are skipped
constexpr int kChunk = 16;          // products summed in the working type before the FP64 add
constexpr double kDependent = 1e-24;  // |residual|^2 / |psi(c)|^2 below which a column is dependent

// (value, index) maximum, the smaller index winning ties
__device__ __forceinline__ void amax(double &v, long long &i, double v2, long long i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

__device__ __forceinline__ void warp_amax(double &v, long long &i) {
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_down_sync(0xffffffffu, v, o);
    const long long i2 = __shfl_down_sync(0xffffffffu, i, o);
    amax(v, i, v2, i2);
  }
}

// sum_i a_i psi_i(r) over the n orbitals (a = nullptr: sum_i psi_i(r)^2), chunks of kChunk products
// in T added in FP64.  psi is [n][N].
template <typename T>
__device__ __forceinline__ double project(const T *__restrict__ psi, int n, long long N, long long r,
                                          const T *__restrict__ a) {
  double p = 0.0;
  int i0 = 0;
  for (; i0 + kChunk <= n; i0 += kChunk) {
    T v[kChunk];
#pragma unroll
    for (int t = 0; t < kChunk; ++t) v[t] = psi[(long long)(i0 + t) * N + r];
    T part = (T)0;
#pragma unroll
    for (int t = 0; t < kChunk; ++t) part += (a ? a[i0 + t] : v[t]) * v[t];
    p += (double)part;
  }
  T part = (T)0;
  for (int i = i0; i < n; ++i) {
    const T v = psi[(long long)i * N + r];
    part += (a ? a[i] : v) * v;
  }
  return p + (double)part;
}

// Residual norms of the candidate columns and their block maxima.
//   u == nullptr: d[r] = |psi(r)|^2 (the start);
//   else:         d[r] -= (u . psi(r))^2 for every column still a candidate (d[r] >= 0).
template <typename T>
__global__ void __launch_bounds__(kUpdNT) scdm_update_kernel(const T *__restrict__ psi, int n, long long N,
                                                             const double *__restrict__ u, double *__restrict__ d,
                                                             double *__restrict__ bval, long long *__restrict__ bidx) {
  __shared__ T us[1024];
  __shared__ double rv[kUpdNT / 32];
  __shared__ long long ri[kUpdNT / 32];
  if (u)
    for (int i = threadIdx.x; i < n; i += blockDim.x) us[i] = (T)u[i];
  __syncthreads();
  double best = -2.0;
  long long bi = N;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N; r += (long long)gridDim.x * blockDim.x) {
    double dr;
    if (!u) {
      dr = project<T>(psi, n, N, r, nullptr);
      d[r] = dr;
    } else {
      dr = d[r];
      if (dr >= 0.0) {
        const double p = project<T>(psi, n, N, r, us);
        dr = fmax(dr - p * p, 0.0);
        d[r] = dr;
      }
    }
    amax(best, bi, dr, r);
  }
  warp_amax(best, bi);
  if ((threadIdx.x & 31) == 0) {
    rv[threadIdx.x >> 5] = best;
    ri[threadIdx.x >> 5] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kUpdNT / 32; ++w) amax(best, bi, rv[w], ri[w]);
    bval[blockIdx.x] = best;
    bidx[blockIdx.x] = bi;
  }
}

// Step k on one CTA: the pivot c_k from the block maxima (it leaves the candidate set), then
// u_k = psi(c_k) orthogonalised against u_0..u_{k-1} by classical Gram-Schmidt applied twice and
// normalised.  Ub is [n][n] with row j = u_j.  A column with no residual left gives u_k = 0 and
// sets *dependent.
template <typename T>
__global__ void __launch_bounds__(kSelNT) scdm_select_kernel(const T *__restrict__ psi, int n, long long N,
                                                             const double *__restrict__ bval,
                                                             const long long *__restrict__ bidx, int nblk,
                                                             double *__restrict__ Ub, int k, int *__restrict__ piv,
                                                             double *__restrict__ d, int *__restrict__ dependent) {
  __shared__ double u[1024], c[1024];
  __shared__ double rv[kSelNT / 32], rv0[kSelNT / 32];
  __shared__ long long ri[kSelNT / 32];
  __shared__ long long chosen;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kSelNT / 32;
  double best = -2.0;
  long long bi = N;
  for (int b = tid; b < nblk; b += kSelNT) amax(best, bi, bval[b], bidx[b]);
  warp_amax(best, bi);
  if (lane == 0) {
    rv[warp] = best;
    ri[warp] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kWarps; ++w) amax(best, bi, rv[w], ri[w]);
    chosen = bi < N ? bi : 0;
    piv[k] = (int)chosen;
    d[chosen] = -1.0;
  }
  __syncthreads();
  const long long cr = chosen;
  double part0 = 0.0;
  for (int i = tid; i < n; i += kSelNT) {
    u[i] = (double)psi[(long long)i * N + cr];
    part0 += u[i] * u[i];
  }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int j = warp; j < k; j += kWarps) {  // c_j = u_j . u, one warp per j
      double s = 0.0;
      for (int i = lane; i < n; i += 32) s += Ub[(long long)j * n + i] * u[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) c[j] = s;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kSelNT) {  // u -= sum_j c_j u_j
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += c[j] * Ub[(long long)j * n + i];
      u[i] -= s;
    }
    __syncthreads();
  }
  double part = 0.0;
  for (int i = tid; i < n; i += kSelNT) part += u[i] * u[i];
  for (int o = 16; o > 0; o >>= 1) {
    part += __shfl_down_sync(0xffffffffu, part, o);
    part0 += __shfl_down_sync(0xffffffffu, part0, o);
  }
  if (lane == 0) {
    rv[warp] = part;
    rv0[warp] = part0;
  }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0, s0 = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      s += rv[w];
      s0 += rv0[w];
    }
    // the chosen column lies in the span of the earlier ones (to rounding): Psi has rank < n
    const bool dep = !(s > kDependent * s0);
    if (dep) *dependent = 1;
    c[0] = dep ? 0.0 : 1.0 / sqrt(s);
  }
  __syncthreads();
  const double inv = c[0];
  for (int i = tid; i < n; i += kSelNT) Ub[(long long)k * n + i] = u[i] * inv;
}

// M[i][j] = psi_i(c_j)
template <typename T>
__global__ void scdm_gather_kernel(const T *__restrict__ psi, int n, long long N, const int *__restrict__ piv,
                                   double *__restrict__ M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e / n, j = e % n;
  M[e] = (double)psi[(long long)i * N + piv[j]];
}

// S = M^T M
__global__ void gram_t_kernel(const double *__restrict__ M, int n, double *__restrict__ S) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e / n, j = e % n;
  double s = 0.0;
  for (int l = 0; l < n; ++l) s += M[(long long)l * n + i] * M[(long long)l * n + j];
  S[e] = s;
}

// f = |S|_F (one CTA)
__global__ void frob_kernel(const double *__restrict__ S, int n, double *__restrict__ f) {
  __shared__ double rv[kSelNT / 32];
  double part = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) part += S[e] * S[e];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) rv[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kSelNT / 32; ++w) s += rv[w];
    *f = sqrt(s);
  }
}

// Y0 = S / f, Z0 = I
__global__ void ns_start_kernel(const double *__restrict__ S, int n, const double *__restrict__ f,
                                double *__restrict__ Y, double *__restrict__ Z) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const double inv = *f > 0.0 ? 1.0 / *f : 0.0;
  Y[e] = S[e] * inv;
  Z[e] = (e / n == e % n) ? 1.0 : 0.0;
}

// Iteration `it`: T = (3 I - Z Y) / 2 and dev[it] = max |T - I|.  Skipped (T left unused) once an
// earlier iteration reached kNsStop.
__global__ void ns_t_kernel(const double *__restrict__ Y, const double *__restrict__ Z, int n,
                            double *__restrict__ Tm, double *__restrict__ dev, int it) {
  if (it > 0 && dev[it - 1] < kNsStop) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double x = 0.0;
  if (e < n * n) {
    const int i = e / n, j = e % n;
    double s = 0.0;
    for (int l = 0; l < n; ++l) s += Z[(long long)i * n + l] * Y[(long long)l * n + j];
    const double t = -0.5 * s + (i == j ? 1.5 : 0.0);
    Tm[e] = t;
    x = fabs(t - (i == j ? 1.0 : 0.0));
    if (!(x == x)) x = 1e300;  // NaN: never converged
  }
  for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_down_sync(0xffffffffu, x, o));
  // non-negative doubles order like their bit patterns
  if ((threadIdx.x & 31) == 0 && x > 0.0)
    atomicMax(reinterpret_cast<unsigned long long *>(dev + it), (unsigned long long)__double_as_longlong(x));
}

// Y' = Y T and Z' = T Z (threads [0, n^2) and [n^2, 2 n^2)); a skipped iteration copies Y and Z.
__global__ void ns_yz_kernel(const double *__restrict__ Y, const double *__restrict__ Z,
                             const double *__restrict__ Tm, int n, double *__restrict__ Y2, double *__restrict__ Z2,
                             const double *__restrict__ dev, int it) {
  const bool skip = it > 0 && dev[it - 1] < kNsStop;
  const int nn = n * n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * nn) return;
  const bool isz = e >= nn;
  const int f = isz ? e - nn : e;
  if (skip) {
    (isz ? Z2 : Y2)[f] = (isz ? Z : Y)[f];
    return;
  }
  const int i = f / n, j = f % n;
  double s = 0.0;
  if (!isz)
    for (int l = 0; l < n; ++l) s += Y[(long long)i * n + l] * Tm[(long long)l * n + j];
  else
    for (int l = 0; l < n; ++l) s += Tm[(long long)i * n + l] * Z[(long long)l * n + j];
  (isz ? Z2 : Y2)[f] = s;
}

// U = M Z / sqrt(f) (Z = (S/f)^{-1/2}) in FP64, and its transpose in the working type
template <typename T>
__global__ void scdm_factor_kernel(const double *__restrict__ M, const double *__restrict__ Z, int n,
                                   const double *__restrict__ f, double *__restrict__ U, T *__restrict__ Ut) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e / n, j = e % n;
  double s = 0.0;
  for (int l = 0; l < n; ++l) s += M[(long long)i * n + l] * Z[(long long)l * n + j];
  s /= sqrt(*f);
  U[e] = s;
  Ut[(long long)j * n + i] = (T)s;
}

struct Layout {
  size_t d, bval, bidx, Ub, M, S, Y0, Y1, Z0, Z1, Tm, U, Ut, f, dev, piv, dependent, total;
};

Layout layout(int n, long long N, size_t elem) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += (bytes + 255) / 256 * 256;
    return at;
  };
  const size_t nn = (size_t)n * n;
  L.d = take(sizeof(double) * (size_t)N);
  L.bval = take(sizeof(double) * kUpdBlocks);
  L.bidx = take(sizeof(long long) * kUpdBlocks);
  L.Ub = take(sizeof(double) * nn);
  L.M = take(sizeof(double) * nn);
  L.S = take(sizeof(double) * nn);
  L.Y0 = take(sizeof(double) * nn);
  L.Y1 = take(sizeof(double) * nn);
  L.Z0 = take(sizeof(double) * nn);
  L.Z1 = take(sizeof(double) * nn);
  L.Tm = take(sizeof(double) * nn);
  L.U = take(sizeof(double) * nn);
  L.Ut = take(elem * nn);
  L.f = take(sizeof(double));
  L.dev = take(sizeof(double) * kNsMax);
  L.piv = take(sizeof(int) * (size_t)n);
  L.dependent = take(sizeof(int));
  L.total = off;
  return L;
}

}  // namespace

int scdm_max_iterations() { return kNsMax; }

size_t scdm_workspace_bytes(int n, long long N, size_t elem) { return layout(n, N, elem).total; }

template <typename T>
cudaError_t launch_scdm(const T *psi, int n, long long N, void *ws, cudaStream_t st, long *launches, ScdmResult *res) {
  const Layout L = layout(n, N, sizeof(T));
  char *w = static_cast<char *>(ws);
  double *d = reinterpret_cast<double *>(w + L.d);
  double *bval = reinterpret_cast<double *>(w + L.bval);
  long long *bidx = reinterpret_cast<long long *>(w + L.bidx);
  double *Ub = reinterpret_cast<double *>(w + L.Ub);
  double *M = reinterpret_cast<double *>(w + L.M);
  double *S = reinterpret_cast<double *>(w + L.S);
  double *Y[2] = {reinterpret_cast<double *>(w + L.Y0), reinterpret_cast<double *>(w + L.Y1)};
  double *Z[2] = {reinterpret_cast<double *>(w + L.Z0), reinterpret_cast<double *>(w + L.Z1)};
  double *Tm = reinterpret_cast<double *>(w + L.Tm);
  double *f = reinterpret_cast<double *>(w + L.f);
  res->piv = reinterpret_cast<int *>(w + L.piv);
  res->U = reinterpret_cast<double *>(w + L.U);
  res->Ut = w + L.Ut;
  res->dev = reinterpret_cast<double *>(w + L.dev);
  res->dependent = reinterpret_cast<int *>(w + L.dependent);
  cudaError_t e = cudaMemsetAsync(res->dev, 0, sizeof(double) * kNsMax, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(res->dependent, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  // column selection: n streaming passes over Psi, each followed by the one-CTA pivot step
  for (int k = 0; k < n; ++k) {
    scdm_update_kernel<T><<<kUpdBlocks, kUpdNT, 0, st>>>(psi, n, N, k ? Ub + (size_t)(k - 1) * n : nullptr, d, bval,
                                                         bidx);
    scdm_select_kernel<T><<<1, kSelNT, 0, st>>>(psi, n, N, bval, bidx, kUpdBlocks, Ub, k, res->piv, d,
                                                res->dependent);
  }
  *launches += 2L * n;
  // Loewdin factor
  const int nn = n * n;
  const unsigned g1 = (unsigned)((nn + 255) / 256), g2 = (unsigned)((2 * nn + 255) / 256);
  scdm_gather_kernel<T><<<g1, 256, 0, st>>>(psi, n, N, res->piv, M);
  gram_t_kernel<<<g1, 256, 0, st>>>(M, n, S);
  frob_kernel<<<1, kSelNT, 0, st>>>(S, n, f);
  ns_start_kernel<<<g1, 256, 0, st>>>(S, n, f, Y[0], Z[0]);
  *launches += 4;
  for (int it = 0; it < kNsMax; ++it) {
    const int a = it & 1;
    ns_t_kernel<<<g1, 256, 0, st>>>(Y[a], Z[a], n, Tm, res->dev, it);
    ns_yz_kernel<<<g2, 256, 0, st>>>(Y[a], Z[a], Tm, n, Y[a ^ 1], Z[a ^ 1], res->dev, it);
  }
  *launches += 2L * kNsMax;
  scdm_factor_kernel<T><<<g1, 256, 0, st>>>(M, Z[kNsMax & 1], n, f, res->U, reinterpret_cast<T *>(res->Ut));
  *launches += 1;
  return cudaGetLastError();
}

template cudaError_t launch_scdm<float>(const float *, int, long long, void *, cudaStream_t, long *, ScdmResult *);
template cudaError_t launch_scdm<double>(const double *, int, long long, void *, cudaStream_t, long *, ScdmResult *);

}  // namespace ace
