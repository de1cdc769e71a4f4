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
#include <cstdint>

#include "ace_internal.h"

namespace ace {
namespace {

constexpr int kSelNT = 256;  // threads of the one-CTA reduction kernel
constexpr int kUpdNT = 256;  // threads of the streaming selection kernels
constexpr int kUpdBlocks = 1024;  // most blocks of a selection pass (sizes the block-maximum arrays)
constexpr int kNsMax = 64;          // Newton-Schulz iterations at most
constexpr int kNsChunk = 16;        // iterations launched between host checks of convergence
constexpr double kNsStop = 1e-12;   // max |T - I| below which the following iterations are skipped
constexpr int kChunk = 8;           // products summed in the working type before the FP64 add
constexpr double kDependent = 1e-24;    // |residual|^2 / |psi(c)|^2 below which a column is dependent
constexpr double kDependent32 = 1e-10;  // the same with FP32 Gram-Schmidt

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

// State of the greedy selection passed to the streaming kernels.  Each pass publishes one
// (maximum, index) per block; the block that publishes last takes the pivot step of the pass, so
// that no separate launch (and no waiting) sits between the passes.
struct SelArgs {
  double *bval;          // [gridDim.x] block maxima of the residual norms
  long long *bidx;       // [gridDim.x] their grid indices
  unsigned int *count;   // blocks of the current pass that have published (the last one resets it)
  void *Ub;              // [n][ldu] of the working type, row j = u_j, ldu = n rounded up to even
                         // (pad column zero)
  int *piv;              // [n]
  int *dependent;        // set when a chosen column lies in the span of the earlier ones
  int k;                 // step whose pivot this pass selects
};

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// Shared memory of a streaming block: u_{k-1} while streaming, the pivot step's vectors afterwards.
template <typename T>
struct __align__(16) ScdmSmem {
  struct {
    T u[1024], c[1024], red2[1024];
  } sel;
  T us[1024];
  double rv[kUpdNT / 32], rv0[kUpdNT / 32];
  long long ri[kUpdNT / 32];
  long long chosen;
  int last;
};

// Pivot step k, run by the whole last block of a pass: the pivot c_k from the block maxima (it
// leaves the candidate set), then u_k = psi(c_k) orthogonalised against u_0..u_{k-1} by classical
// Gram-Schmidt applied twice and normalised, in the working type T.  The basis u_j only steers the
// choice of the pivots (U and Phi are computed from the pivots and Psi alone).  A column whose
// residual is at the rounding level of T (|residual|^2 below kDependent(T) |psi(c_k)|^2) gives
// u_k = 0 and sets *dependent.
template <typename T>
__device__ void pivot_step(const T *__restrict__ psi, long long si, long long sr, int n, long long N, int nblk,
                           double *__restrict__ d, const SelArgs &s, ScdmSmem<T> &sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kUpdNT / 32;
  using V2 = typename Vec2<T>::type;
  T *u = sm.sel.u, *c = sm.sel.c;
  const T *Ub = static_cast<const T *>(s.Ub);
  const int k = s.k;
  double best = -2.0;
  long long bi = N;
  for (int b = tid; b < nblk; b += kUpdNT) amax(best, bi, __ldcg(s.bval + b), __ldcg(s.bidx + b));
  warp_amax(best, bi);
  if (lane == 0) {
    sm.rv[warp] = best;
    sm.ri[warp] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kWarps; ++w) amax(best, bi, sm.rv[w], sm.ri[w]);
    sm.chosen = bi < N ? bi : 0;
    s.piv[k] = (int)sm.chosen;
    d[sm.chosen] = -1.0;
  }
  __syncthreads();
  const long long cr = sm.chosen;
  const int ldu = (n + 1) & ~1, np = ldu / 2;  // Ub row stride (even; the pad column is zero)
  T part0 = (T)0;
  for (int i = tid; i < ldu; i += kUpdNT) {
    u[i] = i < n ? psi[(long long)i * si + cr * sr] : (T)0;
    part0 += u[i] * u[i];
  }
  __syncthreads();
  const V2 *u2 = reinterpret_cast<const V2 *>(u);
  const int S = np <= 64 ? 4 : (np <= 128 ? 2 : 1);  // row slices of the u update (S ldu <= 1024)
  for (int pass = 0; pass < 2; ++pass) {
    // c_j = u_j . u: 16 lanes per row over consecutive double2, four rows per thread per round
    {
      const int seg = tid & 15, rg = tid >> 4;
      for (int j0 = 0; j0 < k; j0 += 64) {  // same trip count for every thread of the block
        const V2 *q[4];
        T a[4] = {(T)0, (T)0, (T)0, (T)0};
#pragma unroll
        for (int t = 0; t < 4; ++t)
          q[t] = reinterpret_cast<const V2 *>(Ub + (long long)min(j0 + rg + 16 * t, k - 1) * ldu);
#pragma unroll 2
        for (int p = seg; p < np; p += 16) {
          const V2 w = u2[p];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const V2 x = q[t][p];
            a[t] += x.x * w.x + x.y * w.y;
          }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          for (int o = 8; o > 0; o >>= 1) a[t] += __shfl_xor_sync(0xffffffffu, a[t], o);
          if (seg == 0 && j0 + rg + 16 * t < k) c[j0 + rg + 16 * t] = a[t];
        }
      }
    }
    __syncthreads();
    // u -= sum_j c_j u_j: S slices of the rows x (256 / S) threads over pairs of u; the slices'
    // partial sums are added in a fixed order
    {
      const int tps = kUpdNT / S, sl = tid / tps, e0 = tid % tps;
      for (int p = e0; p < np; p += tps) {
        T ax = (T)0, ay = (T)0;
#pragma unroll 8
        for (int j = sl; j < k; j += S) {
          const V2 x = reinterpret_cast<const V2 *>(Ub + (long long)j * ldu)[p];
          const T cj = c[j];
          ax += cj * x.x;
          ay += cj * x.y;
        }
        sm.sel.red2[sl * ldu + 2 * p] = ax;
        sm.sel.red2[sl * ldu + 2 * p + 1] = ay;
      }
    }
    __syncthreads();
    for (int i = tid; i < n; i += kUpdNT) {
      T t = (T)0;
      for (int s2 = 0; s2 < S; ++s2) t += sm.sel.red2[s2 * ldu + i];
      u[i] -= t;
    }
    __syncthreads();
  }
  T part = (T)0;
  for (int i = tid; i < n; i += kUpdNT) part += u[i] * u[i];
  for (int o = 16; o > 0; o >>= 1) {
    part += __shfl_down_sync(0xffffffffu, part, o);
    part0 += __shfl_down_sync(0xffffffffu, part0, o);
  }
  if (lane == 0) {
    sm.rv[warp] = (double)part;
    sm.rv0[warp] = (double)part0;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0, t0 = 0.0;
    for (int w = 0; w < kWarps; ++w) {
      t += sm.rv[w];
      t0 += sm.rv0[w];
    }
    // the chosen column lies in the span of the earlier ones (to rounding): Psi has rank < n
    const bool dep = !(t > (sizeof(T) == 4 ? kDependent32 : kDependent) * t0);
    if (dep) *s.dependent = 1;
    c[0] = dep ? (T)0 : (T)(1.0 / sqrt(t));
  }
  __syncthreads();
  const T inv = c[0];
  T *Uw = static_cast<T *>(s.Ub);
  for (int i = tid; i < ldu; i += kUpdNT) Uw[(long long)k * ldu + i] = i < n ? u[i] * inv : (T)0;
}

// End of a pass for one block: publish the block maximum; the last block to publish takes the
// pivot step and resets the counter for the next pass.  Orbital i at point r is psi[i si + r sr].
template <typename T>
__device__ void finish_pass(double best, long long bi, const T *__restrict__ psi, long long si, long long sr, int n,
                            long long N, double *__restrict__ d, const SelArgs &s, ScdmSmem<T> &sm) {
  const int tid = threadIdx.x;
  warp_amax(best, bi);
  if ((tid & 31) == 0) {
    sm.rv[tid >> 5] = best;
    sm.ri[tid >> 5] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < kUpdNT / 32; ++w) amax(best, bi, sm.rv[w], sm.ri[w]);
    s.bval[blockIdx.x] = best;
    s.bidx[blockIdx.x] = bi;
    __threadfence();  // the maximum (and this block's residual norms) before the count
    sm.last = atomicAdd(s.count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!sm.last) return;
  __threadfence();
  pivot_step<T>(psi, si, sr, n, N, gridDim.x, d, s, sm);
  if (tid == 0) *s.count = 0u;
}

// One selection pass, any T and any N (one point per thread per iteration):
//   NORM: d[r] = |psi(r)|^2 (the start);
//   else: d[r] -= (u_{k-1} . psi(r))^2 for every column still a candidate (d[r] >= 0), u_{k-1} = row
//         k-1 of Ub.
// Products are summed in T in chunks of kChunk, the chunks in FP64.
template <typename T, bool NORM>
__global__ void __launch_bounds__(kUpdNT) scdm_pass_kernel(const T *__restrict__ psi, int n, long long N,
                                                           double *__restrict__ d, SelArgs s) {
  __shared__ ScdmSmem<T> sm;
  if (!NORM)
    for (int i = threadIdx.x; i < n; i += kUpdNT)
      sm.us[i] = static_cast<const T *>(s.Ub)[(long long)(s.k - 1) * ((n + 1) & ~1) + i];
  __syncthreads();
  double best = -2.0;
  long long bi = N;
  for (long long r = blockIdx.x * (long long)kUpdNT + threadIdx.x; r < N; r += (long long)gridDim.x * kUpdNT) {
    double dr = NORM ? 0.0 : d[r];
    if (NORM || dr >= 0.0) {
      double p = 0.0;
      for (int i0 = 0; i0 < n; i0 += kChunk) {
        const int i1 = min(n, i0 + kChunk);
        T part = (T)0;
        for (int i = i0; i < i1; ++i) {
          const T v = psi[(long long)i * N + r];
          part += (NORM ? v : sm.us[i]) * v;
        }
        p += (double)part;
      }
      dr = NORM ? p : fmax(dr - p * p, 0.0);
      d[r] = dr;
    }
    amax(best, bi, dr, r);
  }
  finish_pass<T>(best, bi, psi, N, 1, n, N, d, s, sm);
}

// Point-major copy of FP32 orbitals for the streaming passes: pt[r][i] = psi[i][r] for i < n, zero for
// n <= i < ldt (ldt = n rounded up to a multiple of 4, so that every row starts on 16 bytes).
__global__ void scdm_transpose_kernel(const float *__restrict__ psi, int n, long long N, int ldt,
                                      float *__restrict__ pt) {
  __shared__ float tile[32][33];
  const long long r0 = (long long)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += 8) {
    const int i = i0 + y;
    const long long r = r0 + threadIdx.x;
    tile[y][threadIdx.x] = (i < n && r < N) ? psi[(long long)i * N + r] : 0.f;
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += 8) {
    const long long r = r0 + y;
    const int i = i0 + threadIdx.x;
    if (r < N && i < ldt) pt[r * ldt + i] = tile[threadIdx.x][y];
  }
}

__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, a.x * b.x)));
}

// The selection pass for FP32 orbitals in the point-major copy pt [N][ldt].  Every warp takes an
// equal share of the points, 32 at a time in four groups of 8: lane l loads the float4 of orbitals
// 4l..4l+3 (and 4l + 128 m) of the 8 points of a group, so that each warp load reads a whole orbital
// row of one point.  The lanes' partial sums are added over the lanes in FP32 by a pairwise tree (two
// all-reduce levels, then three butterfly levels that leave point l & 7 of the group on lane l), and
// lane l keeps point l of the 32.  Only the residual update itself is FP64 (this GPU's FP64 rate is a
// small fraction of its FP32 rate).
template <bool NORM>
__global__ void __launch_bounds__(kUpdNT, 3) scdm_pass_pt_kernel(const float *__restrict__ pt, int n, int ldt,
                                                                long long N, double *__restrict__ d, SelArgs s) {
  __shared__ __align__(16) ScdmSmem<float> sm;
  const int tid = threadIdx.x, lane = tid & 31;
  const int nf = ldt / 4;  // float4 per point row
  if (!NORM)
    for (int i = tid; i < ldt; i += kUpdNT)
      sm.us[i] = i < n ? static_cast<const float *>(s.Ub)[(long long)(s.k - 1) * ((n + 1) & ~1) + i] : 0.f;
  __syncthreads();
  const float4 *pt4 = reinterpret_cast<const float4 *>(pt);
  const float4 *u4 = reinterpret_cast<const float4 *>(sm.us);
  const long long nwarps = (long long)gridDim.x * (kUpdNT / 32);
  const long long wg = (long long)blockIdx.x * (kUpdNT / 32) + (tid >> 5);
  const long long ra = N * wg / nwarps, rb = N * (wg + 1) / nwarps;
  const unsigned full = 0xffffffffu;
  double best = -2.0;
  long long bi = N;
  for (long long r0 = ra; r0 < rb; r0 += 32) {  // same trip count for the whole warp
    const long long rme = r0 + lane;
    double dr = (!NORM && rme < rb) ? d[rme] : 0.0;  // the residual this lane updates, early
    float mine = 0.f;
#pragma unroll 1
    for (int grp = 0; grp < 4; ++grp) {
      const long long rg = r0 + 8 * grp;
      float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
      for (int f0 = 0; f0 < nf; f0 += 32) {
        const int f = f0 + lane;
        const bool fv = f < nf;
        const float4 uu = (NORM || !fv) ? make_float4(0.f, 0.f, 0.f, 0.f) : u4[f];
        float4 v[8];
        const float4 *base = pt4 + rg * nf + f;
        const int lim = fv ? (int)min(8LL, rb - rg) : 0;  // points of the group inside this warp's share
#pragma unroll
        for (int p = 0; p < 8; ++p)
          v[p] = p < lim ? __ldcs(base + p * nf) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int p = 0; p < 8; ++p) acc[p] += NORM ? dot4(v[p], v[p]) : dot4(uu, v[p]);
      }
#pragma unroll
      for (int p = 0; p < 8; ++p) {
        acc[p] += __shfl_xor_sync(full, acc[p], 16);
        acc[p] += __shfl_xor_sync(full, acc[p], 8);
      }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int j = 0; j < o; ++j) {
          const float send = up ? acc[j] : acc[j + o];
          const float keep = up ? acc[j + o] : acc[j];
          acc[j] = keep + __shfl_xor_sync(full, send, o);
        }
      }
      if ((lane >> 3) == grp) mine = acc[0];  // point rg + (lane & 7) = r0 + lane
    }
    if (rme < rb) {
      const double pm = (double)mine;
      if (NORM)
        dr = pm;
      else if (dr >= 0.0)
        dr = fmax(fma(-pm, pm, dr), 0.0);
      d[rme] = dr;
      amax(best, bi, dr, rme);
    }
  }
  finish_pass<float>(best, bi, pt, 1, ldt, n, N, d, s, sm);
}

// sum_l a[l sa] b[l sb] over l < n, in four interleaved partial sums (independent loads in flight)
__device__ __forceinline__ double strided_dot(const double *__restrict__ a, long long sa, const double *__restrict__ b,
                                              long long sb, int n) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int l = 0;
  for (; l + 4 <= n; l += 4) {
    s0 += a[l * sa] * b[l * sb];
    s1 += a[(l + 1) * sa] * b[(l + 1) * sb];
    s2 += a[(l + 2) * sa] * b[(l + 2) * sb];
    s3 += a[(l + 3) * sa] * b[(l + 3) * sb];
  }
  for (; l < n; ++l) s0 += a[l * sa] * b[l * sb];
  return (s0 + s1) + (s2 + s3);
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
  double s = strided_dot(M + i, n, M + j, n, n);
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

// Whether iteration `it` is skipped: an earlier one reached kNsStop, or stopped converging at the
// rounding level (below 1e-8 and not even a quarter of its predecessor, where quadratic convergence
// would have squared it).  Skipped iterations leave dev[it] = 0, so the later ones skip as well.
__device__ __forceinline__ bool ns_done(const double *__restrict__ dev, int it) {
  if (it == 0) return false;
  const double x = dev[it - 1];
  if (x < kNsStop) return true;
  return it >= 2 && x < 1e-8 && x > 0.25 * dev[it - 2];
}

// Iteration `it`: T = (3 I - Z Y) / 2 and dev[it] = max |T - I|, unless ns_done.
__global__ void ns_t_kernel(const double *__restrict__ Y, const double *__restrict__ Z, int n,
                            double *__restrict__ Tm, double *__restrict__ dev, int it) {
  if (ns_done(dev, it)) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double x = 0.0;
  if (e < n * n) {
    const int i = e / n, j = e % n;
    const double s = strided_dot(Z + (long long)i * n, 1, Y + j, n, n);
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
  const bool skip = ns_done(dev, it);
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
    s = strided_dot(Y + (long long)i * n, 1, Tm + j, n, n);
  else
    s = strided_dot(Tm + (long long)i * n, 1, Z + j, n, n);
  (isz ? Z2 : Y2)[f] = s;
}

// U = M Z / sqrt(f) (Z = (S/f)^{-1/2}) in FP64, and its transpose in the working type
template <typename T>
__global__ void scdm_factor_kernel(const double *__restrict__ M, const double *__restrict__ Z, int n,
                                   const double *__restrict__ f, double *__restrict__ U, T *__restrict__ Ut) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  const int i = e / n, j = e % n;
  double s = strided_dot(M + (long long)i * n, 1, Z + j, n, n);
  s /= sqrt(*f);
  U[e] = s;
  Ut[(long long)j * n + i] = (T)s;
}

struct Layout {
  size_t d, bval, bidx, Ub, M, S, Y0, Y1, Z0, Z1, Tm, U, Ut, f, dev, piv, dependent, count, pt, total;
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
  L.Ub = take(elem * (size_t)n * (n + 1));
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
  L.count = take(sizeof(unsigned int));
  // FP32 working type: the point-major copy [N][n rounded up to a multiple of 4]
  L.pt = take(elem == 4 ? sizeof(float) * (size_t)N * ((n + 3) & ~3) : 0);
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
  void *Ub = w + L.Ub;
  double *M = reinterpret_cast<double *>(w + L.M);
  double *S = reinterpret_cast<double *>(w + L.S);
  double *Y[2] = {reinterpret_cast<double *>(w + L.Y0), reinterpret_cast<double *>(w + L.Y1)};
  double *Z[2] = {reinterpret_cast<double *>(w + L.Z0), reinterpret_cast<double *>(w + L.Z1)};
  double *Tm = reinterpret_cast<double *>(w + L.Tm);
  double *f = reinterpret_cast<double *>(w + L.f);
  unsigned int *count = reinterpret_cast<unsigned int *>(w + L.count);
  res->piv = reinterpret_cast<int *>(w + L.piv);
  res->U = reinterpret_cast<double *>(w + L.U);
  res->Ut = w + L.Ut;
  res->dev = reinterpret_cast<double *>(w + L.dev);
  res->dependent = reinterpret_cast<int *>(w + L.dependent);
  cudaError_t e = cudaMemsetAsync(res->dev, 0, sizeof(double) * kNsMax, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(res->dependent, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  // column selection: n streaming passes over Psi; the last block of each pass takes the pivot step
  SelArgs sa{bval, bidx, count, Ub, res->piv, res->dependent, 0};
  // FP32: the passes stream the point-major copy (whole orbital rows of points per warp load)
  constexpr bool kPointMajor = sizeof(T) == 4;
  const int ldt = (n + 3) & ~3;
  float *pt = reinterpret_cast<float *>(w + L.pt);
  // one resident wave of persistent blocks
  int dev = 0, sms = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = kPointMajor ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scdm_pass_pt_kernel<false>, kUpdNT, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, scdm_pass_kernel<T, false>, kUpdNT, 0);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>((long long)std::max(per_sm, 1) * sms,
                                                                            std::min<long long>(kUpdBlocks,
                                                                                                (N + 255) / 256)));
  e = cudaMemsetAsync(count, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if constexpr (kPointMajor) {
    const dim3 tg((unsigned)((N + 31) / 32), (unsigned)((ldt + 31) / 32)), tb(32, 8);
    scdm_transpose_kernel<<<tg, tb, 0, st>>>(reinterpret_cast<const float *>(psi), n, N, ldt, pt);
    *launches += 1;
  }
  for (int k = 0; k < n; ++k) {
    sa.k = k;
    if constexpr (kPointMajor) {
      if (k == 0)
        scdm_pass_pt_kernel<true><<<grid, kUpdNT, 0, st>>>(pt, n, ldt, N, d, sa);
      else
        scdm_pass_pt_kernel<false><<<grid, kUpdNT, 0, st>>>(pt, n, ldt, N, d, sa);
    } else {
      if (k == 0)
        scdm_pass_kernel<T, true><<<grid, kUpdNT, 0, st>>>(psi, n, N, d, sa);
      else
        scdm_pass_kernel<T, false><<<grid, kUpdNT, 0, st>>>(psi, n, N, d, sa);
    }
  }
  *launches += n;
  // Loewdin factor.  The n x n FP64 products run as one output per thread in 64-thread blocks, so
  // that they spread over most SMs (FP64 throughput per SM is low).
  const int nn = n * n;
  constexpr int kSmallNT = 64;
  const unsigned g1 = (unsigned)((nn + kSmallNT - 1) / kSmallNT), g2 = (unsigned)((2 * nn + kSmallNT - 1) / kSmallNT);
  scdm_gather_kernel<T><<<g1, kSmallNT, 0, st>>>(psi, n, N, res->piv, M);
  gram_t_kernel<<<g1, kSmallNT, 0, st>>>(M, n, S);
  frob_kernel<<<1, kSelNT, 0, st>>>(S, n, f);
  ns_start_kernel<<<g1, kSmallNT, 0, st>>>(S, n, f, Y[0], Z[0]);
  *launches += 4;
  // Newton-Schulz in chunks of kNsChunk iterations; between chunks the host reads the last two
  // deviations and stops launching once the next iteration would be skipped
  int it = 0;
  while (it < kNsMax) {
    for (const int stop = std::min(kNsMax, it + kNsChunk); it < stop; ++it) {
      const int a = it & 1;
      ns_t_kernel<<<g1, kSmallNT, 0, st>>>(Y[a], Z[a], n, Tm, res->dev, it);
      ns_yz_kernel<<<g2, kSmallNT, 0, st>>>(Y[a], Z[a], Tm, n, Y[a ^ 1], Z[a ^ 1], res->dev, it);
      *launches += 2;
    }
    if (it >= kNsMax) break;
    double h[2];
    e = cudaMemcpyAsync(h, res->dev + it - 2, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (h[1] < kNsStop || (h[1] < 1e-8 && h[1] > 0.25 * h[0])) break;  // the test of ns_done
  }
  scdm_factor_kernel<T><<<g1, kSmallNT, 0, st>>>(M, Z[it & 1], n, f, res->U, reinterpret_cast<T *>(res->Ut));
  *launches += 1;
  return cudaGetLastError();
}

template cudaError_t launch_scdm<float>(const float *, int, long long, void *, cudaStream_t, long *, ScdmResult *);
template cudaError_t launch_scdm<double>(const double *, int, long long, void *, cudaStream_t, long *, ScdmResult *);

}  // namespace ace
