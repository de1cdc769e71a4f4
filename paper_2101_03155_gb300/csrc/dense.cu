// dense.cu -- CUDA-core dense steps of the ACE build and application.
//
//   gram:      G[i][j] = scale * sum_r f(X_i(r)) f(Y_j(r)),  f = |.| for the pair screen
//              (section II: int |phi_i phi_j| dr) or identity for M = -dV Phi^T W (App. A) and
//              C = dV xi^T psi.  Products and the sum inside one 4096-point chunk are in T; the
//              chunks are added into the FP64 result.
//   left_mul:  Z = A Y with A small (m x n) and Y (n x K): xi = L^-1 W (xi = W L^-T, App. A) and
//              the ACE application out = -C^T xi (section II).
//   cholesky:  M = (M_raw + M_raw^T)/2; -M = L L^T; L^-1; E_x = (f/2) tr M, all FP64 (App. A).
//   compact:   pair list of the screen (i <= j, sorted) and packs of two pairs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include <cstdint>
#include <cstdlib>

#include "ace_internal.h"
#include "f32x2.cuh"
#include "fft.cuh"

namespace ace {

// ----------------------------------------------------------------------------------------
// Gram: 64 x 64 output tile per CTA, 256 threads with 4 x 4 register tiles, K chunk per CTA.
// ----------------------------------------------------------------------------------------
constexpr int GR_BM = 64, GR_BK = 32, GR_CHUNK = 4096, GR_NT = 256;

// With `partial` non-null the CTA of chunk c writes its scaled tile sums to partial[c] (no
// atomics) and gram_chunks_reduce_kernel adds the chunks in a fixed order: the result is then
// the same bit for bit on every run.
template <typename T, bool ABS>
__global__ void __launch_bounds__(GR_NT) gram_kernel(const T *__restrict__ X, int nx, const T *__restrict__ Y, int ny,
                                                     long long K, double scale, bool upper_only, int nbx,
                                                     double *__restrict__ G, double *__restrict__ partial) {
  __shared__ T xs[GR_BK][GR_BM + 1];
  __shared__ T ys[GR_BK][GR_BM + 1];
  int bi, bj;
  if (upper_only) {
    // blockIdx.x enumerates tile pairs (bi <= bj) row by row
    int idx = blockIdx.x;
    bi = 0;
    while (idx >= nbx - bi) {
      idx -= nbx - bi;
      ++bi;
    }
    bj = bi + idx;
  } else {
    bi = blockIdx.x % nbx;
    bj = blockIdx.x / nbx;
  }
  const int i0 = bi * GR_BM, j0 = bj * GR_BM;
  const long long k0 = (long long)blockIdx.y * GR_CHUNK;
  const long long k1 = min(K, k0 + GR_CHUNK);
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  // acc + comp is a compensated (Kahan) running sum of the 32-point partial sums of each tile
  T acc[4][4], comp[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = comp[a][b] = (T)0;

  for (long long kk = k0; kk < k1; kk += GR_BK) {
    // load 64 rows x 32 k of X and of Y (coalesced along k)
    for (int e = tid; e < GR_BM * GR_BK; e += GR_NT) {
      const int r = e / GR_BK, c = e % GR_BK;
      const long long k = kk + c;
      T xv = (T)0, yv = (T)0;
      if (k < k1) {
        if (i0 + r < nx) xv = X[(long long)(i0 + r) * K + k];
        if (j0 + r < ny) yv = Y[(long long)(j0 + r) * K + k];
      }
      if (ABS) {
        xv = xv < (T)0 ? -xv : xv;
        yv = yv < (T)0 ? -yv : yv;
      }
      xs[c][r] = xv;
      ys[c][r] = yv;
    }
    __syncthreads();
    T part[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) part[a][b] = (T)0;
#pragma unroll 8
    for (int c = 0; c < GR_BK; ++c) {
      T xr[4], yr[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xr[a] = xs[c][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yr[b] = ys[c][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) part[a][b] += xr[a] * yr[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const T y = part[a][b] - comp[a][b];
        const T t = acc[a][b] + y;
        comp[a][b] = (t - acc[a][b]) - y;
        acc[a][b] = t;
      }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
      if (i < nx && j < ny) {
        if (partial)
          partial[((long long)blockIdx.y * nx + i) * ny + j] = scale * (double)acc[a][b];
        else
          atomicAdd(G + (long long)i * ny + j, scale * (double)acc[a][b]);
      }
    }
}

// G_ij = sum over the chunks of partial[c]_ij in chunk order (upper_only: j >= i only)
__global__ void gram_chunks_reduce_kernel(const double *__restrict__ partial, long long chunks, int nx, int ny,
                                          bool upper_only, double *__restrict__ G) {
  const long long ne = (long long)nx * ny;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= ne || (upper_only && e % ny < e / ny)) return;
  double s = 0.0;
  for (long long c = 0; c < chunks; ++c) s += partial[c * ne + e];
  G[e] = s;
}

size_t gram_chunks_bytes(int nx, int ny, long long K) {
  return sizeof(double) * (size_t)((K + GR_CHUNK - 1) / GR_CHUNK) * nx * ny;
}

// FP32 operands: 128 x 64 output tile, 256 threads with 8 x 4 outputs each, k-tiles of 16 staged
// in shared memory (double-buffered, next tile prefetched into registers), FP32 partial sums of 32
// points added into a Kahan-compensated FP32 accumulator, FP64 atomics across 4096-point chunks.
constexpr int G2_BM = 128, G2_BN = 64, G2_BK = 16, G2_NT = 256, G2_CHUNK = 4096;

template <bool ABS>
__global__ void __launch_bounds__(G2_NT, 2) gram_f32_kernel(const float *__restrict__ X, int nx,
                                                            const float *__restrict__ Y, int ny, long long K,
                                                            double scale, bool upper_only, int tiles_i,
                                                            double *__restrict__ G) {
  __shared__ __align__(16) float xs[2][G2_BK][G2_BM + 4];
  __shared__ __align__(16) float ys[2][G2_BK][G2_BN + 4];
  const int ti = blockIdx.x % tiles_i, tj = blockIdx.x / tiles_i;
  const int i0 = ti * G2_BM, j0 = tj * G2_BN;
  if (upper_only && j0 + G2_BN - 1 < i0) return;  // tile entirely below the diagonal
  const long long kb = (long long)blockIdx.y * G2_CHUNK;
  const long long ke = min(K, kb + G2_CHUNK);
  const int ntiles = (int)((ke - kb + G2_BK - 1) / G2_BK);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float acc[8][4], comp[8][4], part[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = comp[a][b] = part[a][b] = 0.f;

  float4 rx[2], ry;
  auto load = [&](int t) {
    const long long k0 = kb + (long long)t * G2_BK;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int f = tid + G2_NT * q, row = f >> 2, kq = (f & 3) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i0 + row < nx && k0 + kq < ke) v = __ldg(reinterpret_cast<const float4 *>(X + (long long)(i0 + row) * K + k0 + kq));
      rx[q] = v;
    }
    {
      const int row = tid >> 2, kq = (tid & 3) * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j0 + row < ny && k0 + kq < ke) v = __ldg(reinterpret_cast<const float4 *>(Y + (long long)(j0 + row) * K + k0 + kq));
      ry = v;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int f = tid + G2_NT * q, row = f >> 2, kq = (f & 3) * 4;
      const float v[4] = {rx[q].x, rx[q].y, rx[q].z, rx[q].w};
#pragma unroll
      for (int c = 0; c < 4; ++c) xs[buf][kq + c][row] = ABS ? fabsf(v[c]) : v[c];
    }
    const int row = tid >> 2, kq = (tid & 3) * 4;
    const float v[4] = {ry.x, ry.y, ry.z, ry.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) ys[buf][kq + c][row] = ABS ? fabsf(v[c]) : v[c];
  };
  if (ntiles > 0) {
    load(0);
    store(0);
  }
  __syncthreads();
  for (int t = 0; t < ntiles; ++t) {
    const int buf = t & 1;
    if (t + 1 < ntiles) load(t + 1);
#pragma unroll
    for (int k = 0; k < G2_BK; ++k) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&xs[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&xs[buf][k][64 + ty * 4]);
      const float4 b = *reinterpret_cast<const float4 *>(&ys[buf][k][tx * 4]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) part[r][c] = fmaf(av[r], bv[c], part[r][c]);
    }
    if ((t & 1) || t + 1 == ntiles) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float y = part[r][c] - comp[r][c];
          const float s = acc[r][c] + y;
          comp[r][c] = (s - acc[r][c]) - y;
          acc[r][c] = s;
          part[r][c] = 0.f;
        }
    }
    if (t + 1 < ntiles) store(buf ^ 1);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = i0 + (r < 4 ? ty * 4 + r : 64 + ty * 4 + (r - 4));
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (i < nx && j < ny && !(upper_only && j < i)) atomicAdd(G + (long long)i * ny + j, scale * (double)acc[r][c]);
    }
  }
}

// ----------------------------------------------------------------------------------------
// Symmetric FP32 Gram (the screen, X = Y, upper triangle): 64 x 64 tiles enumerated over the
// upper triangle of 64-row blocks only, 256 threads with 4 x 4 outputs each, k-step 16, chunks of
// ACE_GS_CHUNK points per CTA.  Products run as packed f32x2 FMAs: the row operand is stored twice in
// shared memory ((a, a) pairs) so that a pair of outputs (c, c + 1) takes one instruction.
// Within a chunk, 32-point FP32 partials are added with Kahan compensation; chunks meet in FP64
// atomics.
// ----------------------------------------------------------------------------------------
// points per CTA and CTAs per SM of the symmetric kernel (the register budget follows)
#ifndef ACE_GS_CHUNK
#define ACE_GS_CHUNK 2048
#endif
#ifndef ACE_GS_MINB
#define ACE_GS_MINB 2
#endif
constexpr int GS_B = 64, GS_BK = 16, GS_NT = 256, GS_CHUNK = ACE_GS_CHUNK;

template <bool ABS>
__global__ void __launch_bounds__(GS_NT, ACE_GS_MINB) gram_sym_f32_kernel(const float *__restrict__ X, int n, long long ld,
                                                                        long long K, double scale,
                                                                        double *__restrict__ G) {
  // (a, a) pairs of the row block and plain values of the column block, double-buffered
  __shared__ __align__(16) float2 xs[2][GS_BK][GS_B + 2];
  __shared__ __align__(16) float ys[2][GS_BK][GS_B + 4];
  // tile t of the upper triangle of nb x nb blocks: row-major over bi <= bj
  int bi = 0, t = blockIdx.x;
  {
    const int nb = (n + GS_B - 1) / GS_B;
    while (t >= nb - bi) {
      t -= nb - bi;
      ++bi;
    }
  }
  const int bj = bi + t;
  const int i0 = bi * GS_B, j0 = bj * GS_B;
  const long long kb = (long long)blockIdx.y * GS_CHUNK;
  const long long ke = min(K, kb + GS_CHUNK);
  const int ntiles = (int)((ke - kb + GS_BK - 1) / GS_BK);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  unsigned long long acc[4][2], comp[4][2], part[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = comp[a][b] = part[a][b] = 0ull;

  // each thread stages one float4 (4 consecutive points) of one row of each block; the global
  // loads run two k-tiles ahead (register sets 0 and 1 alternate)
  const int lrow = tid >> 2, lk = (tid & 3) * 4;
  float4 rx[2], ry[2];
  auto load = [&](int tt, float4 &vx, float4 &vy) {
    const long long k0 = kb + (long long)tt * GS_BK + lk;
    vx = make_float4(0.f, 0.f, 0.f, 0.f);
    vy = vx;
    if (tt < ntiles && k0 < ke) {
      if (i0 + lrow < n) vx = __ldg(reinterpret_cast<const float4 *>(X + (long long)(i0 + lrow) * ld + k0));
      if (j0 + lrow < n) vy = __ldg(reinterpret_cast<const float4 *>(X + (long long)(j0 + lrow) * ld + k0));
    }
  };
  auto store = [&](int buf, const float4 &ux, const float4 &uy) {
    const float vx[4] = {ux.x, ux.y, ux.z, ux.w}, vy[4] = {uy.x, uy.y, uy.z, uy.w};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const float a = ABS ? fabsf(vx[c]) : vx[c];
      xs[buf][lk + c][lrow] = make_float2(a, a);
      ys[buf][lk + c][lrow] = ABS ? fabsf(vy[c]) : vy[c];
    }
  };
  auto compute = [&](int buf, int tt) {
#pragma unroll
    for (int k = 0; k < GS_BK; ++k) {
      const ulonglong2 a01 = *reinterpret_cast<const ulonglong2 *>(&xs[buf][k][ty * 4]);
      const ulonglong2 a23 = *reinterpret_cast<const ulonglong2 *>(&xs[buf][k][ty * 4 + 2]);
      const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&ys[buf][k][tx * 4]);
      const unsigned long long av[4] = {a01.x, a01.y, a23.x, a23.y};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        part[r][0] = f2fma(av[r], b.x, part[r][0]);
        part[r][1] = f2fma(av[r], b.y, part[r][1]);
      }
    }
    if ((tt & 1) || tt + 1 == ntiles) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const unsigned long long y = f2sub(part[r][c], comp[r][c]);
          const unsigned long long sm = f2add(acc[r][c], y);
          comp[r][c] = f2sub(f2sub(sm, acc[r][c]), y);
          acc[r][c] = sm;
          part[r][c] = 0ull;
        }
    }
  };
  load(0, rx[0], ry[0]);
  store(0, rx[0], ry[0]);
  load(1, rx[1], ry[1]);
  __syncthreads();
  // tile tt sits in shared buffer tt & 1; tile tt + 1 in register set (tt + 1) & 1
  for (int tt = 0; tt < ntiles; tt += 2) {
    load(tt + 2, rx[0], ry[0]);
    compute(0, tt);
    store(1, rx[1], ry[1]);
    __syncthreads();
    if (tt + 1 >= ntiles) break;
    load(tt + 3, rx[1], ry[1]);
    compute(1, tt + 1);
    store(0, rx[0], ry[0]);
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float2 v = f2up(acc[r][c]);
      const int j = j0 + tx * 4 + 2 * c;
      if (i < n && j < n && j >= i) atomicAdd(G + (long long)i * n + j, scale * (double)v.x);
      if (i < n && j + 1 < n && j + 1 >= i) atomicAdd(G + (long long)i * n + j + 1, scale * (double)v.y);
    }
  }
}

// Screen contribution of the columns [0, K) of X (rows of stride ld): G += scale * |X| |X|^T on the
// upper triangle (G is not cleared; columns must start on a 16-byte boundary, K % 4 == 0).
cudaError_t launch_screen_cols(const float *X, int n, long long ld, long long K, double scale, double *G,
                               cudaStream_t st) {
  if (K % 4 != 0 || ld % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15)) return cudaErrorInvalidValue;
  const int nb = (n + GS_B - 1) / GS_B;
  const long long chunks = (K + GS_CHUNK - 1) / GS_CHUNK;
  if (chunks > 65535) return cudaErrorInvalidValue;
  gram_sym_f32_kernel<true><<<dim3(nb * (nb + 1) / 2, (unsigned)chunks), GS_NT, 0, st>>>(X, n, ld, K, scale, G);
  return cudaGetLastError();
}

// Screen values within band * rho_cut of the threshold, recomputed from phi so that the pair
// decision does not rest on the tensor-core products (BF16x3: up to 3 * 2^-16 relative error per
// product): O_ij = dV sum_r |phi_i(r) phi_j(r)| with FP32 products summed per thread with Kahan
// compensation in FP32, then across the block's threads in FP64 in a fixed order.  Off-diagonal
// upper-triangle entries only (the diagonal is always kept).  One block per candidate pair.
constexpr int RF_NT = 256;
__global__ void __launch_bounds__(RF_NT) screen_refine_kernel(const float *__restrict__ phi, int n, long long N,
                                                              double dV, double rho_cut, double band,
                                                              double *__restrict__ O) {
  __shared__ double red[RF_NT / 32];
  const long long ne = (long long)n * n;
  for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
    const int i = (int)(e / n), j = (int)(e % n);
    if (i >= j) continue;
    const double o = O[e];  // the same value for every thread: the branch is uniform
    if (!(fabs(o - rho_cut) <= band * rho_cut)) continue;
    const float *a = phi + (long long)i * N, *b = phi + (long long)j * N;
    float sum = 0.f, comp = 0.f;
    for (long long r = threadIdx.x; r < N; r += RF_NT) {
      const float y = fabsf(a[r] * b[r]) - comp;
      const float t = sum + y;
      comp = (t - sum) - y;
      sum = t;
    }
    double v = (double)sum - (double)comp;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < RF_NT / 32; ++w) t += red[w];
      O[e] = dV * t;
    }
    __syncthreads();
  }
}

cudaError_t launch_screen_refine(const float *phi, int n, long long N, double dV, double rho_cut, double band,
                                 double *O, cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long ne = (long long)n * n;
  const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(ne, 2LL * sms));
  screen_refine_kernel<<<grid, RF_NT, 0, st>>>(phi, n, N, dV, rho_cut, band, O);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_gram(const T *X, int nx, const T *Y, int ny, long long K, double scale, bool abs_values,
                        bool upper_only, double *G, cudaStream_t st, double *partial) {
  if constexpr (sizeof(T) == 4) {
    if (K % 4 == 0 && X == Y && nx == ny && upper_only) {
      const int nb = (nx + GS_B - 1) / GS_B;
      const long long chunks = (K + GS_CHUNK - 1) / GS_CHUNK;
      if (chunks > 65535) return cudaErrorInvalidValue;
      cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)nx * ny, st);
      if (e != cudaSuccess) return e;
      dim3 grid(nb * (nb + 1) / 2, (unsigned)chunks);
      if (abs_values)
        gram_sym_f32_kernel<true><<<grid, GS_NT, 0, st>>>(X, nx, K, K, scale, G);
      else
        gram_sym_f32_kernel<false><<<grid, GS_NT, 0, st>>>(X, nx, K, K, scale, G);
      return cudaGetLastError();
    }
    if (K % 4 == 0) {
      const int tiles_i = (nx + G2_BM - 1) / G2_BM, tiles_j = (ny + G2_BN - 1) / G2_BN;
      const long long chunks = (K + G2_CHUNK - 1) / G2_CHUNK;
      if (chunks > 65535) return cudaErrorInvalidValue;
      cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)nx * ny, st);
      if (e != cudaSuccess) return e;
      dim3 grid(tiles_i * tiles_j, (unsigned)chunks);
      if (abs_values)
        gram_f32_kernel<true><<<grid, G2_NT, 0, st>>>(X, nx, Y, ny, K, scale, upper_only, tiles_i, G);
      else
        gram_f32_kernel<false><<<grid, G2_NT, 0, st>>>(X, nx, Y, ny, K, scale, upper_only, tiles_i, G);
      return cudaGetLastError();
    }
  }
  const int nbx = (nx + GR_BM - 1) / GR_BM, nby = (ny + GR_BM - 1) / GR_BM;
  const int tiles = upper_only ? nbx * (nbx + 1) / 2 : nbx * nby;
  const long long chunks = (K + GR_CHUNK - 1) / GR_CHUNK;
  if (chunks > 65535) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * (size_t)nx * ny, st);
  if (e != cudaSuccess) return e;
  dim3 grid(tiles, (unsigned)chunks);
  if (abs_values)
    gram_kernel<T, true><<<grid, GR_NT, 0, st>>>(X, nx, Y, ny, K, scale, upper_only, nbx, G, partial);
  else
    gram_kernel<T, false><<<grid, GR_NT, 0, st>>>(X, nx, Y, ny, K, scale, upper_only, nbx, G, partial);
  e = cudaGetLastError();
  if (e != cudaSuccess || !partial) return e;
  const long long ne = (long long)nx * ny;
  gram_chunks_reduce_kernel<<<(unsigned)((ne + 127) / 128), 128, 0, st>>>(partial, chunks, nx, ny, upper_only, G);
  return cudaGetLastError();
}
template cudaError_t launch_gram<float>(const float *, int, const float *, int, long long, double, bool, bool,
                                        double *, cudaStream_t, double *);
template cudaError_t launch_gram<double>(const double *, int, const double *, int, long long, double, bool, bool,
                                         double *, cudaStream_t, double *);

// ----------------------------------------------------------------------------------------
// Left multiply Z (m x K) = A (m x n) * Y (n x K); 64 x 64 tile, k-step 16, 4 x 4 per thread.
// ----------------------------------------------------------------------------------------
constexpr int LM_BM = 64, LM_BN = 64, LM_BK = 16, LM_NT = 256;

template <typename T>
__global__ void __launch_bounds__(LM_NT) left_mul_kernel(const T *__restrict__ A, int m, int n,
                                                         const T *__restrict__ Y, long long K, T *__restrict__ Z) {
  __shared__ T as[LM_BK][LM_BM + 1];
  __shared__ T ys[LM_BK][LM_BN];
  const int i0 = blockIdx.y * LM_BM;
  const long long c0 = (long long)blockIdx.x * LM_BN;
  const int tid = threadIdx.x, ty = tid / 16, tx = tid % 16;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
  for (int l0 = 0; l0 < n; l0 += LM_BK) {
    for (int e = tid; e < LM_BM * LM_BK; e += LM_NT) {
      const int r = e / LM_BK, c = e % LM_BK;
      as[c][r] = (i0 + r < m && l0 + c < n) ? A[(long long)(i0 + r) * n + l0 + c] : (T)0;
    }
    for (int e = tid; e < LM_BK * LM_BN; e += LM_NT) {
      const int r = e / LM_BN, c = e % LM_BN;
      ys[r][c] = (l0 + r < n && c0 + c < K) ? Y[(long long)(l0 + r) * K + c0 + c] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < LM_BK; ++c) {
      T ar[4], yr[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) ar[a] = as[c][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) yr[b] = ys[c][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += ar[a] * yr[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = i0 + ty + 16 * a;
      const long long c = c0 + tx + 16 * b;
      if (i < m && c < K) Z[(long long)i * K + c] = acc[a][b];
    }
}

template <typename T>
cudaError_t launch_left_mul(const T *A, int m, int n, const T *Y, long long K, T *Z, cudaStream_t st) {
  dim3 grid((unsigned)((K + LM_BN - 1) / LM_BN), (unsigned)((m + LM_BM - 1) / LM_BM));
  left_mul_kernel<T><<<grid, LM_NT, 0, st>>>(A, m, n, Y, K, Z);
  return cudaGetLastError();
}
template cudaError_t launch_left_mul<float>(const float *, int, int, const float *, long long, float *, cudaStream_t);
template cudaError_t launch_left_mul<double>(const double *, int, int, const double *, long long, double *,
                                             cudaStream_t);

// ----------------------------------------------------------------------------------------
// Cholesky of -M, L^-1 and E_x in one CTA (FP64).  A = -M lives in shared memory when n <= 128
// (n^2 doubles), else in a global workspace.  Right-looking factorisation, then the in-place
// inversion of the lower triangle column by column from the last (each column is a triangular
// matrix-vector product with the already inverted trailing block).
// status: 0 ok; 1000000 + j: pivot j of -M not positive; 2000000: non-finite entry in M.
// ----------------------------------------------------------------------------------------
constexpr int CH_NT = 1024;
constexpr int CH_SMEM_MAX_N = 128;

__global__ void __launch_bounds__(CH_NT) cholesky_kernel(const double *__restrict__ M_raw, int n, double spin_factor,
                                                         double *__restrict__ M, double *__restrict__ L,
                                                         double *__restrict__ Linv, double *__restrict__ energy,
                                                         int *__restrict__ status, double *__restrict__ gwork) {
  extern __shared__ double dyn[];
  __shared__ int bad;
  __shared__ double red[CH_NT / 32];
  const bool in_smem = n <= CH_SMEM_MAX_N;
  double *A = in_smem ? dyn : gwork;                       // n * n
  double *tmp = in_smem ? dyn + n * n : gwork + n * n;     // n
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int e = tid; e < n * n; e += CH_NT) {
    const int i = e / n, j = e % n;
    const double v = 0.5 * (M_raw[(long long)i * n + j] + M_raw[(long long)j * n + i]);
    M[e] = v;
    A[e] = -v;
    if (!isfinite(v)) bad = 2000000;
  }
  __syncthreads();
  double part = 0.0;
  for (int k = tid; k < n; k += CH_NT) part += M[(long long)k * n + k];
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < CH_NT / 32; ++w) s += red[w];
    *energy = 0.5 * spin_factor * s;
  }
  if (bad) {
    if (tid == 0) *status = bad;
    return;
  }
  // Right-looking factorisation of the lower triangle, two barriers per step:
  //   (a) column j scaled by 1/L_jj (and copied to col[] for conflict-free reads), L_jj stored;
  //   (b) trailing update A_ik -= L_ij L_kj over the triangle j < k <= i < n, flattened over all
  //       threads; the thread that finishes A_{j+1,j+1} (element 0) takes its square root and
  //       reciprocal for the next step, so no thread waits on a serial pivot computation.
  // The pivot test reads A_jj after the barrier, so every thread takes the same branch.
  double *col = tmp;                       // n: scaled column j
  double *rinv = tmp + n;                  // n: 1 / L_jj
  __shared__ double piv[2];                // sqrt and reciprocal of the next pivot
  if (tid == 0) {
    const double d0 = A[0];
    piv[0] = sqrt(d0);
    piv[1] = 1.0 / piv[0];
  }
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    const double d = A[j * n + j];
    if (!(d > 0.0) || !isfinite(d)) {
      if (tid == 0) *status = 1000000 + j;
      return;
    }
    const double r = piv[0], ri = piv[1];
    for (int i = j + 1 + tid; i < n; i += CH_NT) {
      const double v = A[i * n + j] * ri;
      A[i * n + j] = v;
      col[i] = v;
    }
    if (tid == 0) rinv[j] = ri;
    __syncthreads();
    if (tid == 0) A[j * n + j] = r;  // after the barrier: every thread has read the pivot d
    const int m = n - 1 - j;  // trailing rows j+1 .. n-1
    const int T = m * (m + 1) / 2;
    for (int e = tid; e < T; e += CH_NT) {
      // row q of the trailing triangle starts at q (q + 1) / 2
      int q = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
      while (q * (q + 1) / 2 > e) --q;
      while ((q + 1) * (q + 2) / 2 <= e) ++q;
      const int i = j + 1 + q, k = j + 1 + (e - q * (q + 1) / 2);
      const double v = A[i * n + k] - col[i] * col[k];
      A[i * n + k] = v;
      if (e == 0 && v > 0.0 && isfinite(v)) {  // i == k == j + 1: the next pivot
        piv[0] = sqrt(v);
        piv[1] = 1.0 / piv[0];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += CH_NT) {
    const int i = e / n, j = e % n;
    L[e] = (j <= i) ? A[e] : 0.0;
  }
  // Inverse: L = U D with U = L D^-1 unit lower (U_ik = L_ik / L_kk) and D = diag(L), so
  // L^-1 = D^-1 Y with Y = U^-1.  Y by right-looking forward substitution from Y = I:
  //   step k: Y_ic -= U_ik Y_kc  for i > k, c <= k   (Y_kk = 1; Y_kc final after step k - 1).
  // Y_ic (c < i) lives in the unused upper triangle at A[c][i]; column k of U is staged in a
  // double buffer during the previous step, so one barrier per step suffices.
  double *ucol = tmp + 2 * n;              // 2 n: columns k (even / odd) of U
  for (int i = 1 + tid; i < n; i += CH_NT) ucol[i] = A[i * n] * rinv[0];
  for (int e = tid; e < n * n; e += CH_NT) {
    const int i = e / n, c = e % n;
    if (c > i) A[e] = 0.0;                 // Y starts at the identity (unit diagonal implicit)
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const double *u = ucol + (k & 1) * n;
    double *unext = ucol + ((k + 1) & 1) * n;
    if (k + 1 < n)
      for (int i = k + 2 + tid; i < n; i += CH_NT) unext[i] = A[i * n + k + 1] * rinv[k + 1];
    // rectangle i in (k, n), c in [0, k]: lanes along i (contiguous in the upper triangle)
    const int rows = n - 1 - k, cols = k + 1;
    for (int e = tid; e < rows * cols; e += CH_NT) {
      const int c = e / rows, i = k + 1 + (e - c * rows);
      const double ykc = (c == k) ? 1.0 : A[c * n + k];
      A[c * n + i] -= u[i] * ykc;
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += CH_NT) {
    const int i = e / n, c = e % n;
    Linv[e] = (c < i) ? A[c * n + i] * rinv[i] : (c == i ? rinv[i] : 0.0);
  }
  if (tid == 0) *status = 0;
}

// ----------------------------------------------------------------------------------------
// The same factorisation on a cluster of CHC_C CTAs, for n <= CHC_MAX_N.  This GPU retires about
// two FP64 FMA per clock per SM, so the one-CTA kernel above is bound by one SM's FP64 pipe; here
// the work is spread over CHC_C SMs.
//   - Every CTA holds the whole symmetrised -M in shared memory (row stride lda = n | 1, odd, so
//     that a column walk does not hit one bank).  Each CTA symmetrises an eighth of the elements
//     and writes them into every CTA's copy (distributed shared memory) and into M.
//   - Columns are dealt in panels of CHC_B, panel p owned by CTA p % CHC_C.  After panel p is
//     published (a cluster barrier), every other CTA copies it from the owner's shared memory and
//     applies its rank-CHC_B update to the columns it owns.
//   - Look-ahead: the owner of panel p + 1 first updates only that panel's columns, factors it with
//     four warps (the panel in registers, one row group per warp and SM sub-partition, r and L_kj
//     published by warp 0 through shared memory) and arrives at the cluster barrier; its other
//     columns are updated after the arrival.
//     Every other CTA arrives right after its copy and updates its columns before it waits, so the
//     chain from one panel to the next is a copy, an 8-column update and the panel factorisation.
//   - Afterwards every CTA holds all of L; the columns of L^-1 are dealt in pairs, two per warp,
//     in an order that balances the FP64 work over the CTAs.  A warp holds its two columns in
//     registers (lane l: rows l, l + 32, l + 64, l + 96) and runs forward substitution: at step k
//     X_kc (final) is broadcast by a shuffle, the rows i > k take X_ic -= L_ik X_kc (only the row
//     groups below k), and row k + 1, then final, is scaled by 1 / L_(k+1)(k+1).
//   - A non-positive or non-finite pivot is written into every CTA's flag before the barrier, so all
//     CTAs leave the panel loop at the same point; the outputs then carry the same status codes as
//     above.
// Every element's arithmetic is fixed by the algorithm, not by the schedule: the panel updates of an
// element are applied in panel order (each a sum over the panel's columns in order, then one
// subtraction), and the substitution takes the steps k in order, so the result repeats bit for bit.
// All waits are hardware barriers (CTA and cluster); no CTA reads another's shared memory after the
// cluster barrier that follows the last panel.
// ----------------------------------------------------------------------------------------
namespace cg = cooperative_groups;
constexpr int CHC_NT = 256;
constexpr int CHC_C = 8;
constexpr int CHC_B = 8;
constexpr int CHC_MAX_N = 128;
constexpr int CHC_OWN = 16;  // columns a CTA owns at most: 128 / (8 x 8) panels of 8
static_assert(CHC_MAX_N <= CHC_C * CHC_B * (CHC_OWN / CHC_B), "own columns per CTA");
static_assert(CHC_MAX_N <= 2 * CHC_C * (CHC_NT / 32), "two columns of L^-1 per warp");
static_assert(CHC_MAX_N <= 128, "four rows per lane, four row groups in the panel factorisation");
static_assert(CHC_NT >= 128, "four warps factor a panel");

__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ bool finite_bits(double v) {
  return ((__double_as_longlong(v) >> 52) & 0x7ff) != 0x7ff;
}

// Panel (columns c0 .. c0 + w - 1, rows c0 .. n - 1, stored at columns s0 .. s0 + w - 1 of A) factored
// right-looking by the CTA's first NW warps, spread over the SM sub-partitions: an FP64 warp
// instruction issues once per about 64 cycles on a sub-partition, so one warp holding all rows would
// serialise several times the instructions.  Warp m holds rows c0 + lane + 32 m in registers.  For column j, warp 0 takes the pivot d (lane j),
// r = 1 / sqrt(d), scales its rows, and publishes r and the panel rows' scaled L_kj (k < CHC_B)
// through xch (double-buffered by column parity, so one named barrier per column suffices); then
// every warp scales its rows and updates the panel's later columns.  The arithmetic of every
// element is that of a one-warp right-looking factorisation.  Returns 0, or 1000000 + the column of
// a non-positive or non-finite pivot (the same in all NW warps).  Call with threads 0 .. 32 NW - 1;
// the panel must have at most 32 NW rows.
template <int NW>
__device__ __forceinline__ int chc_factor_panel(double *A, int lda, int n, int c0, int s0, int w, double *xch,
                                                int *xflag) {
  const int lane = threadIdx.x & 31, wm = threadIdx.x >> 5, h = n - c0, i = lane + 32 * wm;
  double a[CHC_B];
#pragma unroll
  for (int j = 0; j < CHC_B; ++j) a[j] = (i < h && j < w) ? A[(c0 + i) * lda + s0 + j] : 0.0;
  int status = 0;
#pragma unroll
  for (int j = 0; j < CHC_B; ++j) {
    if (j < w && status == 0) {
      double *buf = xch + (j & 1) * (CHC_B + 1);  // [k]: scaled L_(c0+k)(c0+j), [CHC_B]: r
      if (wm == 0) {
        const double d = __shfl_sync(0xffffffffu, a[j], j);  // row c0 + j: lane j of warp 0
        const long long bits = __double_as_longlong(d);
        const bool ok = bits > 0 && ((bits >> 52) & 0x7ff) != 0x7ff;  // d > 0 and finite
        double r = 0.0;
        if (ok) {
          r = rsqrt(d);
          if (lane > j) a[j] *= r;
          else if (lane == j) a[j] = d * r;
        }
        if (lane < CHC_B) buf[lane] = a[j];
        if (lane == 0) {
          buf[CHC_B] = r;
          xflag[j & 1] = ok ? 0 : 1000000 + c0 + j;
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * NW) : "memory");
      status = xflag[j & 1];
      if (status == 0) {
        if (wm > 0) a[j] *= buf[CHC_B];  // rows c0 + 32 and below, all past the pivot
#pragma unroll
        for (int k = j + 1; k < CHC_B; ++k) {
          if (k < w) {
            const double lkj = buf[k];
            if (wm > 0 || lane >= k) a[k] -= a[j] * lkj;
          }
        }
      }
    }
  }
  if (i < h) {
#pragma unroll
    for (int j = 0; j < CHC_B; ++j)
      if (j < w) A[(c0 + i) * lda + s0 + j] = a[j];
  }
  return status;
}

__global__ void __cluster_dims__(CHC_C, 1, 1) __launch_bounds__(CHC_NT)
    cholesky_cluster_kernel(const double *__restrict__ M_raw, int n, double spin_factor, double *__restrict__ M,
                            double *__restrict__ L, double *__restrict__ Linv, double *__restrict__ energy,
                            int *__restrict__ status) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double dyn[];
  __shared__ int bad;   // non-finite input: written into every CTA before the first barrier
  __shared__ int pf;    // pivot failure met by this CTA while it factors a panel
  __shared__ int fail;  // pivot failure of a panel's owner, written into every CTA before the
                        // cluster barrier and read only after it
  __shared__ int own[CHC_OWN];  // the columns this CTA owns, ascending (-1: none)
  __shared__ double red[CHC_NT / 32];
  __shared__ double xch[2 * (CHC_B + 1)];  // panel factorisation: r and the scaled panel rows
  __shared__ int xflag[2];
  const int rank = (int)cluster.block_rank(), tid = threadIdx.x;
  const int lda = n | 1;
  double *A = dyn;                          // n x lda
  double *rinv = dyn + (size_t)n * lda;     // n: 1 / L_kk
  const int P = (n + CHC_B - 1) / CHC_B;
  if (tid == 0) {
    bad = 0;
    pf = 0;
    fail = 0;
    int m = 0;
    for (int p = rank; p < P; p += CHC_C)
      for (int c = p * CHC_B; c < min(n, (p + 1) * CHC_B); ++c) own[m++] = c;
    for (; m < CHC_OWN; ++m) own[m] = -1;
  }
  cluster.sync();  // every CTA has started and cleared its flags before any write across CTAs
  // -M symmetrised: this CTA's eighth of the elements, M_sym = (M_raw + M_raw^T) / 2 written to M
  // and its negative into every CTA's A
  {
    double *Aq[CHC_C];
#pragma unroll
    for (int q = 0; q < CHC_C; ++q) Aq[q] = cluster.map_shared_rank(A, q);
    constexpr int U = CHC_MAX_N * CHC_MAX_N / (CHC_NT * CHC_C);  // elements per thread at n = 128
    const int nn = n * n;
    double s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = (u * CHC_C + rank) * CHC_NT + tid;
      s[u] = 0.0;
      if (e < nn) {
        const int i = e / n, j = e - (e / n) * n;
        s[u] = i == j ? M_raw[e] : 0.5 * (M_raw[e] + M_raw[j * n + i]);
      }
    }
    bool ok = true;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = (u * CHC_C + rank) * CHC_NT + tid;
      if (e < nn) {
        const int i = e / n, j = e - (e / n) * n;
        M[e] = s[u];
        ok = ok && finite_bits(s[u]);
        const double v = __longlong_as_double(__double_as_longlong(s[u]) ^ (long long)0x8000000000000000ull);
#pragma unroll
        for (int q = 0; q < CHC_C; ++q) Aq[q][i * lda + j] = v;
      }
    }
    if (!ok)
      for (int q = 0; q < CHC_C; ++q) *cluster.map_shared_rank(&bad, q) = 2000000;  // every CTA sees it
  }
  if (rank == 0) {
    double part = 0.0;
    for (int k = tid; k < n; k += CHC_NT) part += M_raw[k * n + k];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < CHC_NT / 32; ++w) t += red[w];
      *energy = 0.5 * spin_factor * t;
    }
  }
  cluster.sync();  // A complete in every CTA, bad the same everywhere
  // panel 0 by its owner
  if (!bad && rank == 0) {
    if (tid < 128) {
      const int r = chc_factor_panel<4>(A, lda, n, 0, 0, min(n, CHC_B), xch, xflag);
      if (tid == 0) pf = r;
    }
    __syncthreads();
    if (pf && tid < CHC_C) *cluster.map_shared_rank(&fail, tid) = pf;
  }
  cluster.sync();  // panel 0 final in its owner's shared memory (or the failure announced)
  const int lane16 = tid & 15, row16 = tid >> 4;  // (own column, row) lanes of the column-parallel update
  for (int p = 0; p < P; ++p) {
    if (bad || fail) break;  // the same in every CTA after the barrier
    const int c0 = p * CHC_B, c1 = min(n, c0 + CHC_B), w = c1 - c0, owner = p % CHC_C;
    if (rank != owner) {  // rows c0.. of the panel's columns from the owner, four loads in flight
      const double *src = cluster.map_shared_rank(A, owner);
      const int ne = (n - c0) * CHC_B;
      for (int base = tid; base < ne; base += 4 * CHC_NT) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = base + u * CHC_NT, c = e & (CHC_B - 1);
          v[u] = (e < ne && c < w) ? src[(c0 + (e >> 3)) * lda + c0 + c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = base + u * CHC_NT, c = e & (CHC_B - 1);
          if (e < ne && c < w) A[(c0 + (e >> 3)) * lda + c0 + c] = v[u];
        }
      }
    }
    __syncthreads();  // the panel, and the previous panel's updates of this CTA's columns, complete
    const bool ahead = p + 1 < P && rank == (p + 1) % CHC_C;
    const int c2 = min(n, c1 + CHC_B);
    if (ahead) {
      // rank-w update of the next panel's columns k in [c1, c2), rows i >= k, then its factorisation
      const int col = tid & (CHC_B - 1), rl = tid >> 3, k = c1 + col;
      if (k < c2)
        for (int i = c1 + rl; i < n; i += CHC_NT / CHC_B) {
          if (i < k) continue;
          double acc = 0.0;
          for (int j = c0; j < c1; ++j) acc += A[i * lda + j] * A[k * lda + j];
          A[i * lda + k] -= acc;
        }
      __syncthreads();
      if (tid < 128) {
        const int r = chc_factor_panel<4>(A, lda, n, c1, c1, c2 - c1, xch, xflag);
        if (tid == 0) pf = r;
      }
      __syncthreads();
      if (pf && tid < CHC_C) *cluster.map_shared_rank(&fail, tid) = pf;
    }
    cluster_arrive_release();  // the next panel is published once every CTA has arrived
    // rank-w update of this CTA's other columns k >= c1 (k >= c2 for the look-ahead owner), rows i >= k
    {
      const int k = own[lane16];
      if (k >= (ahead ? c2 : c1))
        for (int i = k + row16; i < n; i += CHC_NT / 16) {
          double acc = 0.0;
          for (int j = c0; j < c1; ++j) acc += A[i * lda + j] * A[k * lda + j];
          A[i * lda + k] -= acc;
        }
    }
    cluster_wait_acquire();
  }
  cluster.sync();  // no CTA reads another's shared memory past this point
  if (bad || fail) {
    if (rank == 0 && tid == 0) *status = bad ? bad : fail;
    return;
  }
  for (int e = tid; e < n * CHC_OWN; e += CHC_NT) {
    const int i = e / CHC_OWN, cc = e % CHC_OWN, c = own[cc];
    if (c < 0) continue;
    L[(long long)i * n + c] = (i >= c) ? A[i * lda + c] : 0.0;
  }
  for (int k = tid; k < n; k += CHC_NT) rinv[k] = 1.0 / A[k * lda + k];
  __syncthreads();
  {
    const int lane = tid & 31, wp = tid >> 5;
    // column pairs (2t, 2t + 1), dealt so that every CTA gets early and late columns alike
    const int t = CHC_C * wp + ((wp & 1) ? CHC_C - 1 - rank : rank);
    const int ca = 2 * t < n ? 2 * t : -1, cb = 2 * t + 1 < n ? 2 * t + 1 : -1;
    double xa[4], xb[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = lane + 32 * m;
      xa[m] = (ca >= 0 && i == ca) ? rinv[ca] : 0.0;
      xb[m] = (cb >= 0 && i == cb) ? rinv[cb] : 0.0;
    }
    if (ca >= 0) {
#pragma unroll
      for (int kb = 0; kb < 4; ++kb) {
        // steps k in this row group; the last step, n - 2, makes row n - 1 final
        const int kbeg = max(ca, 32 * kb), kend = min(n - 1, 32 * kb + 32);
        for (int k = kbeg; k < kend; ++k) {
          const int lk = k & 31;
          const double xka = __shfl_sync(0xffffffffu, xa[kb], lk), xkb = __shfl_sync(0xffffffffu, xb[kb], lk);
          const bool ub = cb >= 0 && k >= cb;
#pragma unroll
          for (int m = kb; m < 4; ++m) {
            const int i = lane + 32 * m;
            if (i > k && i < n) {
              const double lik = A[i * lda + k];
              xa[m] -= lik * xka;
              if (ub) xb[m] -= lik * xkb;
            }
          }
          // row k + 1 is final: lane (k + 1) & 31 of row group kb, or lane 0 of group kb + 1
          if (lk != 31) {
            if (lane == lk + 1) {
              const double s = rinv[k + 1];
              xa[kb] *= s;
              if (ub) xb[kb] *= s;
            }
          } else if (kb < 3) {
            if (lane == 0) {
              const double s = rinv[k + 1];
              xa[kb + 1] *= s;
              if (ub) xb[kb + 1] *= s;
            }
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int i = lane + 32 * m;
      if (i < n) {
        if (ca >= 0) Linv[(long long)i * n + ca] = i >= ca ? xa[m] : 0.0;
        if (cb >= 0) Linv[(long long)i * n + cb] = i >= cb ? xb[m] : 0.0;
      }
    }
  }
  if (rank == 0 && tid == 0) *status = 0;
}

// ----------------------------------------------------------------------------------------
// The factorisation for CHC_MAX_N < n <= CHW_MAX_N on a cluster of CHC_C CTAs whose shared memory
// holds only their own columns: all of -M does not fit one SM at these sizes.
//   - Panel p (8 columns) is owned by CTA p % CHC_C, which keeps its panels' columns, all rows,
//     in `own` (local column 8 (p / CHC_C) + j, odd row stride).  Each CTA symmetrises its own
//     columns straight from M_raw and writes them to M.
//   - The panel loop is that of the kernel above: after panel p is published, every CTA copies it
//     (rows c0..n-1) from its owner into its panel buffer p & 1; the owner of panel p + 1 updates that
//     panel's columns, factors it (eight warps, one row group each) and arrives at the cluster
//     barrier; every CTA updates its other columns before it waits.
//   - Afterwards each CTA writes its columns of L, and of L^T into the workspace (row c of L^T is
//     column c of L); after a cluster barrier, the columns of L^-1 are dealt in groups of four, one
//     group per warp, in an order that balances the FP64 work over the CTAs.  Forward substitution
//     holds a warp's four columns in registers (lane l: rows l + 32 m) and reads column k of L from
//     shared memory, where 32 rows of L^T at a time are staged (in the space of `own`).
// Status codes as above.
// ----------------------------------------------------------------------------------------
constexpr int CHW_MAX_N = 256;
constexpr int CHW_LDO = 33;  // own-column block: up to 32 columns per CTA, odd row stride
constexpr int CHW_LDP = 9;   // panel buffer row stride
static_assert(CHW_MAX_N <= CHC_C * CHC_B * 4, "four panels per CTA at most");
static_assert(CHW_MAX_N <= 4 * CHC_C * (CHC_NT / 32), "four columns of L^-1 per warp");
static_assert(CHW_MAX_N <= 32 * (CHC_NT / 32), "one row group per warp in the panel factorisation");
static_assert(32 * CHW_MAX_N <= CHW_MAX_N * CHW_LDO, "a 32-row slab of L^T fits in the own-column block");

__global__ void __cluster_dims__(CHC_C, 1, 1) __launch_bounds__(CHC_NT)
    cholesky_cluster_wide_kernel(const double *__restrict__ M_raw, int n, double spin_factor, double *__restrict__ M,
                                 double *__restrict__ L, double *__restrict__ Linv, double *__restrict__ energy,
                                 int *__restrict__ status, double *__restrict__ Lt) {
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ double dyn[];
  __shared__ int bad, pf, fail;
  __shared__ double red[CHC_NT / 32];
  __shared__ double xch[2 * (CHC_B + 1)];
  __shared__ int xflag[2];
  const int rank = (int)cluster.block_rank(), tid = threadIdx.x;
  double *own = dyn;                              // n x CHW_LDO
  // two n x CHW_LDP panel buffers, panel p in buffer p & 1: after arriving at the barrier a thread
  // still reads panel p while a faster one, past the wait, may already copy panel p + 1
  double *pbuf = own + (size_t)n * CHW_LDO;
  double *rinv = pbuf + 2 * (size_t)n * CHW_LDP;  // n
  const int P = (n + CHC_B - 1) / CHC_B;
  if (tid == 0) {
    bad = 0;
    pf = 0;
    fail = 0;
  }
  cluster.sync();  // every CTA has started and cleared its flags before any write across CTAs
  // own columns of -M_sym (all rows), M_sym written to M: local column lc = 8 t + j holds column
  // c = 8 (rank + CHC_C t) + j
  {
    bool ok = true;
    for (int e = tid; e < n * 32; e += CHC_NT) {
      const int i = e >> 5, lc = e & 31, c = CHC_B * (rank + CHC_C * (lc >> 3)) + (lc & 7);
      if (c >= n) continue;
      const double v = i == c ? M_raw[(long long)c * n + c]
                              : 0.5 * (M_raw[(long long)i * n + c] + M_raw[(long long)c * n + i]);
      M[(long long)i * n + c] = v;
      ok = ok && finite_bits(v);
      own[i * CHW_LDO + lc] = __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
    }
    if (!ok)
      for (int q = 0; q < CHC_C; ++q) *cluster.map_shared_rank(&bad, q) = 2000000;
  }
  if (rank == 0) {
    double part = 0.0;
    for (int k = tid; k < n; k += CHC_NT) part += M_raw[(long long)k * n + k];
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < CHC_NT / 32; ++w) t += red[w];
      *energy = 0.5 * spin_factor * t;
    }
  }
  cluster.sync();  // own columns complete, bad the same everywhere
  if (!bad && rank == 0) {
    const int r = chc_factor_panel<CHC_NT / 32>(own, CHW_LDO, n, 0, 0, min(n, CHC_B), xch, xflag);
    if (tid == 0) pf = r;
    __syncthreads();
    if (pf && tid < CHC_C) *cluster.map_shared_rank(&fail, tid) = pf;
  }
  cluster.sync();  // panel 0 final in its owner's shared memory (or the failure announced)
  for (int p = 0; p < P; ++p) {
    if (bad || fail) break;  // the same in every CTA after the barrier
    const int c0 = p * CHC_B, c1 = min(n, c0 + CHC_B), w = c1 - c0, owner = p % CHC_C;
    const int s_p = CHC_B * (p / CHC_C);  // the panel's columns in its owner's block
    double *pb = pbuf + (size_t)(p & 1) * n * CHW_LDP;
    {
      // rows c0.. of the panel into the panel buffer (from the owner's block; the owner's own copy
      // is local), four loads in flight
      const double *src = rank == owner ? own : cluster.map_shared_rank(own, owner);
      const int ne = (n - c0) * CHC_B;
      for (int base = tid; base < ne; base += 4 * CHC_NT) {
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = base + u * CHC_NT, c = e & (CHC_B - 1);
          v[u] = (e < ne && c < w) ? src[(c0 + (e >> 3)) * CHW_LDO + s_p + c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = base + u * CHC_NT, c = e & (CHC_B - 1);
          if (e < ne && c < w) pb[(c0 + (e >> 3)) * CHW_LDP + c] = v[u];
        }
      }
    }
    __syncthreads();  // the panel copied, and the previous panel's updates of this CTA's columns done
    const bool ahead = p + 1 < P && rank == (p + 1) % CHC_C;
    const int c2 = min(n, c1 + CHC_B);
    if (ahead) {
      const int s_n = CHC_B * ((p + 1) / CHC_C);
      const int col = tid & (CHC_B - 1), rl = tid >> 3, k = c1 + col;
      if (k < c2)
        for (int i = c1 + rl; i < n; i += CHC_NT / CHC_B) {
          if (i < k) continue;
          double acc = 0.0;
          for (int j = 0; j < w; ++j) acc += pb[i * CHW_LDP + j] * pb[k * CHW_LDP + j];
          own[i * CHW_LDO + s_n + col] -= acc;
        }
      __syncthreads();
      const int r = chc_factor_panel<CHC_NT / 32>(own, CHW_LDO, n, c1, s_n, c2 - c1, xch, xflag);
      if (tid == 0) pf = r;
      __syncthreads();
      if (pf && tid < CHC_C) *cluster.map_shared_rank(&fail, tid) = pf;
    }
    cluster_arrive_release();  // the next panel is published once every CTA has arrived
    {
      // rank-w update of this CTA's other columns k >= c1 (k >= c2 for the look-ahead owner), rows i >= k
      const int lc = tid & 31, rl = tid >> 5;
      const int k = CHC_B * (rank + CHC_C * (lc >> 3)) + (lc & 7);
      if (k < n && k >= (ahead ? c2 : c1))
        for (int i = k + rl; i < n; i += CHC_NT / 32) {
          double acc = 0.0;
          for (int j = 0; j < w; ++j) acc += pb[i * CHW_LDP + j] * pb[k * CHW_LDP + j];
          own[i * CHW_LDO + lc] -= acc;
        }
    }
    cluster_wait_acquire();
  }
  cluster.sync();  // no CTA reads another's shared memory past this point
  if (bad || fail) {
    if (rank == 0 && tid == 0) *status = bad ? bad : fail;
    return;
  }
  // this CTA's columns of L (row-major, zeros above the diagonal) and of L^T (row c = column c of L)
  for (int e = tid; e < n * 32; e += CHC_NT) {
    const int i = e >> 5, lc = e & 31, c = CHC_B * (rank + CHC_C * (lc >> 3)) + (lc & 7);
    if (c >= n) continue;
    const double v = own[i * CHW_LDO + lc];
    L[(long long)i * n + c] = i >= c ? v : 0.0;
    if (i >= c) Lt[(long long)c * n + i] = v;
  }
  __threadfence();
  cluster.sync();  // every column of L^T written
  for (int k = tid; k < n; k += CHC_NT) rinv[k] = 1.0 / __ldcg(Lt + (long long)k * n + k);
  {
    double *S = own;  // 32 rows of L^T at a time
    const int lane = tid & 31, wp = tid >> 5;
    const int t = CHC_C * wp + ((wp & 1) ? CHC_C - 1 - rank : rank);  // group of columns 4t .. 4t + 3
    int cq[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) cq[q] = 4 * t + q < n ? 4 * t + q : -1;
    __syncthreads();  // rinv complete
    double x[4][8];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int m = 0; m < 8; ++m) x[q][m] = (cq[q] >= 0 && lane + 32 * m == cq[q]) ? rinv[cq[q]] : 0.0;
#pragma unroll
    for (int kb = 0; kb < 8; ++kb) {
      const int k_lo = 32 * kb, k_hi = min(n, 32 * kb + 32);
      if (k_lo >= n) break;  // the same in every thread
      __syncthreads();      // the previous slab is no longer read
      for (int e = tid; e < (k_hi - k_lo) * n; e += CHC_NT) {
        const int kk = e / n, i = e - kk * n;
        S[e] = i > k_lo + kk ? __ldcg(Lt + (long long)(k_lo + kk) * n + i) : 0.0;
      }
      __syncthreads();
      if (cq[0] >= 0) {
        // steps k in this slab; the last step, n - 2, makes row n - 1 final
        for (int k = max(cq[0], k_lo); k < min(n - 1, k_hi); ++k) {
          const int lk = k & 31;
          double xk[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) xk[q] = __shfl_sync(0xffffffffu, x[q][kb], lk);
          const double *Sk = S + (k - k_lo) * n;
#pragma unroll
          for (int m = kb; m < 8; ++m) {
            const int i = lane + 32 * m;
            if (i > k && i < n) {
              const double lik = Sk[i];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (cq[q] >= 0 && k >= cq[q]) x[q][m] -= lik * xk[q];
            }
          }
          // row k + 1 is final: lane (k + 1) & 31 of row group kb, or lane 0 of group kb + 1
          if (lk != 31) {
            if (lane == lk + 1) {
              const double sc = rinv[k + 1];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (cq[q] >= 0 && k >= cq[q]) x[q][kb] *= sc;
            }
          } else if (kb < 7) {
            if (lane == 0) {
              const double sc = rinv[k + 1];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (cq[q] >= 0 && k >= cq[q]) x[q][kb + 1] *= sc;
            }
          }
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int i = lane + 32 * m;
      if (i < n) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (cq[q] >= 0) Linv[(long long)i * n + cq[q]] = i >= cq[q] ? x[q][m] : 0.0;
      }
    }
  }
  if (rank == 0 && tid == 0) *status = 0;
}

static bool cluster_cholesky_off() {
  static const bool off = [] {
    const char *v = std::getenv("ACE_CHOLESKY_ONE_CTA");
    return v && *v && *v != '0';
  }();
  return off;
}

// Once per device and kernel: the shared-memory limit for the largest n, and whether such a cluster
// fits (state[dev]: 0 unknown, 1 usable, -1 not).
template <typename K>
static bool cluster_ready(K kernel, size_t smax, int *state, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return false;
  if (state[dev] == 0) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax);
    int clusters = 0;
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(CHC_C);
      cfg.blockDim = dim3(CHC_NT);
      cfg.dynamicSmemBytes = smax;
      cfg.stream = st;
      e = cudaOccupancyMaxActiveClusters(&clusters, kernel, &cfg);
    }
    cudaGetLastError();
    state[dev] = (e == cudaSuccess && clusters > 0) ? 1 : -1;
  }
  return state[dev] == 1;
}

cudaError_t launch_cholesky(const double *M_raw, int n, double spin_factor, double *M, double *L, double *Linv,
                            double *energy, int *status, double *gwork, cudaStream_t st) {
  if (!cluster_cholesky_off() && n <= CHC_MAX_N) {
    static int state[64] = {};
    const size_t smax = sizeof(double) * ((size_t)CHC_MAX_N * (CHC_MAX_N | 1) + (size_t)CHC_MAX_N);
    if (cluster_ready(cholesky_cluster_kernel, smax, state, st)) {
      const size_t smem = sizeof(double) * ((size_t)n * (n | 1) + (size_t)n);
      cholesky_cluster_kernel<<<CHC_C, CHC_NT, smem, st>>>(M_raw, n, spin_factor, M, L, Linv, energy, status);
      return cudaGetLastError();
    }
  }
  if (!cluster_cholesky_off() && n > CHC_MAX_N && n <= CHW_MAX_N && gwork != nullptr) {
    // columns spread over the cluster; gwork (n x n doubles at least) holds L^T
    static int state[64] = {};
    const size_t smax = sizeof(double) * (size_t)CHW_MAX_N * (CHW_LDO + 2 * CHW_LDP + 1);
    if (cluster_ready(cholesky_cluster_wide_kernel, smax, state, st)) {
      const size_t smem = sizeof(double) * (size_t)n * (CHW_LDO + 2 * CHW_LDP + 1);
      cholesky_cluster_wide_kernel<<<CHC_C, CHC_NT, smem, st>>>(M_raw, n, spin_factor, M, L, Linv, energy, status,
                                                                 gwork);
      return cudaGetLastError();
    }
  }
  const size_t smem = n <= CH_SMEM_MAX_N ? sizeof(double) * ((size_t)n * n + 4 * n) : 0;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(cholesky_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (n > CH_SMEM_MAX_N && gwork == nullptr) return cudaErrorInvalidValue;
  cholesky_kernel<<<1, CH_NT, smem, st>>>(M_raw, n, spin_factor, M, L, Linv, energy, status, gwork);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Screen compaction (one CTA): keep (i <= j) iff i == j or rho_cut <= 0 or O_ij >= rho_cut,
// in lexicographic order; packs = consecutive pairs two at a time.  Also writes the symmetric O.
// ----------------------------------------------------------------------------------------
constexpr int CP_NT = 1024;

__global__ void __launch_bounds__(CP_NT) compact_kernel(const double *__restrict__ O, int n, double rho_cut,
                                                        int2 *__restrict__ pairs, int4 *__restrict__ packs,
                                                        int *__restrict__ count, double *__restrict__ O_sym) {
  __shared__ int warp_sums[CP_NT / 32];
  __shared__ int running;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) running = 0;
  for (int base = tid; base < n * n; base += 4 * CP_NT) {  // four loads in flight per thread
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = base + u * CP_NT, i = e / n, j = e % n;
      v[u] = e < n * n ? ((i <= j) ? O[e] : O[(long long)j * n + i]) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (base + u * CP_NT < n * n) O_sym[base + u * CP_NT] = v[u];
  }
  __syncthreads();
  const long long total = (long long)n * (n + 1) / 2;
  for (long long base = 0; base < total; base += CP_NT) {
    const long long e = base + tid;
    int keep = 0, i = 0, j = 0;
    if (e < total) {
      // row-major enumeration of the upper triangle: row i holds n - i entries
      // row i starts at s(i) = i (2n - i + 1) / 2; take the largest i with s(i) <= e (an FP32
      // estimate, made exact by the integer corrections below; FP64 is slow on this GPU)
      const float b = 2.0f * (float)n + 1.0f;
      i = (int)((b - sqrtf(fmaxf(b * b - 8.0f * (float)e, 0.0f))) * 0.5f);
      if (i < 0) i = 0;
      if (i > n - 1) i = n - 1;
      while (i > 0 && (long long)i * (2 * n - i + 1) / 2 > e) --i;
      while ((long long)(i + 1) * (2 * n - i) / 2 <= e) ++i;
      j = i + (int)(e - (long long)i * (2 * n - i + 1) / 2);
      const double o = O[(long long)i * n + j];
      keep = (i == j) || (rho_cut <= 0.0) || (o >= rho_cut);
    }
    const unsigned ballot = __ballot_sync(0xffffffffu, keep);
    const int prefix = __popc(ballot & ((1u << lane) - 1u));
    if (lane == 0) warp_sums[wid] = __popc(ballot);
    __syncthreads();
    int off = running;
    for (int w = 0; w < wid; ++w) off += warp_sums[w];
    if (keep) pairs[off + prefix] = make_int2(i, j);
    __syncthreads();
    if (tid == 0) {
      int s = 0;
      for (int w = 0; w < CP_NT / 32; ++w) s += warp_sums[w];
      running += s;
    }
    __syncthreads();
  }
  const int np = running;
  const int nk = (np + 1) / 2;
  for (int p = tid; p < nk; p += CP_NT) {
    const int2 a = pairs[2 * p];
    const int2 b = (2 * p + 1 < np) ? pairs[2 * p + 1] : make_int2(-1, -1);
    packs[p] = make_int4(a.x, a.y, b.x, b.y);
  }
  if (tid == 0) *count = np;
}

cudaError_t launch_screen_compact(const double *O, int n, double rho_cut, int2 *pairs, int4 *packs, int *count,
                                  double *O_sym, cudaStream_t st) {
  compact_kernel<<<1, CP_NT, 0, st>>>(O, n, rho_cut, pairs, packs, count, O_sym);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Queue assembly: the pack lists of several builds, concatenated in build order.  Every CTA forms
// the prefix of the pack counts (nb is small) and copies a grid-strided share of the packs.
// ----------------------------------------------------------------------------------------
constexpr int QA_NT = 256;

__global__ void __launch_bounds__(QA_NT) queue_assemble_kernel(const QueueSrc *__restrict__ src, int nb,
                                                               int4 *__restrict__ out, int *__restrict__ pack_build,
                                                               int *__restrict__ np_out) {
  __shared__ int off[kQueueMaxBuilds + 1];
  if (threadIdx.x == 0) {
    int o = 0;
    for (int b = 0; b < nb; ++b) {
      off[b] = o;
      o += (__ldcg(src[b].count) + 1) / 2;
    }
    off[nb] = o;
    if (blockIdx.x == 0) *np_out = o;
  }
  __syncthreads();
  const int total = off[nb];
  for (int q = blockIdx.x * QA_NT + threadIdx.x; q < total; q += gridDim.x * QA_NT) {
    int lo = 0, hi = nb - 1;  // the last build whose list starts at or before q (never an empty one)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= q)
        lo = mid;
      else
        hi = mid - 1;
    }
    out[q] = src[lo].packs[q - off[lo]];
    pack_build[q] = lo;
  }
}

// One CTA per (plane i1, orbital a): the plane's max |phi|, and the orbital's max by an atomic max
// on the bit pattern (non-negative floats order as their bits do).
constexpr int PM_NT = 256;
__global__ void __launch_bounds__(PM_NT) plane_max_kernel(const float *__restrict__ phi, int n1, long long npl,
                                                         float *__restrict__ pmax, float *__restrict__ gmax) {
  __shared__ float red[PM_NT / 32];
  const int i1 = blockIdx.x, a = blockIdx.y;
  const float *p = phi + ((long long)a * n1 + i1) * npl;
  float m = 0.f;
  if ((npl & 3) == 0 && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
    for (long long e = threadIdx.x; e < npl / 4; e += PM_NT) {
      const float4 v = __ldg(q + e);
      m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
  } else {
    for (long long e = threadIdx.x; e < npl; e += PM_NT) m = fmaxf(m, fabsf(__ldg(p + e)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < PM_NT / 32; ++w) m = fmaxf(m, red[w]);
    pmax[(long long)a * n1 + i1] = m;
    atomicMax(reinterpret_cast<int *>(gmax + a), __float_as_int(m));
  }
}

cudaError_t launch_plane_max(const float *phi, int norb, int n1, long long npl, float *pmax, float *gmax,
                             cudaStream_t st) {
  if (norb < 1 || norb > 65535) return cudaErrorInvalidValue;
  plane_max_kernel<<<dim3(n1, norb), PM_NT, 0, st>>>(phi, n1, npl, pmax, gmax);
  return cudaGetLastError();
}

__global__ void flag_fanout_kernel(const int *src, int *const *dst, int n) {
  if (__ldcg(src) == 0) return;
  for (int i = threadIdx.x; i < n; i += blockDim.x) *dst[i] = 1;
}

cudaError_t launch_flag_fanout(const int *src, int *const *dst, int n, cudaStream_t st) {
  flag_fanout_kernel<<<1, 128, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_queue_assemble(const QueueSrc *src, int nb, int4 *packs_out, int *pack_build, int *np_out,
                                  cudaStream_t st) {
  if (nb < 1 || nb > kQueueMaxBuilds) return cudaErrorInvalidValue;
  queue_assemble_kernel<<<2 * 152, QA_NT, 0, st>>>(src, nb, packs_out, pack_build, np_out);
  return cudaGetLastError();
}

// ----------------------------------------------------------------------------------------
// Elementwise precision conversion with scale.
// ----------------------------------------------------------------------------------------
template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, long long count, double scale) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (Tout)(scale * (double)in[i]);
}

template <typename Tin, typename Tout>
cudaError_t launch_convert(const Tin *in, Tout *out, long long count, double scale, cudaStream_t st) {
  const int nt = 256;
  const long long blocks = min((count + nt - 1) / nt, (long long)152 * 16);
  if (count == 0) return cudaSuccess;
  convert_kernel<Tin, Tout><<<(unsigned)blocks, nt, 0, st>>>(in, out, count, scale);
  return cudaGetLastError();
}
template cudaError_t launch_convert<double, float>(const double *, float *, long long, double, cudaStream_t);
template cudaError_t launch_convert<float, double>(const float *, double *, long long, double, cudaStream_t);
template cudaError_t launch_convert<double, double>(const double *, double *, long long, double, cudaStream_t);
template cudaError_t launch_convert<float, float>(const float *, float *, long long, double, cudaStream_t);

}  // namespace ace

namespace ace {
// A[c][k] = scale * C[k][c] (C is n x m FP64, A is m x n in T)
template <typename T>
__global__ void transpose_scale_kernel(const double *__restrict__ C, int n, int m, double scale, T *__restrict__ A) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * m; e += gridDim.x * blockDim.x) {
    const int c = e / n, k = e % n;
    A[e] = (T)(scale * C[(long long)k * m + c]);
  }
}
template <typename T>
cudaError_t launch_transpose_scale(const double *C, int n, int m, double scale, T *A, cudaStream_t st) {
  const int nt = 256;
  const int blocks = (int)min((long long)(n * m + nt - 1) / nt, 4096LL);
  transpose_scale_kernel<T><<<blocks > 0 ? blocks : 1, nt, 0, st>>>(C, n, m, scale, A);
  return cudaGetLastError();
}
template cudaError_t launch_transpose_scale<float>(const double *, int, int, double, float *, cudaStream_t);
template cudaError_t launch_transpose_scale<double>(const double *, int, int, double, double *, cudaStream_t);
}  // namespace ace
