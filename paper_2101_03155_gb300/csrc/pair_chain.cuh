// pair_chain.cuh -- the five pencil passes that turn packed orbital pairs into W contributions.
//
// For each pack (a,b),(c,d):  z = phi_a phi_b + i phi_c phi_d          (pair densities, Eq. vx)
//   z~ = FFT3(z);  z~ *= 4 pi / (N |G|^2)  (G = 0 dropped)               (Eq. e:vij in reciprocal space)
//   z = IFFT3(z~) = v_ab + i v_cd                                        (kernel real and even)
//   W_a += v_ab phi_b, W_b += v_ab phi_a, W_c += v_cd phi_d, W_d += v_cd phi_c   (Eq. vx; i = j once)
//
// The 3D transform is three sets of 1D pencils.  Each CTA owns TILE lines of one axis of one
// pack, stages them in shared memory (odd pitch), and runs a two-stage transform L = R1 * R2
// with both factors as register DFTs:
//   stage 1, task (t, n2): DFT_R1 over n1 of line[n1 R2 + n2], twiddle w_L^{n2 k1}, store at k1 R2 + n2
//   stage 2, task (t, k1): DFT_R2 over n2 of line[k1 R2 + n2]; X[k1 + R1 k2] stored at k1 R2 + k2
// so natural index k sits at pos(k) = (k % R1) R2 + k / R1; the copy-out undoes that.  The axis-1
// pass keeps stage-2 results in registers, multiplies by the kernel, and runs the inverse stages
// (inverse DFT_R2, conjugate twiddle, then inverse DFT_R1) which return natural order.
// Global accesses are coalesced: axis-3 tiles are TILE whole rows (contiguous), axis-1/2 tiles are
// TILE neighbouring columns, read and written as TILE-wide contiguous runs.
#pragma once

#include "ace_internal.h"
#include "fft.cuh"

// Every axis length 2^a 3^b 5^c up to 256, in four groups compiled in separate translation units
// (pair_chain_[abcd]_f{32,64}.cu); the axis-1 pass of the plane chain (conv) takes lengths up to 160.
#define ACE_LENGTHS_A(X) X(2) X(3) X(4) X(5) X(6) X(8) X(9) X(10) X(12) X(15) X(16) X(18) X(20) X(24) X(25) X(27) X(30) X(32) X(36)
#define ACE_LENGTHS_B(X) X(40) X(45) X(48) X(50) X(54) X(60) X(64) X(72) X(75) X(80) X(81) X(90) X(96) X(100)
#define ACE_LENGTHS_C(X) X(108) X(120) X(125) X(128) X(135) X(144) X(150) X(160) X(162) X(180)
#define ACE_LENGTHS_D(X) X(192) X(200) X(216) X(225) X(240) X(243) X(250) X(256)
#define ACE_CONV_LENGTHS_C(X) X(108) X(120) X(125) X(128) X(135) X(144) X(150) X(160)
#define ACE_PASS_LENGTHS(X) ACE_LENGTHS_A(X) ACE_LENGTHS_B(X) ACE_LENGTHS_C(X) ACE_LENGTHS_D(X)

namespace ace {

// Pencil tile: 16 lines of L points (odd pitch), or 8 where 16 would not fit in 48 KB of static
// shared memory (FP64 beyond about 190 points).
template <typename T, int L>
struct PassShape {
  static constexpr int R1 = Factor<L>::R1;
  static constexpr int R2 = Factor<L>::R2;
  static constexpr int TILE = (16LL * (L + 1) + L) * (long long)sizeof(cpx<T>) <= 48LL * 1024 ? 16 : 8;
  static constexpr int LP = L + 1;  // odd pitch: lanes over lines hit distinct banks
  static constexpr int NT = TILE * (R1 > R2 ? R1 : R2);
};

template <typename T>
__device__ __forceinline__ cpx<T> conjc(cpx<T> a) {
  return {a.x, -a.y};
}

// stage 1 of the two-stage transform in direction D (twiddled unless TWIDDLE is false)
template <typename T, int L, int D, bool TWIDDLE>
__device__ __forceinline__ void pencil_stage1(cpx<T> *s, const cpx<T> *tw, int tvalid) {
  using S = PassShape<T, L>;
  for (int task = threadIdx.x; task < S::TILE * S::R2; task += S::NT) {
    const int t = task % S::TILE, n2 = task / S::TILE;
    if (t >= tvalid) continue;
    cpx<T> *line = s + t * S::LP;
    cpx<T> x[S::R1];
#pragma unroll
    for (int n1 = 0; n1 < S::R1; ++n1) x[n1] = line[n1 * S::R2 + n2];
    Dft<S::R1, D, T>::run(x);
#pragma unroll
    for (int k1 = 0; k1 < S::R1; ++k1) {
      cpx<T> v = x[k1];
      if (TWIDDLE && k1 > 0) {
        const cpx<T> w = tw[n2 * k1];
        v = cmul(v, D < 0 ? w : conjc(w));
      }
      line[k1 * S::R2 + n2] = v;
    }
  }
}

template <typename T, int L, int D>
__device__ __forceinline__ void pencil_stage2(cpx<T> *s, int tvalid) {
  using S = PassShape<T, L>;
  for (int task = threadIdx.x; task < S::TILE * S::R1; task += S::NT) {
    const int t = task % S::TILE, k1 = task / S::TILE;
    if (t >= tvalid) continue;
    cpx<T> *line = s + t * S::LP + k1 * S::R2;
    cpx<T> x[S::R2];
#pragma unroll
    for (int n2 = 0; n2 < S::R2; ++n2) x[n2] = line[n2];
    Dft<S::R2, D, T>::run(x);
#pragma unroll
    for (int k2 = 0; k2 < S::R2; ++k2) line[k2] = x[k2];
  }
}

template <int L>
__device__ __forceinline__ int perm_pos(int k) {
  return (k % Factor<L>::R1) * Factor<L>::R2 + k / Factor<L>::R1;
}

template <typename T, int L, int MODE>
__global__ void __launch_bounds__((PassShape<T, L>::NT)) pair_pass_kernel(PairPassArgs<T> a) {
  using S = PassShape<T, L>;
  constexpr int TILE = S::TILE, LP = S::LP, NT = S::NT;
  __shared__ cpx<T> s[TILE * LP];
  __shared__ cpx<T> tw[L];

  const int tid = threadIdx.x;
  const int4 pk = a.packs[a.pack0 + blockIdx.y];
  cpx<T> *z = a.scratch + (long long)blockIdx.y * a.N;

  for (int e = tid; e < L; e += NT) tw[e] = a.tw[e];

  constexpr bool AXIS3 = (MODE == PASS_FWD3_PAIR || MODE == PASS_INV3_ACC);
  long long base, Ns;
  int tvalid;
  if (AXIS3) {
    const long long rows = (long long)a.n1 * a.n2;
    const long long row0 = (long long)blockIdx.x * TILE;
    tvalid = (int)min((long long)TILE, rows - row0);
    base = row0 * L;
    Ns = 1;
  } else if (MODE == PASS_CONV1) {
    const long long cols = (long long)a.n2 * a.n3;
    const long long c0 = (long long)blockIdx.x * TILE;
    tvalid = (int)min((long long)TILE, cols - c0);
    base = c0;
    Ns = cols;
  } else {  // axis 2
    const int tpi = (a.n3 + TILE - 1) / TILE;
    const int i1 = blockIdx.x / tpi;
    const int i30 = (blockIdx.x % tpi) * TILE;
    tvalid = min(TILE, a.n3 - i30);
    base = (long long)i1 * a.n2 * a.n3 + i30;
    Ns = a.n3;
  }

  // ---- copy in ----
  if (MODE == PASS_FWD3_PAIR) {
    const T *pa = a.phi + (long long)pk.x * a.N + base;
    const T *pb = a.phi + (long long)pk.y * a.N + base;
    const bool two = pk.z >= 0;
    const T *pc = a.phi + (long long)(two ? pk.z : 0) * a.N + base;
    const T *pd = a.phi + (long long)(two ? pk.w : 0) * a.N + base;
    for (int e = tid; e < tvalid * L; e += NT) {
      const int t = e / L, n = e - t * L;
      const T re = pa[e] * pb[e];
      const T im = two ? pc[e] * pd[e] : (T)0;
      s[t * LP + n] = cpx<T>{re, im};
    }
  } else if (AXIS3) {
    const cpx<T> *src = z + base;
    for (int e = tid; e < tvalid * L; e += NT) {
      const int t = e / L, n = e - t * L;
      s[t * LP + n] = src[e];
    }
  } else {
    const cpx<T> *src = z + base;
    for (int e = tid; e < TILE * L; e += NT) {
      const int n = e / TILE, t = e - n * TILE;
      if (t < tvalid) s[t * LP + n] = src[(long long)n * Ns + t];
    }
  }
  __syncthreads();

  // ---- transform ----
  if (MODE == PASS_CONV1) {
    pencil_stage1<T, L, -1, true>(s, tw, tvalid);
    __syncthreads();
    for (int task = tid; task < TILE * S::R1; task += NT) {
      const int t = task % TILE, k1 = task / TILE;
      if (t >= tvalid) continue;
      cpx<T> *line = s + t * LP + k1 * S::R2;
      cpx<T> x[S::R2];
#pragma unroll
      for (int n2 = 0; n2 < S::R2; ++n2) x[n2] = line[n2];
      Dft<S::R2, -1, T>::run(x);
      const T *kcol = a.kernel + base + t;
#pragma unroll
      for (int k2 = 0; k2 < S::R2; ++k2) {
        const T kv = kcol[(long long)(k1 + S::R1 * k2) * Ns];
        x[k2] = cscale(x[k2], kv);
      }
      Dft<S::R2, +1, T>::run(x);
#pragma unroll
      for (int n2 = 0; n2 < S::R2; ++n2) {
        cpx<T> v = x[n2];
        if (n2 > 0 && k1 > 0) v = cmul(v, conjc(tw[n2 * k1]));
        line[n2] = v;
      }
    }
    __syncthreads();
    pencil_stage1<T, L, +1, false>(s, tw, tvalid);  // inverse DFT_R1: natural order out
    __syncthreads();
  } else {
    constexpr int D = (MODE == PASS_INV2 || MODE == PASS_INV3_ACC) ? +1 : -1;
    pencil_stage1<T, L, D, true>(s, tw, tvalid);
    __syncthreads();
    pencil_stage2<T, L, D>(s, tvalid);
    __syncthreads();
  }

  // ---- copy out ----
  if (MODE == PASS_INV3_ACC) {
    const long long oa = (long long)pk.x * a.N + base, ob = (long long)pk.y * a.N + base;
    const bool two = pk.z >= 0;
    const long long oc = (long long)(two ? pk.z : 0) * a.N + base, od = (long long)(two ? pk.w : 0) * a.N + base;
    const bool diag1 = pk.x == pk.y, diag2 = pk.z == pk.w;
    for (int e = tid; e < tvalid * L; e += NT) {
      const int t = e / L, k = e - t * L;
      const cpx<T> v = s[t * LP + perm_pos<L>(k)];
      atomicAdd(a.W + oa + e, v.x * a.phi[ob + e]);
      if (!diag1) atomicAdd(a.W + ob + e, v.x * a.phi[oa + e]);
      if (two) {
        atomicAdd(a.W + oc + e, v.y * a.phi[od + e]);
        if (!diag2) atomicAdd(a.W + od + e, v.y * a.phi[oc + e]);
      }
    }
  } else if (MODE == PASS_FWD3_PAIR) {
    cpx<T> *dst = z + base;
    for (int e = tid; e < tvalid * L; e += NT) {
      const int t = e / L, k = e - t * L;
      dst[e] = s[t * LP + perm_pos<L>(k)];
    }
  } else if (MODE == PASS_CONV1) {
    cpx<T> *dst = z + base;
    for (int e = tid; e < TILE * L; e += NT) {
      const int k = e / TILE, t = e - k * TILE;
      if (t < tvalid) dst[(long long)k * Ns + t] = s[t * LP + k];
    }
  } else {
    cpx<T> *dst = z + base;
    for (int e = tid; e < TILE * L; e += NT) {
      const int k = e / TILE, t = e - k * TILE;
      if (t < tvalid) dst[(long long)k * Ns + t] = s[t * LP + perm_pos<L>(k)];
    }
  }
}

// ---------------------------------------------------------------------------------------
// Axis-1 pass of the plane chain: for 32 neighbouring (p2, p3) columns of one pack, forward
// transform along i1, multiply by the Coulomb table, inverse transform.  Stage 1 reads its
// elements straight from the scratch and the last inverse stage writes straight back (lanes
// over the 32 columns: coalesced); only the two exchanges in between go through shared memory.
// ---------------------------------------------------------------------------------------
template <int L, int V = 0>
struct ConvShape {
  static constexpr int R1 = Factor<L>::R1, R2 = Factor<L>::R2;
  // columns per CTA (lanes over columns): 32, or 16 in variant 2 (a half-warp per row, 128 bytes)
  static constexpr int TILE = V == 2 ? 16 : 32;
  static constexpr int LP = L + 1;
  // threads: 128 up to 108 points (more CTAs per SM), 256 for the longer pencils (measured on
  // 96, 128 and 160 points); variant 1 takes the other count, variant 2 128; ACE_CONV_NT overrides
  // the default
#ifdef ACE_CONV_NT
  static constexpr int NT0 = ACE_CONV_NT;
#else
  static constexpr int NT0 = L > 108 ? 256 : 128;
#endif
  static constexpr int NT = V == 0 ? NT0 : (V == 1 ? (NT0 == 128 ? 256 : 128) : 128);
  static_assert(NT % TILE == 0, "whole column tiles per pass of the threads");
};

template <typename T, int L, int V>
__global__ void __launch_bounds__(ConvShape<L, V>::NT) conv_pencil_kernel(PairPassArgs<T> a) {
  using S = ConvShape<L, V>;
  constexpr int R1 = S::R1, R2 = S::R2, TILE = S::TILE, LP = S::LP, NT = S::NT;
  constexpr int ROWS = NT / TILE;  // task rows handled at once
  __shared__ cpx<T> s[TILE * LP];
  __shared__ cpx<T> tw[L];
  const int tid = threadIdx.x;
  for (int e = tid; e < L; e += NT) tw[e] = a.tw[e];
  const long long cols = (long long)a.n2 * a.n3;
  const long long c0 = (long long)blockIdx.x * TILE;
  const int Ns = (int)cols;  // stride between consecutive i1 (fits: N < 2^31)
  cpx<T> *z = a.scratch + (long long)blockIdx.y * a.N + c0;
  const T *kc = a.kernel + c0;
  const int t = tid % TILE, row = tid / TILE;
  const bool valid = c0 + t < cols;
  __syncthreads();
  // stage 1 (forward): tasks (t, n2), n2 = row + ROWS q
#pragma unroll
  for (int q = 0; q < (TILE * R2 + NT - 1) / NT; ++q) {
    const int n2 = row + ROWS * q;
    if (n2 < R2 && valid) {
      cpx<T> x[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = z[(n1 * R2 + n2) * Ns + t];
      Dft<R1, -1, T>::run(x);
      cpx<T> *line = s + t * LP + n2;
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) line[k1 * R2] = k1 ? cmul(x[k1], tw[n2 * k1]) : x[0];
    }
  }
  __syncthreads();
  // stage 2 (forward), kernel multiply, inverse stage A: tasks (t, k1)
#pragma unroll
  for (int q = 0; q < (TILE * R1 + NT - 1) / NT; ++q) {
    const int k1 = row + ROWS * q;
    if (k1 < R1 && valid) {
      cpx<T> *blk = s + t * LP + k1 * R2;
      cpx<T> x[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) x[n2] = blk[n2];
      Dft<R2, -1, T>::run(x);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) x[k2] = cscale(x[k2], __ldg(kc + (k1 + R1 * k2) * Ns + t));
      Dft<R2, +1, T>::run(x);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) blk[n2] = (n2 && k1) ? cmul(x[n2], conjc(tw[n2 * k1])) : x[n2];
    }
  }
  __syncthreads();
  // inverse stage B: tasks (t, n2); natural order i1 = n1 R2 + n2 straight to the scratch
#pragma unroll
  for (int q = 0; q < (TILE * R2 + NT - 1) / NT; ++q) {
    const int n2 = row + ROWS * q;
    if (n2 < R2 && valid) {
      const cpx<T> *line = s + t * LP + n2;
      cpx<T> x[R1];
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) x[k1] = line[k1 * R2];
      Dft<R1, +1, T>::run(x);
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) z[(n1 * R2 + n2) * Ns + t] = x[n1];
    }
  }
}

template <typename T, int L, int V>
cudaError_t launch_conv_LV(const PairPassArgs<T> &a, int npacks, cudaStream_t st) {
  using S = ConvShape<L, V>;
  const long long cols = (long long)a.n2 * a.n3;
  dim3 grid((unsigned)((cols + S::TILE - 1) / S::TILE), npacks);
  conv_pencil_kernel<T, L, V><<<grid, S::NT, 0, st>>>(a);
  return cudaGetLastError();
}

// The axis-1 pass in the pencil tile a.conv_tile selects (FP32; the FP64 form keeps the default).
template <typename T, int L>
cudaError_t launch_conv_L(const PairPassArgs<T> &a, int npacks, cudaStream_t st) {
  if constexpr (sizeof(T) == 4) {
    if (a.conv_tile == 1) return launch_conv_LV<T, L, 1>(a, npacks, st);
    if (a.conv_tile == 2) return launch_conv_LV<T, L, 2>(a, npacks, st);
  }
  return launch_conv_LV<T, L, 0>(a, npacks, st);
}

template <typename T, int L>
cudaError_t launch_pass_L(int mode, const PairPassArgs<T> &a, int npacks, cudaStream_t st) {
  using S = PassShape<T, L>;
  dim3 grid;
  if (mode == PASS_FWD3_PAIR || mode == PASS_INV3_ACC) {
    grid.x = (unsigned)(((long long)a.n1 * a.n2 + S::TILE - 1) / S::TILE);
  } else if (mode == PASS_CONV1) {
    grid.x = (unsigned)(((long long)a.n2 * a.n3 + S::TILE - 1) / S::TILE);
  } else {
    grid.x = (unsigned)(a.n1 * ((a.n3 + S::TILE - 1) / S::TILE));
  }
  grid.y = npacks;
  switch (mode) {
    case PASS_FWD3_PAIR: pair_pass_kernel<T, L, PASS_FWD3_PAIR><<<grid, S::NT, 0, st>>>(a); break;
    case PASS_FWD2: pair_pass_kernel<T, L, PASS_FWD2><<<grid, S::NT, 0, st>>>(a); break;
    case PASS_CONV1: pair_pass_kernel<T, L, PASS_CONV1><<<grid, S::NT, 0, st>>>(a); break;
    case PASS_INV2: pair_pass_kernel<T, L, PASS_INV2><<<grid, S::NT, 0, st>>>(a); break;
    case PASS_INV3_ACC: pair_pass_kernel<T, L, PASS_INV3_ACC><<<grid, S::NT, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}


// Launchers of one length group (instantiated in pair_chain_[abcd]_f{32,64}.cu): true when L
// belongs to the group, with the launch status in *e.
#define ACE_PASS_CASE(L_)                                 \
  case L_:                                                \
    *e = launch_pass_L<T, L_>(mode, a, npacks, st);       \
    return true;
#define ACE_CONV_CASE(L_)                                 \
  case L_:                                                \
    *e = launch_conv_L<T, L_>(a, npacks, st);             \
    return true;
#define ACE_DEFINE_GROUP(NAME, TYPE, PASS_LIST, CONV_LIST)                                                   \
  bool pass_##NAME(int L, int mode, const PairPassArgs<TYPE> &a, int npacks, cudaStream_t st, cudaError_t *e) { \
    using T = TYPE;                                                                                           \
    switch (L) {                                                                                              \
      PASS_LIST(ACE_PASS_CASE)                                                                                \
      default: return false;                                                                                  \
    }                                                                                                         \
  }                                                                                                           \
  bool conv_##NAME(int L, const PairPassArgs<TYPE> &a, int npacks, cudaStream_t st, cudaError_t *e) {           \
    using T = TYPE;                                                                                           \
    switch (L) {                                                                                              \
      CONV_LIST(ACE_CONV_CASE)                                                                                \
      default: return false;                                                                                  \
    }                                                                                                         \
  }
#define ACE_NO_LENGTHS(X)

}  // namespace ace
