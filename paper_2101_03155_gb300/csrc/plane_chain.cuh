// plane_chain.cuh -- three-pass pair-potential chain: forward plane FFT (axes 3 and 2 of one
// N2 x N3 plane in shared memory), the axis-1 pencil pass (forward, kernel multiply, inverse), and
// the inverse plane FFT fused with the accumulation of W (Eq. vx, Eq. e:vij in reciprocal space).
//
// Spectrum layout in the scratch: [pack][i1][p2][p3] where p2, p3 are the positions the two-stage
// transform leaves its output in (natural index k = k1 + R1 k2 sits at p = k1 R2 + k2).  The
// axis-1 pass reads the Coulomb table in the same permuted layout, and the inverse plane pass
// starts from permuted input and returns natural order, so no reordering pass is needed.
//
// The inverse pass handles a group of packs whose pairs share the first orbital i (pairs (i, j1),
// (i, j2), ...).  With one pack per group (the default) the two W_i contributions of the pack are
// added with one atomic per point; with larger groups they are summed in shared memory over the
// group first.  W_j += v_ij phi_i are atomic adds.  Global accesses go one point per lane
// (coalesced) so that the shared-memory side stays free of bank conflicts.
#pragma once

#include "ace_internal.h"
#include "fft.cuh"

// unroll depth of the global-load loops (forward copy-in, inverse epilogue): loads of several
// iterations are issued before the first one is used
#ifndef ACE_FWD_UNROLL
#define ACE_FWD_UNROLL 4
#endif
#ifndef ACE_INV_UNROLL
#define ACE_INV_UNROLL 4
#endif
#define ACE_PRAGMA(x) _Pragma(#x)
#define ACE_UNROLL(n) ACE_PRAGMA(unroll n)

namespace ace {

// FP32 plane kernels: CTAs per SM that shared memory allows (at most ACE_PLANE_MAXB), used as the
// register budget so that registers do not lower that residency.  FP64 kernels keep the
// compiler's choice (one or two CTAs fit by shared memory there).
#ifndef ACE_PLANE_MAXB
#define ACE_PLANE_MAXB 3
#endif
template <typename T, int N2, int N3, bool ACC>
constexpr int plane_min_blocks() {
  constexpr long long bytes =
      (long long)sizeof(cpx<T>) * (N2 * (N3 + 1) + N2 + N3) + (ACC ? (long long)sizeof(T) * N2 * N3 : 0);
  constexpr long long fit = (227LL * 1024) / bytes;
  if (sizeof(T) != 4) return 1;
  return fit < 1 ? 1 : (fit > ACE_PLANE_MAXB ? ACE_PLANE_MAXB : (int)fit);
}

template <int N2, int N3>
struct PlaneShape {
  static constexpr int R1c = Factor<N2>::R1, R2c = Factor<N2>::R2;  // axis 2 (columns of the plane)
  static constexpr int R1r = Factor<N3>::R1, R2r = Factor<N3>::R2;  // axis 3 (rows of the plane)
  static constexpr int PP = N3 + 1;                                  // odd pitch (complex elements)
  static constexpr int NPTS = N2 * N3;
  static_assert(N3 % 4 == 0, "rows are processed in groups of four points");
};

// Per-thread walk over the tasks (l, m), l < NL, m < NM, of one stage (l fastest).  When NT is a
// multiple of NL a thread keeps one l and steps m by NT / NL, so the split of the task index is done
// once per thread instead of once per task.
template <int NL, int NM, int NT, typename F>
__device__ __forceinline__ void for_tasks(F &&f) {
  if constexpr (NT % NL == 0) {
    constexpr int STEP = NT / NL;
    const int l = threadIdx.x % NL;
#pragma unroll 1
    for (int m = threadIdx.x / NL; m < NM; m += STEP) f(l, m);
  } else {
#pragma unroll 1
    for (int task = threadIdx.x; task < NL * NM; task += NT) f(task % NL, task / NL);
  }
}

template <typename T, int NT>
struct PlaneStages {
  // stage 1 over NL lines of length L (element p of line l at s[l*LS + p*PS]):
  //   tasks (l, n2): DFT_R1 over n1 of x[n1 R2 + n2]; optional twiddle w_L^{D n2 k1}; result k1 at k1 R2 + n2
  template <int L, int NL, int LS, int PS, int D, bool TW>
  static __device__ __forceinline__ void stage1(cpx<T> *s, const cpx<T> *tw) {
    constexpr int R1 = Factor<L>::R1, R2 = Factor<L>::R2;
    for_tasks<NL, R2, NT>([&](int l, int n2) {
      cpx<T> *line = s + l * LS + n2 * PS;
      cpx<T> x[R1];
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) x[n1] = line[n1 * R2 * PS];
      Dft<R1, D, T>::run(x);
#pragma unroll
      for (int k1 = 0; k1 < R1; ++k1) {
        cpx<T> v = x[k1];
        if (TW && k1 > 0) {
          const cpx<T> w = tw[n2 * k1];
          v = cmul(v, D < 0 ? w : cpx<T>{w.x, -w.y});
        }
        line[k1 * R2 * PS] = v;
      }
    });
  }
  // stage 2: tasks (l, k1): DFT_R2 of the contiguous block k1 R2 + n2; output k2 at k1 R2 + k2
  template <int L, int NL, int LS, int PS, int D>
  static __device__ __forceinline__ void stage2(cpx<T> *s) {
    constexpr int R1 = Factor<L>::R1, R2 = Factor<L>::R2;
    for_tasks<NL, R1, NT>([&](int l, int k1) {
      cpx<T> *blk = s + l * LS + k1 * R2 * PS;
      cpx<T> x[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) x[n2] = blk[n2 * PS];
      Dft<R2, D, T>::run(x);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) blk[k2 * PS] = x[k2];
    });
  }
  // inverse stage A (permuted input): tasks (l, k1): inverse DFT_R2 over k2 of the block
  // k1 R2 + k2, conjugate twiddle w_L^{+n2 k1}; result n2 at k1 R2 + n2.  The k1 = 0 twiddles are
  // the table's exact 1 + 0i, so every n2 > 0 term is multiplied without a branch on k1.
  template <int L, int NL, int LS, int PS>
  static __device__ __forceinline__ void inv_stageA(cpx<T> *s, const cpx<T> *tw) {
    constexpr int R1 = Factor<L>::R1, R2 = Factor<L>::R2;
    for_tasks<NL, R1, NT>([&](int l, int k1) {
      cpx<T> *blk = s + l * LS + k1 * R2 * PS;
      cpx<T> x[R2];
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) x[k2] = blk[k2 * PS];
      Dft<R2, +1, T>::run(x);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) {
        cpx<T> v = x[n2];
        if (n2 > 0) {
          const cpx<T> w = tw[n2 * k1];
          v = cmul(v, cpx<T>{w.x, -w.y});
        }
        blk[n2 * PS] = v;
      }
    });
  }
};

// Walk over the points e = tid + it NT of an N2 x N3 plane: f(it, e, si) with si = i2 PP + i3 the
// padded shared-memory index.  When NT is a multiple of N3 the row of a thread's point advances by
// NT / N3 per step, so si needs no division.
template <int N2, int N3, int NT, int UNROLL, typename F>
__device__ __forceinline__ void for_points(F &&f) {
  constexpr int NPTS = N2 * N3, PP = N3 + 1;
  const int tid = threadIdx.x;
  if constexpr (NT % N3 == 0 && NPTS % NT == 0) {
    const int si0 = tid + tid / N3;
#pragma unroll UNROLL
    for (int it = 0; it < NPTS / NT; ++it) f(tid + it * NT, si0 + it * (NT + NT / N3));
  } else {
#pragma unroll UNROLL
    for (int e = tid; e < NPTS; e += NT) {
      const int i2 = e / N3;
      f(e, e + i2 * (PP - N3));
    }
  }
}

// Load of a complex value through L2 only (data written earlier by other CTAs of a running grid
// must not be served from this SM's L1)
__device__ __forceinline__ cpx<float> ldcg_cpx(const cpx<float> *p) {
  const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
  return cpx<float>{v.x, v.y};
}
__device__ __forceinline__ cpx<double> ldcg_cpx(const cpx<double> *p) {
  const double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
  return cpx<double>{v.x, v.y};
}

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
  static __device__ __forceinline__ void load(const float *p, float (&v)[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
  }
  static __device__ __forceinline__ void add(float *p, const float (&v)[4]) {
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  }
};
template <>
struct Vec4<double> {
  static __device__ __forceinline__ void load(const double *p, double (&v)[4]) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
  }
  static __device__ __forceinline__ void add(double *p, const double (&v)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) atomicAdd(p + k, v[k]);
  }
};

// ---------------------------------------------------------------------------------------
// Bodies shared by the per-batch kernels below and the persistent chain kernel.
// ---------------------------------------------------------------------------------------

// Forward transform of plane i1 (offset off = i1 N2 N3) of pack pk: the pair densities
// z = phi_a phi_b + i phi_c phi_d, axes 3 and 2, the permuted spectrum plane written to dst.
// Uses s (N2 x PP complex) and the twiddles tw2, tw3 in shared memory; starts with a barrier-free
// load and ends without a barrier.
template <typename T, int N2, int N3, int NT>
__device__ __forceinline__ void plane_forward(const T *__restrict__ phi, long long N, long long off, int4 pk,
                                              cpx<T> *s, const cpx<T> *tw2, const cpx<T> *tw3, cpx<T> *dst) {
  using S = PlaneShape<N2, N3>;
  using F = PlaneStages<T, NT>;
  const T *pa = phi + (long long)pk.x * N + off;
  const T *pb = phi + (long long)pk.y * N + off;
  if (pk.z == pk.x) {
    // row pack (a, b), (a, d): z = phi_a (phi_b + i phi_d), three planes read
    const T *pd = phi + (long long)pk.w * N + off;
    for_points<N2, N3, NT, ACE_FWD_UNROLL>([&](int e, int si) {
      const T fa = __ldg(pa + e);
      s[si] = cpx<T>{fa * __ldg(pb + e), fa * __ldg(pd + e)};
    });
  } else if (pk.z >= 0) {
    const T *pc = phi + (long long)pk.z * N + off;
    const T *pd = phi + (long long)pk.w * N + off;
    for_points<N2, N3, NT, ACE_FWD_UNROLL>([&](int e, int si) {
      s[si] = cpx<T>{__ldg(pa + e) * __ldg(pb + e), __ldg(pc + e) * __ldg(pd + e)};
    });
  } else {
    for_points<N2, N3, NT, ACE_FWD_UNROLL>([&](int e, int si) {
      s[si] = cpx<T>{__ldg(pa + e) * __ldg(pb + e), (T)0};
    });
  }
  __syncthreads();
  // axis 3 (rows): natural -> permuted
  F::template stage1<N3, N2, S::PP, 1, -1, true>(s, tw3);
  __syncthreads();
  F::template stage2<N3, N2, S::PP, 1, -1>(s);
  __syncthreads();
  // axis 2 (columns): stage 1 in shared memory, stage 2 straight to the scratch plane
  F::template stage1<N2, N3, 1, S::PP, -1, true>(s, tw2);
  __syncthreads();
  for_tasks<N3, S::R1c, NT>([&](int p3, int k1) {
    cpx<T> x[S::R2c];
#pragma unroll
    for (int n2 = 0; n2 < S::R2c; ++n2) x[n2] = s[(k1 * S::R2c + n2) * S::PP + p3];
    Dft<S::R2c, -1, T>::run(x);
#pragma unroll
    for (int k2 = 0; k2 < S::R2c; ++k2) dst[(k1 * S::R2c + k2) * N3 + p3] = x[k2];
  });
}

// Drops the 128-byte lines that lie wholly inside [base, base + bytes) from L2 without writing
// them back (their contents become undefined); the CTA's threads share the lines.
template <int NT>
__device__ __forceinline__ void l2_discard(const void *base, size_t bytes) {
  const unsigned long long b = reinterpret_cast<unsigned long long>(base);
  const unsigned long long first = (b + 127) & ~127ull, end = (b + bytes) & ~127ull;
  for (unsigned long long a = first + 128ull * threadIdx.x; a < end; a += 128ull * NT)
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}

// Inverse transform of one permuted spectrum plane src (read through L2 only: it was written
// by other CTAs) into natural order in s: axes 2 and 3.  Ends with a barrier; src is read only
// before the first barrier.
template <typename T, int N2, int N3, int NT>
__device__ __forceinline__ void plane_inverse(const cpx<T> *src, cpx<T> *s, const cpx<T> *tw2, const cpx<T> *tw3) {
  using S = PlaneShape<N2, N3>;
  using F = PlaneStages<T, NT>;
  // axis 2 inverse, stage A straight from the scratch plane (permuted rows p2 = k1 R2c + k2);
  // the k1 = 0 twiddles are the table's exact 1 + 0i
  for_tasks<N3, S::R1c, NT>([&](int p3, int k1) {
    cpx<T> x[S::R2c];
#pragma unroll
    for (int k2 = 0; k2 < S::R2c; ++k2) x[k2] = ldcg_cpx(src + (k1 * S::R2c + k2) * N3 + p3);
    Dft<S::R2c, +1, T>::run(x);
#pragma unroll
    for (int n2 = 0; n2 < S::R2c; ++n2) {
      cpx<T> v = x[n2];
      if (n2 > 0) {
        const cpx<T> w = tw2[n2 * k1];
        v = cmul(v, cpx<T>{w.x, -w.y});
      }
      s[(k1 * S::R2c + n2) * S::PP + p3] = v;
    }
  });
  __syncthreads();
  F::template stage1<N2, N3, 1, S::PP, +1, false>(s, tw2);  // inverse stage B: natural rows
  __syncthreads();
  F::template inv_stageA<N3, N2, S::PP, 1>(s, tw3);
  __syncthreads();
  F::template stage1<N3, N2, S::PP, 1, +1, false>(s, tw3);  // natural columns
  __syncthreads();
}

// W accumulation of one pack from v = v_ab + i v_cd at the natural points of plane offset off
// (Eq. vx): W_a += v_ab phi_b (+ v_ad phi_d for a row pack), W_b += v_ab phi_a, W_c += v_cd phi_d,
// W_d += v_cd phi_c, diagonal pairs once.  With acc (a group's shared first orbital) the W_a terms
// are summed into acc instead.
template <typename T, int N2, int N3, int NT>
__device__ __forceinline__ void plane_accumulate(const T *__restrict__ phi, T *W, long long N, long long off, int4 pk,
                                                 const cpx<T> *s, T *acc) {
  const bool two = pk.z >= 0;
  const bool same_a = two && pk.z == pk.x;
  const T *fa = phi + (long long)pk.x * N + off;
  const T *fb = phi + (long long)pk.y * N + off;
  const T *fc = phi + (long long)(two ? pk.z : 0) * N + off;
  const T *fd = phi + (long long)(two ? pk.w : 0) * N + off;
  T *wa = W + (long long)pk.x * N + off;
  T *wb = W + (long long)pk.y * N + off;
  T *wc = W + (long long)(two ? pk.z : 0) * N + off;
  T *wd = W + (long long)(two ? pk.w : 0) * N + off;
  auto last = [&](auto &&epi) {
    for_points<N2, N3, NT, ACE_INV_UNROLL>([&](int e, int si) { epi(e, s[si]); });
  };
  if (!acc && same_a && pk.y != pk.x && pk.w != pk.x) {
    // row pack (a, b), (a, d) with b, d != a: W_a += v_ab phi_b + v_ad phi_d, W_b += v_ab phi_a,
    // W_d += v_ad phi_a  (v = v_ab + i v_ad)
    last([&](int e, cpx<T> v) {
      const T pa_ = __ldg(fa + e), pb_ = __ldg(fb + e), pd_ = __ldg(fd + e);
      atomicAdd(wa + e, v.x * pb_ + v.y * pd_);
      atomicAdd(wb + e, v.x * pa_);
      atomicAdd(wd + e, v.y * pa_);
    });
  } else {
    // any pack: v = v_ab + i v_cd
    last([&](int e, cpx<T> v) {
      const T pa_ = __ldg(fa + e), pb_ = __ldg(fb + e);
      const T pc_ = two ? __ldg(fc + e) : (T)0, pd_ = two ? __ldg(fd + e) : (T)0;
      const T to_a = v.x * pb_ + (same_a ? v.y * pd_ : (T)0);
      if (acc) {
        acc[e] += to_a;  // pk.x == the group's row (and pk.z too when two)
      } else {
        atomicAdd(wa + e, to_a);
        if (two && !same_a) atomicAdd(wc + e, v.y * pd_);
      }
      if (pk.y != pk.x) atomicAdd(wb + e, v.x * pa_);
      if (two && pk.w != pk.z) atomicAdd(wd + e, v.y * pc_);
    });
  }
}

// ---------------------------------------------------------------------------------------
// Plane skip (mixed form).  Localized orbitals leave most of the cell with negligible values.
// On plane i1, the pair density phi_a phi_b is negligible when the product of the two orbitals'
// plane maxima is at most rel times the product of their overall maxima: its forward transform is
// then a zero plane.  The pack's W terms on plane i1 are products of the potential with the pack's
// orbitals, so when every orbital of the pack is at most rel times its maximum there, the inverse
// plane and its accumulation are skipped.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool fwd_plane_negligible(const float *pm, const float *gm, int n1, int i1, int4 pk,
                                                     float rel) {
  const bool ab = __ldg(pm + pk.x * n1 + i1) * __ldg(pm + pk.y * n1 + i1) <= rel * __ldg(gm + pk.x) * __ldg(gm + pk.y);
  if (pk.z < 0) return ab;
  return ab && __ldg(pm + pk.z * n1 + i1) * __ldg(pm + pk.w * n1 + i1) <= rel * __ldg(gm + pk.z) * __ldg(gm + pk.w);
}
__device__ __forceinline__ bool inv_plane_negligible(const float *pm, const float *gm, int n1, int i1, int4 pk,
                                                     float rel) {
  bool s = __ldg(pm + pk.x * n1 + i1) <= rel * __ldg(gm + pk.x) && __ldg(pm + pk.y * n1 + i1) <= rel * __ldg(gm + pk.y);
  if (pk.z >= 0)
    s = s && __ldg(pm + pk.z * n1 + i1) <= rel * __ldg(gm + pk.z) && __ldg(pm + pk.w * n1 + i1) <= rel * __ldg(gm + pk.w);
  return s;
}
// A zero spectrum plane (the forward transform of a negligible density plane).
template <typename T, int NPTS, int NT>
__device__ __forceinline__ void zero_plane(cpx<T> *dst) {
  for (int e = threadIdx.x; e < NPTS; e += NT) dst[e] = cpx<T>{(T)0, (T)0};
}

// ---------------------------------------------------------------------------------------
// Forward plane pass: one CTA per (plane i1, pack).
// ---------------------------------------------------------------------------------------
template <typename T, int N2, int N3, int NT>
__global__ void __launch_bounds__(NT, (plane_min_blocks<T, N2, N3, false>())) plane_fwd_kernel(PlaneArgs<T> a) {
  using S = PlaneShape<N2, N3>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *s = reinterpret_cast<cpx<T> *>(smem_raw);
  cpx<T> *tw2 = s + N2 * S::PP;
  cpx<T> *tw3 = tw2 + N2;
  const int tid = threadIdx.x;
  const int i1 = blockIdx.x;
  const int pidx = a.pack0 + blockIdx.y;
  const int4 pk = a.packs[pidx];
  for (int e = tid; e < N2; e += NT) tw2[e] = a.tw2[e];
  for (int e = tid; e < N3; e += NT) tw3[e] = a.tw3[e];
  const long long off = (long long)i1 * S::NPTS;
  if (a.skip_rel > 0.f && fwd_plane_negligible(a.pmax, a.gmax, a.n1, i1, pk, a.skip_rel)) {
    zero_plane<T, S::NPTS, NT>(a.scratch + (long long)(pidx - a.batch0) * a.N + off);
    return;
  }
  plane_forward<T, N2, N3, NT>(a.phi, a.N, off, pk, s, tw2, tw3, a.scratch + (long long)(pidx - a.batch0) * a.N + off);
}

// ---------------------------------------------------------------------------------------
// Inverse plane pass fused with the W accumulation: one CTA per (plane i1, group).
// Group g covers packs [gstart, gstart + glen); grow >= 0 means every pair of the group has
// first orbital grow (accumulated in shared memory), grow < 0 a single mixed pack.
// ---------------------------------------------------------------------------------------
template <typename T, int N2, int N3, int NT, bool ACC>
__global__ void __launch_bounds__(NT, (plane_min_blocks<T, N2, N3, ACC>())) plane_inv_kernel(PlaneArgs<T> a) {
  using S = PlaneShape<N2, N3>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *s = reinterpret_cast<cpx<T> *>(smem_raw);
  cpx<T> *tw2 = s + N2 * S::PP;
  cpx<T> *tw3 = tw2 + N2;
  T *acc = reinterpret_cast<T *>(tw3 + N3);  // NPTS values when ACC
  const int tid = threadIdx.x;
  const int i1 = blockIdx.x;
  const int4 grp = a.groups[a.group0 + blockIdx.y];  // (start pack, count, row, unused)
  const int grow = grp.z;
  for (int e = tid; e < N2; e += NT) tw2[e] = a.tw2[e];
  for (int e = tid; e < N3; e += NT) tw3[e] = a.tw3[e];
  const bool use_acc = ACC && grow >= 0;
  if (use_acc)
    for (int e = tid; e < S::NPTS; e += NT) acc[e] = (T)0;
  const long long off = (long long)i1 * S::NPTS;
  for (int q = 0; q < grp.y; ++q) {
    const int pidx = grp.x + q;
    const int4 pk = a.packs[pidx];
    __syncthreads();  // previous pack's epilogue has finished reading s
    if (!(a.skip_rel > 0.f && inv_plane_negligible(a.pmax, a.gmax, a.n1, i1, pk, a.skip_rel))) {
      plane_inverse<T, N2, N3, NT>(a.scratch + (long long)(pidx - a.batch0) * a.N + off, s, tw2, tw3);
      plane_accumulate<T, N2, N3, NT>(a.phi, a.W, a.N, off, pk, s, use_acc ? acc : nullptr);
    }
    // the spectrum plane was this pack's last use of it: its lines leave L2 without a write-back
    // (here, where few registers are live; every read of it ended at plane_inverse's first barrier)
    if (a.hints & 1) l2_discard<NT>(a.scratch + (long long)(pidx - a.batch0) * a.N + off, sizeof(cpx<T>) * S::NPTS);
  }
  if (use_acc) {
    __syncthreads();
    T *wr = a.W + (long long)grow * a.N + off;
    for (int e = tid; e < S::NPTS; e += NT) atomicAdd(wr + e, acc[e]);
  }
}

// The dynamic shared-memory limit of a kernel, set once per device (a driver call per launch
// would cost about as much host time as the launch itself).
template <typename Kern>
inline cudaError_t smem_attr_once(Kern k, size_t bytes, unsigned long long &done_bits) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (__atomic_load_n(&done_bits, __ATOMIC_ACQUIRE) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) __atomic_fetch_or(&done_bits, bit, __ATOMIC_RELEASE);
  return e;
}

// Threads of a plane CTA: as many warps as the register file allows for the CTAs that shared
// memory fits on an SM (FP32: exactly 3 CTAs -> 448 threads at 40 registers, 2 -> 768, 1 -> 1024;
// smaller planes, which fit more CTAs, keep 384); FP64 planes keep 384 (twice the registers per
// complex value).  ACE_PLANE_NT overrides.
template <typename T, int N2, int N3>
constexpr int plane_threads() {
#ifdef ACE_PLANE_NT
  return ACE_PLANE_NT;
#else
  constexpr long long bytes = (long long)sizeof(cpx<T>) * (N2 * (N3 + 1) + N2 + N3);
  constexpr long long fit = (227LL * 1024) / bytes;
  if (sizeof(T) != 4) return 384;
  return fit > 3 ? 384 : (fit == 3 ? 448 : (fit == 2 ? 768 : 1024));
#endif
}

template <typename T, int N2, int N3>
struct PlaneLaunch {
  static constexpr int NT = plane_threads<T, N2, N3>();
  static size_t fwd_smem() { return sizeof(cpx<T>) * (N2 * PlaneShape<N2, N3>::PP + N2 + N3); }
  static size_t inv_smem(bool acc) {
    return fwd_smem() + (acc ? sizeof(T) * (size_t)N2 * N3 : 0);
  }
  static bool fits(bool acc) { return inv_smem(acc) <= 227 * 1024 && fwd_smem() <= 227 * 1024; }

  static cudaError_t fwd(const PlaneArgs<T> &a, int npacks, cudaStream_t st) {
    const size_t sm = fwd_smem();
    static unsigned long long done = 0;
    cudaError_t e = smem_attr_once(plane_fwd_kernel<T, N2, N3, NT>, sm, done);
    if (e != cudaSuccess) return e;
    plane_fwd_kernel<T, N2, N3, NT><<<dim3(a.n1, npacks), NT, sm, st>>>(a);
    return cudaGetLastError();
  }
  static cudaError_t inv(const PlaneArgs<T> &a, int ngroups, bool acc, cudaStream_t st) {
    const size_t sm = inv_smem(acc);
    cudaError_t e;
    if (acc) {
      static unsigned long long done_acc = 0;
      e = smem_attr_once(plane_inv_kernel<T, N2, N3, NT, true>, sm, done_acc);
      if (e != cudaSuccess) return e;
      plane_inv_kernel<T, N2, N3, NT, true><<<dim3(a.n1, ngroups), NT, sm, st>>>(a);
    } else {
      static unsigned long long done = 0;
      e = smem_attr_once(plane_inv_kernel<T, N2, N3, NT, false>, sm, done);
      if (e != cudaSuccess) return e;
      plane_inv_kernel<T, N2, N3, NT, false><<<dim3(a.n1, ngroups), NT, sm, st>>>(a);
    }
    return cudaGetLastError();
  }
};

}  // namespace ace
