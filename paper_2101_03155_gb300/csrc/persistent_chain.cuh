// persistent_chain.cuh -- the whole pair-potential chain of a build (or of several builds on one
// grid) as one persistent kernel that walks the uneven screened pack list (Eq. vx with Eq. e:vij
// evaluated in reciprocal space).
//
// Tasks.  For pack p (two pairs, z = rho_ab + i rho_cd) held in scratch slot p % S:
//   F(p, i1)  forward plane: pair densities of plane i1, axes 3 and 2 (plane_forward)
//   C(p, g)   pencil group g of G columns: axis 1 forward, Coulomb multiply, axis 1 inverse
//   I(p, i1)  inverse plane: axes 2 and 3, then W += v phi (plane_inverse, plane_accumulate)
// C(p, .) needs every F(p, .), I(p, .) needs every C(p, .), and F(p, .) needs every I(p - S, .)
// (the slot's previous pack).  Counters per pack record finished tasks.
//
// Queue.  CTAs take task numbers from one global counter.  Task number t lies in round
// r = t / RS of RS = N1 + NC + N1 numbers: first the I tasks of pack r - 2 lag, then the C tasks of
// pack r - lag, then the F tasks of pack r.  Every dependency of a task lies in an earlier round,
// so it was taken earlier by a CTA that is running it or has finished it: the lowest-numbered
// unfinished task can always proceed, and the walk cannot deadlock, whatever the number of
// resident CTAs.  With lag rounds between the stages of one pack, a task rarely finds its inputs
// unfinished; when it does, thread 0 polls the counter with an acquire load (bounded in time:
// after wait_ns, 2 s by default, the kernel sets the error word and every CTA leaves).
//
// Memory order.  A task ends with a CTA barrier, then thread 0 fences and increments the pack's
// counter; a dependent task's thread 0 reads the counter with acquire semantics before a CTA
// barrier, and scratch data is read through L2 only (ld.global.cg), never from a stale L1 line.
#pragma once

#include "plane_chain.cuh"

namespace ace {


// Pencil columns per C task: as many as the plane work area holds, at most ACE_PERSIST_GMAX.
#ifndef ACE_PERSIST_GMAX
#define ACE_PERSIST_GMAX 128
#endif
template <typename T, int N1, int N2, int N3>
struct PersistShape {
  static constexpr int WORK_PLANE = N2 * (N3 + 1);
  static constexpr int G0 = WORK_PLANE / (N1 + 1);
  static constexpr int G = G0 > ACE_PERSIST_GMAX ? ACE_PERSIST_GMAX : G0;
  static constexpr int COLS = N2 * N3;
  static constexpr int NC = (COLS + G - 1) / G;
  static constexpr int WORK = WORK_PLANE > G * (N1 + 1) ? WORK_PLANE : G * (N1 + 1);
  // twiddle tables: one per distinct axis length
  static constexpr int NTW = N1 + (N2 == N1 ? 0 : N2) + ((N3 == N1 || N3 == N2) ? 0 : N3);
  static size_t smem() { return sizeof(cpx<T>) * (size_t)(WORK + NTW) + 16; }
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int *p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Axis-1 pass of one pack on the G columns [c0, c0 + G) of its scratch slot z ([N1][cols]):
// forward stage 1 (DFT_R1 + twiddle) straight from the scratch, stage 2 with the multiply by the
// permuted Coulomb table and the inverse stage A in registers, inverse stage B straight back to the
// scratch in natural order; two exchanges through shared memory (lanes over columns: coalesced).
template <typename T, int L, int G, int NT>
__device__ __forceinline__ void pencil_convolve(cpx<T> *z, const T *__restrict__ Kperm, int cols, int c0, cpx<T> *s,
                                                const cpx<T> *tw) {
  constexpr int LP = L + 1, R1 = Factor<L>::R1, R2 = Factor<L>::R2;
  const int gv = min(G, cols - c0);
  cpx<T> *zc = z + c0;
  // forward stage 1: tasks (t, n2): DFT_R1 over n1 of column t at i1 = n1 R2 + n2
  for_tasks<G, R2, NT>([&](int t, int n2) {
    if (t >= gv) return;
    cpx<T> x[R1];
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) x[n1] = ldcg_cpx(zc + (long long)(n1 * R2 + n2) * cols + t);
    Dft<R1, -1, T>::run(x);
    cpx<T> *line = s + t * LP + n2;
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) line[k1 * R2] = k1 ? cmul(x[k1], tw[n2 * k1]) : x[0];
  });
  __syncthreads();
  // forward stage 2, kernel multiply, inverse stage A: tasks (t, k1)
  for_tasks<G, R1, NT>([&](int t, int k1) {
    if (t >= gv) return;
    cpx<T> *blk = s + t * LP + k1 * R2;
    cpx<T> x[R2];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) x[n2] = blk[n2];
    Dft<R2, -1, T>::run(x);
    const T *kc = Kperm + c0 + t;
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) x[k2] = cscale(x[k2], __ldg(kc + (long long)(k1 + R1 * k2) * cols));
    Dft<R2, +1, T>::run(x);
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
      cpx<T> v = x[n2];
      if (n2 > 0) {
        const cpx<T> w = tw[n2 * k1];
        v = cmul(v, cpx<T>{w.x, -w.y});
      }
      blk[n2] = v;
    }
  });
  __syncthreads();
  // inverse stage B: tasks (t, n2); natural order i1 = n1 R2 + n2 straight to the scratch
  for_tasks<G, R2, NT>([&](int t, int n2) {
    if (t >= gv) return;
    const cpx<T> *line = s + t * LP + n2;
    cpx<T> x[R1];
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) x[k1] = line[k1 * R2];
    Dft<R1, +1, T>::run(x);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) zc[(long long)(n1 * R2 + n2) * cols + t] = x[n1];
  });
}

// Resident CTAs per SM the register budget is set for: the plane kernels' count unless
// ACE_PERSIST_MINB (a build-time setting) lowers it, which gives the pencil tasks more registers.
template <typename T, int N2, int N3>
constexpr int persist_min_blocks() {
#ifdef ACE_PERSIST_MINB
  return plane_min_blocks<T, N2, N3, false>() < ACE_PERSIST_MINB ? plane_min_blocks<T, N2, N3, false>()
                                                                 : ACE_PERSIST_MINB;
#else
  return plane_min_blocks<T, N2, N3, false>();
#endif
}

template <typename T, int N1, int N2, int N3, int NT>
__global__ void __launch_bounds__(NT, (persist_min_blocks<T, N2, N3>()))
    chain_persistent_kernel(PersistArgs<T> a) {
  using S = PlaneShape<N2, N3>;
  using P = PersistShape<T, N1, N2, N3>;
  constexpr int G = P::G, NC = P::NC, RS = 2 * N1 + NC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T> *s = reinterpret_cast<cpx<T> *>(smem_raw);
  cpx<T> *tw1 = s + P::WORK;
  cpx<T> *tw2 = (N2 == N1) ? tw1 : tw1 + N1;
  cpx<T> *tw3 = (N3 == N1) ? tw1 : ((N3 == N2) ? tw2 : tw1 + N1 + (N2 == N1 ? 0 : N2));
  int *sh = reinterpret_cast<int *>(tw1 + P::NTW);  // [0] next task number, [1] leave
  const int tid = threadIdx.x;
  for (int e = tid; e < N1; e += NT) tw1[e] = a.tw1[e];
  if (N2 != N1)
    for (int e = tid; e < N2; e += NT) tw2[e] = a.tw2[e];
  if (N3 != N1 && N3 != N2)
    for (int e = tid; e < N3; e += NT) tw3[e] = a.tw3[e];
  const int np = a.npacks_d ? __ldcg(a.npacks_d) : a.npacks;
  const long long total = (long long)RS * (np + 2 * a.lag);
  if (tid == 0) sh[0] = atomicAdd(a.ticket, 1);
  for (;;) {
    __syncthreads();  // sh[0] holds this CTA's next task number
    const int t = sh[0];
    __syncthreads();
    if (t >= total) break;
    int nxt = 0;
    if (tid == 0) nxt = atomicAdd(a.ticket, 1);  // taken now, stored at the end of the task
    const int r = t / RS, o = t - r * RS;
    int kind, p, idx;
    if (o < N1) {
      kind = 2, p = r - 2 * a.lag, idx = o;
    } else if (o < N1 + NC) {
      kind = 1, p = r - a.lag, idx = o - N1;
    } else {
      kind = 0, p = r, idx = o - N1 - NC;
    }
    const bool live = p >= 0 && p < np;
    if (tid == 0) {
      int leave = *reinterpret_cast<volatile int *>(a.err);
      if (live && !leave) {
        const int *cnt = nullptr;
        int need = 0;
        if (kind == 0 && p >= a.nslots) cnt = a.counters + 2 * np + (p - a.nslots), need = N1;
        if (kind == 1) cnt = a.counters + p, need = N1;
        if (kind == 2) cnt = a.counters + np + p, need = NC;
        if (kind == 1 && a.stall) cnt = a.stall, need = 1;  // test of the give-up path
        if (cnt && ld_acquire(cnt) < need) {
          const unsigned long long t0 = global_ns();
          while (ld_acquire(cnt) < need) {
            if (*reinterpret_cast<volatile int *>(a.err)) {
              leave = 1;
              break;
            }
            if (global_ns() - t0 > a.wait_ns) {
              atomicExch(a.err, 1);
              leave = 1;
              break;
            }
            __nanosleep(200);
          }
        }
      }
      sh[1] = leave;
    }
    __syncthreads();
    if (sh[1]) break;
    if (live) {
      const int b = a.pack_build ? a.pack_build[p] : 0;
      const ChainBuild<T> bd = a.builds[b];
      const int4 pk = a.packs[p];
      cpx<T> *slot = a.scratch + (long long)(p % a.nslots) * a.N;
      const bool skip = a.skip_rel > 0.f && bd.pmax;
      if (kind == 0) {
        const long long off = (long long)idx * S::NPTS;
        if (skip && fwd_plane_negligible(bd.pmax, bd.gmax, N1, idx, pk, a.skip_rel))
          zero_plane<T, S::NPTS, NT>(slot + off);
        else
          plane_forward<T, N2, N3, NT>(bd.phi, a.N, off, pk, s, tw2, tw3, slot + off);
      } else if (kind == 1) {
        pencil_convolve<T, N1, G, NT>(slot, bd.Kperm, S::NPTS, idx * G, s, tw1);
      } else {
        const long long off = (long long)idx * S::NPTS;
        if (!(skip && inv_plane_negligible(bd.pmax, bd.gmax, N1, idx, pk, a.skip_rel))) {
          plane_inverse<T, N2, N3, NT>(slot + off, s, tw2, tw3);
          plane_accumulate<T, N2, N3, NT>(bd.phi, bd.W, a.N, off, pk, s, nullptr);
        }
        if (a.hints & 1) l2_discard<NT>(slot + off, sizeof(cpx<T>) * S::NPTS);  // the plane's last use
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        red_release_add(a.counters + kind * np + p, 1);
      }
    }
    if (tid == 0) sh[0] = nxt;
  }
}

template <typename T, int N1, int N2, int N3>
struct PersistLaunch {
  static constexpr int NT = plane_threads<T, N2, N3>();
  static constexpr int NC = PersistShape<T, N1, N2, N3>::NC;
  static size_t smem() { return PersistShape<T, N1, N2, N3>::smem(); }
  // resident CTAs per SM of this kernel (0: does not fit)
  static int blocks_per_sm() {
    static unsigned long long done = 0;
    if (smem_attr_once(chain_persistent_kernel<T, N1, N2, N3, NT>, smem(), done) != cudaSuccess) return 0;
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, chain_persistent_kernel<T, N1, N2, N3, NT>, NT, smem()) !=
        cudaSuccess)
      return 0;
    return b;
  }
  static cudaError_t launch(const PersistArgs<T> &a, int grid, cudaStream_t st) {
    chain_persistent_kernel<T, N1, N2, N3, NT><<<grid, NT, smem(), st>>>(a);
    return cudaGetLastError();
  }
};

}  // namespace ace
