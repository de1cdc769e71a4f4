// gemm_tc.cu -- the dense contractions of the mixed form on the 5th-generation tensor cores
// (tcgen05, sm_103a) as BF16x3 split products:
//   a = a_hi + a_lo, a_hi = bf16(a), a_lo = bf16(a - a_hi);  a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi
// accumulated in FP32 in tensor memory (TMEM).
//
//   tc_gram:     G = scale * X Y^T  (M = -dV Phi^T W of App. A; C = dV xi^T psi of the ACE
//                application).  Each CTA sums one chunk of grid points (256 by default) in FP32 in
//                TMEM and writes a 128 x 128 partial; a second kernel adds the chunks in FP64 in a
//                fixed order.  Longer FP32 chunks lose accuracy in the tensor-core accumulator.
//   tc_left_mul: Z = A Y with A small (xi = L^-1 W, i.e. xi = W L^-T of App. A; out = -C^T xi).
//
// Operands are staged through registers (FP32 -> bf16 hi/lo) into shared memory in the K-major,
// no-swizzle canonical layout: 8 x 8 "core matrices" of 128 contiguous bytes, K-adjacent core
// matrices LBO = 128 B apart, row-group-adjacent ones SBO = 512 B apart (a 32-wide K step).  One
// thread issues the MMAs (M = 128, N = 128, K = 16 each) and commits them to an mbarrier; every
// wait on an mbarrier is bounded and reports a timeout through *err instead of hanging.
#include <cuda.h>  // CUtensorMap and its enums (types only; the encoder is reached through cudart)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <mutex>

#include "ace_internal.h"
#include "f32x2.cuh"

namespace ace {
namespace tc {

constexpr int NT = 128;        // four warps: warp w reads TMEM lanes 32w .. 32w + 31
constexpr int NT2 = 256;       // TMA kernels: warps w and w + 4 share TMEM lanes 32w .. 32w + 31
constexpr int BM = 128;        // UMMA M
constexpr int BN = 128;        // UMMA N
constexpr int BK = 32;         // K per pipeline stage (two K = 16 MMAs)
constexpr uint32_t LBO = 128;  // bytes between K-adjacent core matrices
constexpr uint32_t SBO = 512;  // bytes between row-adjacent core-matrix groups (BK / 8 * 128)
constexpr uint32_t TILE_BYTES = BM * BK * 2;  // one bf16 operand tile (8 KB)
constexpr uint32_t kWaitLimit = 1u << 22;     // try_wait polls before a wait is declared stuck
constexpr int kGramChunkDefault = 256;        // grid points summed in FP32 (in TMEM) before the FP64 sum

// instruction descriptor of tcgen05.mma kind::f16: D = F32 (bits 4-5), A = B = BF16 (bits 7-9,
// 10-12), both K-major (bits 15, 16 clear), N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4 (16-29), SBO >> 4 (32-45),
// descriptor version 1 (bits 46-47), base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((LBO >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init_n(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// bounded wait for the phase with the given parity (at most `limit` polls); false if it never
// completed
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit = kWaitLimit) {
  for (uint32_t it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Two-stage commit tracking: commits on barrier s complete its phases in order.
struct Pipe {
  uint32_t phase[2];
  int pending[2];
  __device__ __forceinline__ void init() {
    phase[0] = phase[1] = 0u;
    pending[0] = pending[1] = 0;
  }
  // wait for the outstanding commit of stage s (if any); false on timeout
  __device__ __forceinline__ bool drain(uint64_t *mbar, int s) {
    if (!pending[s]) return true;
    const bool ok = mbar_wait(smem_u32(&mbar[s]), phase[s]);
    phase[s] ^= 1u;
    pending[s] = 0;
    return ok;
  }
};

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this thread's TMEM lane from registers (completion: tmem_st_wait)
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const float (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}
__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane (load waits for its data)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15]))
      : "memory");
}

// first 1024-byte aligned address of the dynamic shared array, as an offset from it (so that the
// compiler keeps the shared state space and emits LDS / STS rather than generic accesses)
__device__ __forceinline__ unsigned char *align1024(unsigned char *dyn) {
  return dyn + ((1024u - (smem_u32(dyn) & 1023u)) & 1023u);
}

// byte offset of element (row, k) of a 128 x 32 K-major tile in the canonical layout
__device__ __forceinline__ uint32_t tile_off(int row, int k) {
  return (uint32_t)(row >> 3) * SBO + (uint32_t)(k >> 3) * LBO + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// ---- TMA (cp.async.bulk.tensor) into shared memory, completion counted on an mbarrier ----
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
// box at (x, y) of a 2D tensor map (x innermost, a multiple of 4 FP32 = 16 bytes)
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
      : "memory");
}

// box at (x, y) of a 2D tensor map from shared memory (bulk-group completion)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// wait until at most N committed bulk groups still read their shared-memory source
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// wait until every committed bulk group has completed its writes
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// bf16 hi/lo of two values at once: hi = bf16_rn(x) for the pair (one packed conversion), the
// residuals x - hi in FP32 (exact: hi carries the top bits of x), lo = bf16_rn(residual)
__device__ __forceinline__ void split2(float x0, float x1, uint32_t &hi, uint32_t &lo) {
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));  // x0 in the low half
  const float h0 = __uint_as_float(hi << 16), h1 = __uint_as_float(hi & 0xFFFF0000u);
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(x1 - h1), "f"(x0 - h0));
}

// 16-byte core-matrix row: 8 bf16 (hi) and 8 bf16 (lo) of 8 consecutive K-values of one row
__device__ __forceinline__ void split8(const float (&x)[8], uint4 &hi, uint4 &lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) split2(x[2 * i], x[2 * i + 1], h[i], l[i]);
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// One operand row (32 K-values) per thread, held in registers between load and store.
struct Row32 {
  float v[32];
};

// row r of a row-major matrix (ld = K), K-values [k0, k0 + 32); zero past nrows
__device__ __forceinline__ void load_row(const float *__restrict__ M, long long ld, int r, int nrows, long long k0,
                                         Row32 &out) {
  if (r < nrows) {
    const float4 *src = reinterpret_cast<const float4 *>(M + (long long)r * ld + k0);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 t = __ldg(src + q);
      out.v[4 * q] = t.x;
      out.v[4 * q + 1] = t.y;
      out.v[4 * q + 2] = t.z;
      out.v[4 * q + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 32; ++q) out.v[q] = 0.f;
  }
}

// the thread's row of a 128 x 32 tile: four 16-byte stores into each of the hi and lo tiles
// (lanes are consecutive rows, so each quarter-warp writes 128 contiguous bytes)
__device__ __forceinline__ void store_row(const Row32 &r, int row, unsigned char *hi, unsigned char *lo) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = r.v[8 * q + i];
    uint4 h, l;
    split8(x, h, l);
    const uint32_t off = tile_off(row, 8 * q);
    *reinterpret_cast<uint4 *>(hi + off) = h;
    *reinterpret_cast<uint4 *>(lo + off) = l;
  }
}

// K-values [16 h, 16 h + 16) of the thread's row of a 128 x 32 tile (two 16-byte stores into each
// of the hi and lo tiles)
__device__ __forceinline__ void store_half_row(const float (&v)[16], int row, int h, unsigned char *hi,
                                               unsigned char *lo) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = v[8 * q + i];
    uint4 hv, lv;
    split8(x, hv, lv);
    const uint32_t off = tile_off(row, 16 * h + 8 * q);
    *reinterpret_cast<uint4 *>(hi + off) = hv;
    *reinterpret_cast<uint4 *>(lo + off) = lv;
  }
}

// column c of Y (row-major n x K), K-rows [l0, l0 + 32): 32 scalar loads, coalesced across lanes
__device__ __forceinline__ void load_col(const float *__restrict__ Y, long long ld, int l0, int nl, long long c,
                                         Row32 &out) {
#pragma unroll
  for (int j = 0; j < 32; ++j) out.v[j] = (l0 + j < nl) ? __ldg(Y + (long long)(l0 + j) * ld + c) : 0.f;
}

struct SmemLayout {
  // two pipeline stages x {A_hi, A_lo, B_hi, B_lo}
  static constexpr uint32_t kStage = 4 * TILE_BYTES;
  static constexpr uint32_t kBytes = 2 * kStage + 2048;  // + barriers / TMEM address, + alignment slack
};

// ----------------------------------------------------------------------------------------
// Gram: partial[chunk][i][j] = sum_{r in chunk} X[i][r] Y[j][r], 128 x 128 tile per CTA.
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) tc_gram_kernel(const float *__restrict__ X, int nx, const float *__restrict__ Y,
                                                     int ny, long long K, int chunk, int tiles_x,
                                                     float *__restrict__ partial, int *__restrict__ err) {
  extern __shared__ unsigned char dyn[];
  unsigned char *base = align1024(dyn);
  uint64_t *mbar = reinterpret_cast<uint64_t *>(base + 2 * SmemLayout::kStage);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int ti = blockIdx.x % tiles_x, tj = blockIdx.x / tiles_x;
  const int i0 = ti * BM, j0 = tj * BN;
  const long long kb = (long long)blockIdx.y * chunk;
  const long long ke = min(K, kb + chunk);
  const int nsteps = (int)((ke - kb) / BK);

  if (warp == 0) tmem_alloc(tmem_slot, 128);
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]));
    mbar_init(smem_u32(&mbar[1]));
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  Pipe pipe;
  pipe.init();
  bool ok = true;
  Row32 nx_a, nx_b;  // prefetched rows of the next K-step
  if (nsteps > 0) {
    load_row(X, K, i0 + tid, nx, kb, nx_a);
    load_row(Y, K, j0 + tid, ny, kb, nx_b);
  }
  for (int it = 0; it < nsteps; ++it) {
    const int s = it & 1;
    unsigned char *st = base + s * SmemLayout::kStage;
    const Row32 cur_a = nx_a, cur_b = nx_b;
    if (it + 1 < nsteps) {
      const long long k1 = kb + (long long)(it + 1) * BK;
      load_row(X, K, i0 + tid, nx, k1, nx_a);
      load_row(Y, K, j0 + tid, ny, k1, nx_b);
    }
    ok = pipe.drain(mbar, s);  // the MMAs that last read this stage are done
    if (__syncthreads_or(!ok)) {
      ok = false;
      break;
    }
    store_row(cur_a, tid, st, st + TILE_BYTES);
    store_row(cur_b, tid, st + 2 * TILE_BYTES, st + 3 * TILE_BYTES);
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a_hi = smem_u32(st), a_lo = a_hi + TILE_BYTES, b_hi = a_hi + 2 * TILE_BYTES,
                     b_lo = a_hi + 3 * TILE_BYTES;
#pragma unroll
      for (int ks = 0; ks < BK / 16; ++ks) {
        const uint32_t o = ks * 2 * LBO;
        mma(tmem, sdesc(a_hi + o), sdesc(b_hi + o), (it > 0 || ks > 0) ? 1u : 0u);
        mma(tmem, sdesc(a_hi + o), sdesc(b_lo + o), 1u);
        mma(tmem, sdesc(a_lo + o), sdesc(b_hi + o), 1u);
      }
      commit(smem_u32(&mbar[s]));
    }
    pipe.pending[s] = 1;
  }
  // every commit waited for (also after a timeout, so that no MMA is in flight at dealloc)
  const bool d0 = pipe.drain(mbar, 0), d1 = pipe.drain(mbar, 1);
  ok = !__syncthreads_or(!(ok && d0 && d1));
  tc_fence_after();
  if (ok) {
    const int i = i0 + 32 * warp + (tid & 31);
    float *dst = partial + ((long long)blockIdx.y * nx + i) * ny;
#pragma unroll 1
    for (int cb = 0; cb < BN / 32; ++cb) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * cb, v);
      if (nsteps == 0) {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = 0.f;
      }
      const int jb = j0 + 32 * cb;
      if (i < nx) {
        if ((ny & 3) == 0 && jb + 32 <= ny) {
          float4 *d4 = reinterpret_cast<float4 *>(dst + jb);  // 128 contiguous bytes of row i
#pragma unroll
          for (int c = 0; c < 8; ++c) d4[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
        } else {
#pragma unroll
          for (int c = 0; c < 32; ++c)
            if (jb + c < ny) dst[jb + c] = v[c];
        }
      }
    }
  } else if (tid == 0) {
    atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// Chunk partials summed in FP64 in two fixed-order levels: block (e-range, group g) adds chunks
// g*per .. g*per + per - 1 for 256 consecutive entries into part2[g][e]; then G = scale * sum_g.
constexpr int kReduceGroups = 64;
__global__ void gram_reduce_kernel(const float *__restrict__ partial, int nchunks, int ne,
                                   double *__restrict__ part2) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  const int per = (nchunks + kReduceGroups - 1) / kReduceGroups;
  const int c0 = blockIdx.y * per, c1 = min(nchunks, c0 + per);
  double s = 0.0;
#pragma unroll 8
  for (int c = c0; c < c1; ++c) s += (double)__ldg(partial + (long long)c * ne + e);
  part2[(long long)blockIdx.y * ne + e] = s;
}
__global__ void gram_reduce2_kernel(const double *__restrict__ part2, int ne, double scale, double *__restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
  for (int g = 0; g < kReduceGroups; ++g) s += part2[(long long)g * ne + e];
  G[e] = scale * s;
}

// ----------------------------------------------------------------------------------------
// Left multiply: Z[i][c] = sum_l A[i][l] Y[l][c] for rows [i0, i0 + 128) of A (m x n) and
// column tiles of 128, persistent over the column tiles.  The A rows are split into bf16 hi/lo
// once per CTA and stay in shared memory (n/32 K-steps of 2 x 8 KB); each K-step of Y is staged
// one column per thread (32 coalesced scalar loads, prefetched one step ahead).
// ----------------------------------------------------------------------------------------
__global__ void __launch_bounds__(NT) tc_left_mul_kernel(const float *__restrict__ A, int m, int n,
                                                         const float *__restrict__ Y, long long K, float *__restrict__ Z,
                                                         int *__restrict__ err) {
  extern __shared__ unsigned char dyn[];
  unsigned char *base = align1024(dyn);
  const int nsteps = (n + BK - 1) / BK;
  unsigned char *a_tiles = base;                            // nsteps x {hi, lo}
  unsigned char *b_stage = base + (size_t)nsteps * 2 * TILE_BYTES;  // 2 stages x {hi, lo}
  uint64_t *mbar = reinterpret_cast<uint64_t *>(b_stage + 2 * 2 * TILE_BYTES);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int i0 = blockIdx.y * BM;
  const long long ntiles = K / BN;

  if (warp == 0) tmem_alloc(tmem_slot, 128);
  if (tid == 0) {
    mbar_init(smem_u32(&mbar[0]));
    mbar_init(smem_u32(&mbar[1]));
    mbar_init_fence();
  }
  // resident A: row i0 + tid, all K-steps
  for (int it = 0; it < nsteps; ++it) {
    Row32 r;
    if (i0 + tid < m) {
#pragma unroll
      for (int j = 0; j < 32; ++j) r.v[j] = (it * BK + j < n) ? __ldg(A + (long long)(i0 + tid) * n + it * BK + j) : 0.f;
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) r.v[j] = 0.f;
    }
    unsigned char *t = a_tiles + (size_t)it * 2 * TILE_BYTES;
    store_row(r, tid, t, t + TILE_BYTES);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  Pipe pipe;
  pipe.init();
  bool ok = true;
  Row32 nxt;
  long long t0 = blockIdx.x;
  if (t0 < ntiles) load_col(Y, K, 0, n, t0 * BN + tid, nxt);
  for (long long t = t0; t < ntiles && ok; t += gridDim.x) {
    const long long c0 = t * BN;
    for (int it = 0; it < nsteps; ++it) {
      const int s = it & 1;
      unsigned char *st = b_stage + s * 2 * TILE_BYTES;
      const Row32 cur = nxt;
      // prefetch the next K-step of this tile, or the first K-step of the next tile
      if (it + 1 < nsteps) {
        load_col(Y, K, (it + 1) * BK, n, c0 + tid, nxt);
      } else if (t + gridDim.x < ntiles) {
        load_col(Y, K, 0, n, (t + gridDim.x) * BN + tid, nxt);
      }
      ok = pipe.drain(mbar, s);
      if (__syncthreads_or(!ok)) {
        ok = false;
        break;
      }
      store_row(cur, tid, st, st + TILE_BYTES);
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_hi = smem_u32(a_tiles + (size_t)it * 2 * TILE_BYTES), a_lo = a_hi + TILE_BYTES;
        const uint32_t b_hi = smem_u32(st), b_lo = b_hi + TILE_BYTES;
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint32_t o = ks * 2 * LBO;
          mma(tmem, sdesc(a_hi + o), sdesc(b_hi + o), (it > 0 || ks > 0) ? 1u : 0u);
          mma(tmem, sdesc(a_hi + o), sdesc(b_lo + o), 1u);
          mma(tmem, sdesc(a_lo + o), sdesc(b_hi + o), 1u);
        }
        commit(smem_u32(&mbar[s]));
      }
      pipe.pending[s] = 1;
    }
    if (!ok) break;
    // wait for every MMA of this tile, then read D (lane = row i, columns = c)
    const bool d0 = pipe.drain(mbar, 0), d1 = pipe.drain(mbar, 1);
    ok = !__syncthreads_or(!(d0 && d1));
    if (!ok) break;
    tc_fence_after();
    const int i = i0 + 32 * warp + (tid & 31);
#pragma unroll 1
    for (int cb = 0; cb < BN / 32; ++cb) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32 * cb, v);
      if (i < m) {
        float4 *dst = reinterpret_cast<float4 *>(Z + (long long)i * K + c0 + 32 * cb);
#pragma unroll
        for (int c = 0; c < 8; ++c) dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
      }
    }
    tc_fence_before();
    __syncthreads();  // D is read before the next tile's first MMA overwrites it
  }
  if (!ok) {
    pipe.drain(mbar, 0);  // bounded: leave no MMA in flight before TMEM is released
    pipe.drain(mbar, 1);
    if (tid == 0) atomicExch(err, 1);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 128);
}

// ----------------------------------------------------------------------------------------
// Left multiply fed by TMA: Z[i][c] = sum_l A[i][l] Y[l][c] for rows [i0, i0 + 128) of A.
//   - A rows: split into bf16 hi/lo once per CTA, resident in shared memory (n/32 K-steps).
//   - Y: boxes of 32 rows x 128 columns (16 KB FP32) arrive by TMA in a ring of `ring` stages,
//     issued `ring` items ahead by thread 0; an item is one (column tile, K-step).
//   - Each thread splits column `tid` of a box into the K-major B tile (two B buffers, so that
//     the split of item q overlaps the MMAs of item q - 1).
//   - Two TMEM accumulators: tile j accumulates in accumulator j & 1 while the epilogue of
//     tile j - 1 reads the other one.
// Every wait is bounded; after a timeout the kernel waits (bounded) for its copies and MMAs in
// flight, releases TMEM and reports through *err.
// ----------------------------------------------------------------------------------------
constexpr uint32_t kLmBox = BK * BN * 4;   // one Y box: 32 rows x 128 FP32 columns
constexpr uint32_t kEpiBox = BM * 32 * 4;  // one Z box: 128 rows x 32 FP32 columns

__global__ void __launch_bounds__(NT2, 1) tc_left_mul_tma_kernel(const float *__restrict__ A, int m, int n,
                                                                const __grid_constant__ CUtensorMap tmY,
                                                                const __grid_constant__ CUtensorMap tmZ, long long K,
                                                                int ring, int *__restrict__ err) {
  extern __shared__ unsigned char dyn[];
  unsigned char *base = align1024(dyn);
  const int nsteps = (n + BK - 1) / BK;
  unsigned char *a_tiles = base;                                    // nsteps x {hi, lo}
  unsigned char *b_ops = a_tiles + (size_t)nsteps * 2 * TILE_BYTES;  // 2 buffers x {hi, lo}
  unsigned char *epi = b_ops + 2 * 2 * TILE_BYTES;                  // 2 x 128 rows x 32 FP32 (swizzled)
  unsigned char *boxes = epi + 2 * kEpiBox;                         // ring x kLmBox
  uint64_t *full = reinterpret_cast<uint64_t *>(boxes + (size_t)ring * kLmBox);
  uint64_t *mmad = full + ring;  // MMAs of the items that read B buffer b
  uint64_t *accf = mmad + 2;     // every MMA of the tile in accumulator a
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accf + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int quarter = warp & 3, half = warp >> 2;  // TMEM lane quarter; K-half / column half
  const int col = tid & 127;                       // row of the A tile / column of the Y box
  const int i0 = blockIdx.y * BM;
  // a last tile of fewer than BN columns reads zeros past column K (the map's bounds) and stores
  // only its columns below K
  const long long ntiles = (K + BN - 1) / BN;
  const long long mytiles = ntiles > (long long)blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const long long Q = mytiles * nsteps;

  if (warp == 0) tmem_alloc(tmem_slot, 256);
  if (tid == 0) {
    for (int r = 0; r < ring; ++r) mbar_init(smem_u32(&full[r]));
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&mmad[b]));
      mbar_init(smem_u32(&accf[b]));
    }
    mbar_init_fence();
  }
  __syncthreads();
  // items are numbered q = tile_slot * nsteps + kstep; the producer walks them with counters
  int p_stage = 0, p_step = 0;
  long long p_tile = blockIdx.x;
  auto issue_next = [&]() {  // thread 0: the next item into stage p_stage
    const uint32_t mb = smem_u32(&full[p_stage]);
    mbar_expect_tx(mb, kLmBox);
    tma_load_2d(smem_u32(boxes + (size_t)p_stage * kLmBox), &tmY, (int)(p_tile * BN), p_step * BK, mb);
    if (++p_stage == ring) p_stage = 0;
    if (++p_step == nsteps) {
      p_step = 0;
      p_tile += gridDim.x;
    }
  };
  const int Qi = (int)Q;
  int issued = Qi < ring ? Qi : ring;
  if (tid == 0)
    for (int k = 0; k < issued; ++k) issue_next();
  // resident A: row i0 + col, K-values [16 half, 16 half + 16) of every K-step (overlaps the first copies)
  for (int it = 0; it < nsteps; ++it) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int k = it * BK + 16 * half + j;
      v[j] = (i0 + col < m && k < n) ? __ldg(A + (long long)(i0 + col) * n + k) : 0.f;
    }
    unsigned char *t = a_tiles + (size_t)it * 2 * TILE_BYTES;
    store_half_row(v, col, half, t, t + TILE_BYTES);
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  Pipe pipe;
  pipe.init();
  bool ok = true;
  int q = 0;
  auto epilogue = [&](int j) -> bool {
    const int a = j & 1;
    const bool w = mbar_wait(smem_u32(&accf[a]), (uint32_t)((j >> 1) & 1));
    if (__syncthreads_or(!w)) return false;
    tc_fence_after();
    const long long c0 = (blockIdx.x + (long long)j * gridDim.x) * BN;
    const int row = 32 * quarter + (tid & 31);  // TMEM lane = row of the tile
    // two rounds: warps 0-3 stage column block r in buffer 0, warps 4-7 block r + 2 in buffer 1
#pragma unroll 1
    for (int r = 0; r < 2; ++r) {
      const int cb = r + 2 * half;
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)a * BN + 32 * cb, v);
      unsigned char *eb = epi + (size_t)half * kEpiBox;
      if (tid == 0) bulk_wait_read<0>();  // both buffers have been read by the previous stores
      __syncthreads();
      // row `row`: 128 bytes, 16-byte chunk q at position q ^ (row & 7) (the map's 128-byte swizzle)
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<float4 *>(eb + row * 128 + ((q ^ (row & 7)) << 4)) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        if (c0 + 32 * r < K) tma_store_2d(&tmZ, (int)(c0 + 32 * r), i0, smem_u32(epi));
        if (c0 + 32 * (r + 2) < K) tma_store_2d(&tmZ, (int)(c0 + 32 * (r + 2)), i0, smem_u32(epi + kEpiBox));
        bulk_commit();
      }
    }
    tc_fence_before();
    __syncthreads();  // accumulator a is read before tile j + 2 writes it
    return true;
  };
  int stage = 0, st = 0, j = 0;
  uint32_t fpar = 0;  // parity of the current pass over the ring
  for (; q < Qi; ++q) {
    const int b = q & 1;
    const bool got = mbar_wait(smem_u32(&full[stage]), fpar);
    const bool freed = pipe.drain(mmad, b);
    if (__syncthreads_or(!(got && freed))) {
      ok = false;
      break;
    }
    {
      // column `col` of the box, rows [16 half, 16 half + 16)
      float v[16];
      const float *box = reinterpret_cast<const float *>(boxes + (size_t)stage * kLmBox);
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = box[(16 * half + k) * BN + col];
      unsigned char *bt = b_ops + (size_t)b * 2 * TILE_BYTES;
      store_half_row(v, col, half, bt, bt + TILE_BYTES);
    }
    fence_async_smem();
    __syncthreads();  // the box is consumed and the B tile written
    if (tid == 0) {
      if (issued < Qi) {
        issue_next();
        ++issued;
      }
      tc_fence_after();
      const uint32_t acc = tmem + (uint32_t)(j & 1) * BN;
      const uint32_t a_hi = smem_u32(a_tiles + (size_t)st * 2 * TILE_BYTES), a_lo = a_hi + TILE_BYTES;
      const uint32_t b_hi = smem_u32(b_ops + (size_t)b * 2 * TILE_BYTES), b_lo = b_hi + TILE_BYTES;
#pragma unroll
      for (int ks = 0; ks < BK / 16; ++ks) {
        const uint32_t o = ks * 2 * LBO;
        mma(acc, sdesc(a_hi + o), sdesc(b_hi + o), (st > 0 || ks > 0) ? 1u : 0u);
        mma(acc, sdesc(a_hi + o), sdesc(b_lo + o), 1u);
        mma(acc, sdesc(a_lo + o), sdesc(b_hi + o), 1u);
      }
      commit(smem_u32(&mmad[b]));
      if (st == nsteps - 1) commit(smem_u32(&accf[j & 1]));
    } else if (issued < Qi) {
      ++issued;  // every thread tracks what thread 0 has issued
    }
    pipe.pending[b] = 1;
    const bool first = st == 0;
    if (++stage == ring) {
      stage = 0;
      fpar ^= 1u;
    }
    if (first && j > 0 && !epilogue(j - 1)) {
      ok = false;
      ++q;  // item q was consumed
      break;
    }
    if (++st == nsteps) {
      st = 0;
      ++j;
    }
  }
  if (ok && Qi > 0) ok = epilogue((int)mytiles - 1);
  if (!ok) {
    // bounded waits for the copies still in flight (items q .. issued - 1) and the last MMAs
    for (int r = q; r < issued; ++r) mbar_wait(smem_u32(&full[r % ring]), (uint32_t)((r / ring) & 1));
    pipe.drain(mmad, 0);
    pipe.drain(mmad, 1);
    if (tid == 0) atomicExch(err, 1);
  }
  if (tid == 0) bulk_wait_all();  // the stores have left shared memory before the CTA exits
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// ----------------------------------------------------------------------------------------
// Gram fed by TMA: partial[s][i][j] = sum over the chunks of split s of sum_r X[i][r] Y[j][r] for
// one 128 x 128 tile, as a warp-specialised pipeline (no CTA barrier per K-step):
//   - warp 20 (TMA): X and Y boxes of 128 rows x 32 points (16 KB FP32, 128-byte swizzled) into a
//     ring of `ring` stages, each stage refilled once the split warps have read it;
//   - warps 0-15 (split): warps 0-7 take the rows of the X box, warps 8-15 those of the Y box, two
//     threads per row (16 K-values each), split them into bf16 hi/lo and store them into the
//     K-major A or B tiles of one of `nops` operand buffers;
//   - warp 21 (MMA, one lane): three BF16 products per 16-point K-slice into one of two TMEM
//     accumulators; each chunk of `cs` K-steps stays in FP32 in one accumulator (a longer FP32
//     accumulation in the tensor core loses accuracy);
//   - warps 16-19 (fold, TMEM lane quarter warp & 3): add each finished chunk to a running sum kept
//     in TMEM with Kahan compensation (sum and compensation in TMEM columns 256-383 and 384-511),
//     release the accumulator, and at the end write the split's sum minus its compensation in
//     FP64; a second kernel adds the splits in FP64 in a fixed order.
// Every wait is bounded; a wait that gives up raises a shared flag that ends every role, the TMA
// warp waits (bounded) for its boxes in flight and the MMA lane for its last commit before the
// tensor memory is released.
// ----------------------------------------------------------------------------------------
constexpr uint32_t kGBox = BM * BK * 4;  // 128 rows x 32 FP32
constexpr int GW_SPLIT = 16;                           // split warps: two threads per row
constexpr int GW_FOLD0 = GW_SPLIT, GW_TMA = GW_SPLIT + 4, GW_MMA = GW_SPLIT + 5;
constexpr int GW_NT = (GW_SPLIT + 6) * 32;             // + 4 fold warps, the TMA warp, the MMA warp
constexpr int GW_OPS = 3;                // operand buffers (bf16 hi/lo tiles of both operands)

template <bool ABS>
__global__ void __launch_bounds__(GW_NT, 1) tc_gram_tma_kernel(const __grid_constant__ CUtensorMap tmX,
                                                              const __grid_constant__ CUtensorMap tmY, int nx, int ny,
                                                              long long c0, long long K, int cs, int tiles_x,
                                                              int ring, int nops, double *__restrict__ partial,
                                                              int *__restrict__ err, uint32_t first_wait) {
  extern __shared__ unsigned char dyn[];
  unsigned char *base = align1024(dyn);
  unsigned char *ops = base;                                       // nops x {A_hi, A_lo, B_hi, B_lo}
  unsigned char *boxes = ops + (size_t)nops * 4 * TILE_BYTES;     // ring x {X box, Y box}
  uint64_t *box_full = reinterpret_cast<uint64_t *>(boxes + (size_t)ring * 2 * kGBox);
  uint64_t *box_empty = box_full + ring;  // 8 split-warp arrivals
  uint64_t *op_full = box_empty + ring;   // 8 split-warp arrivals
  uint64_t *op_empty = op_full + nops;    // MMA commit
  uint64_t *acc_full = op_empty + nops;   // MMA commit after a chunk's last K-step
  uint64_t *acc_empty = acc_full + 2;     // 4 fold-warp arrivals
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ti = blockIdx.x % tiles_x, tj = blockIdx.x / tiles_x;
  const int i0 = ti * BM, j0 = tj * BN;
  // X and Y are the same matrix (the screen) and this tile is on the diagonal: one box per K-step
  // serves both operands
  const bool diag = ABS && ti == tj;
  // this split's K-steps: whole chunks [c_lo, c_hi) of cs steps (the last chunk may be short)
  const long long KS = K / BK, C = (KS + cs - 1) / cs;
  const long long c_lo = (long long)blockIdx.y * C / gridDim.y, c_hi = (long long)(blockIdx.y + 1) * C / gridDim.y;
  const long long ks_lo = c_lo * cs, ks_hi = min(KS, c_hi * (long long)cs);
  const int Q = (int)(ks_hi > ks_lo ? ks_hi - ks_lo : 0);
  const int NCH = (Q + cs - 1) / cs;

  if (warp == 0) tmem_alloc(tmem_slot, 512);
  if (tid == 0) {
    for (int r = 0; r < ring; ++r) {
      mbar_init(smem_u32(&box_full[r]));
      mbar_init_n(smem_u32(&box_empty[r]), GW_SPLIT);
    }
    for (int b = 0; b < nops; ++b) {
      mbar_init_n(smem_u32(&op_full[b]), GW_SPLIT);
      mbar_init(smem_u32(&op_empty[b]));
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&acc_full[a]));
      mbar_init_n(smem_u32(&acc_empty[a]), 4);
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // bounded wait for use `use` of a barrier (parity use & 1) that also leaves when another role has
  // given up; false = leave
  auto wait = [&](uint64_t *bar, int use, uint32_t limit) -> bool {
    const uint32_t mb = smem_u32(bar), parity = (uint32_t)(use & 1);
    for (uint32_t it = 0; it < limit; it += 64) {
      if (mbar_wait(mb, parity, 64)) return true;
      if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
  };

  if (warp == GW_TMA) {
    // ---- TMA: K-step q into stage q % ring once step q - ring has been read ----
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < Q; ++q) {
        const int stage = q % ring;
        if (q >= ring && !wait(&box_empty[stage], q / ring - 1, kWaitLimit)) break;
        const uint32_t mb = smem_u32(&box_full[stage]);
        unsigned char *bx = boxes + (size_t)stage * 2 * kGBox;
        const int x = (int)(c0 + (ks_lo + q) * BK);
        mbar_expect_tx(mb, diag ? kGBox : 2 * kGBox);
        tma_load_2d(smem_u32(bx), &tmX, x, i0, mb);
        if (!diag) tma_load_2d(smem_u32(bx + kGBox), &tmY, x, j0, mb);
        issued = q + 1;
      }
      // no box may still be landing when the CTA ends: wait (bounded) for the last ones
      for (int q = issued > ring ? issued - ring : 0; q < issued; ++q)
        mbar_wait(smem_u32(&box_full[q % ring]), (uint32_t)((q / ring) & 1));
    }
  } else if (warp == GW_MMA) {
    // ---- MMA lane: three products per K-slice; a chunk per accumulator ----
    if (lane == 0) {
      int last = -1;  // last K-step whose MMAs were committed
      for (int q = 0; q < Q; ++q) {
        const int b = q % nops, kin = q % cs, cl = q / cs, a = cl & 1;
        if (kin == 0 && cl >= 2 && !wait(&acc_empty[a], (cl >> 1) - 1, kWaitLimit)) break;
        if (!wait(&op_full[b], q / nops, kWaitLimit)) break;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)a * BN;
        const uint32_t a_hi = smem_u32(ops + (size_t)b * 4 * TILE_BYTES), a_lo = a_hi + TILE_BYTES;
        const uint32_t b_hi = a_hi + 2 * TILE_BYTES, b_lo = a_hi + 3 * TILE_BYTES;
#pragma unroll
        for (int ks = 0; ks < BK / 16; ++ks) {
          const uint32_t o = ks * 2 * LBO;
          mma(acc, sdesc(a_hi + o), sdesc(b_hi + o), (kin > 0 || ks > 0) ? 1u : 0u);
          mma(acc, sdesc(a_hi + o), sdesc(b_lo + o), 1u);
          mma(acc, sdesc(a_lo + o), sdesc(b_hi + o), 1u);
        }
        commit(smem_u32(&op_empty[b]));
        if (kin == cs - 1 || q == Q - 1) commit(smem_u32(&acc_full[a]));
        last = q;
      }
      // the tensor memory is released at the end: wait (bounded) for the last MMAs
      if (last >= 0) mbar_wait(smem_u32(&op_empty[last % nops]), (uint32_t)((last / nops) & 1));
    }
  } else if (warp >= GW_FOLD0) {
    // ---- fold warps: TMEM lanes 32 (warp & 3) .. + 31, all 128 columns, 16 at a time ----
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    {
      float z[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) z[c] = 0.f;
#pragma unroll 1
      for (int cb = 0; cb < 8; ++cb) {
        tmem_st16(tmem + lane_off + 256 + 16 * cb, z);
        tmem_st16(tmem + lane_off + 384 + 16 * cb, z);
      }
      tmem_st_wait();
    }
    bool ok = true;
    for (int c = 0; c < NCH; ++c) {
      const int a = c & 1;
      // every lane polls; the lanes may leave the poll loop apart, and the TMEM loads and stores
      // below are warp-collective (.sync.aligned): reconverge first
      const bool got = wait(&acc_full[a], c >> 1, kWaitLimit);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      tc_fence_after();
#pragma unroll 1
      for (int cb = 0; cb < 8; ++cb) {
        float x[16], sm[16], cp[16];
        tmem_ld16(tmem + lane_off + (uint32_t)a * BN + 16 * cb, x);
        tmem_ld16(tmem + lane_off + 256 + 16 * cb, sm);
        tmem_ld16(tmem + lane_off + 384 + 16 * cb, cp);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
          const float y = x[e] - cp[e];
          const float t = sm[e] + y;
          cp[e] = (t - sm[e]) - y;
          sm[e] = t;
        }
        tmem_st16(tmem + lane_off + 256 + 16 * cb, sm);
        tmem_st16(tmem + lane_off + 384 + 16 * cb, cp);
      }
      tmem_st_wait();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&acc_empty[a]));
    }
    if (ok && !*abort_flag) {
      const int i = i0 + 32 * (warp & 3) + lane;
      double *dst = partial + ((long long)blockIdx.y * nx + i) * ny;
#pragma unroll 1
      for (int cb = 0; cb < 8; ++cb) {
        float sm[16], cp[16];
        tmem_ld16(tmem + lane_off + 256 + 16 * cb, sm);
        tmem_ld16(tmem + lane_off + 384 + 16 * cb, cp);
        const int jb = j0 + 16 * cb;
        if (i < nx) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (jb + e < ny) dst[jb + e] = (double)sm[e] - (double)cp[e];
        }
      }
    }
  } else {
    // ---- split warps: warps 0-7 take X rows into the A tiles, warps 8-15 Y rows into the B
    // tiles; a thread takes the K-values [16 h, 16 h + 16) of row `row` (h = bit 7 of its index);
    // row `row` of a box holds its 16-byte chunk k4 at position k4 ^ (row & 7) ----
    const int row = tid & 127, h = (tid >> 7) & 1, half = tid >> 8;
    for (int q = 0; q < Q; ++q) {
      const int stage = q % ring, b = q % nops;
      // the first wait may be given fewer polls (a test of the give-up path)
      if (!__all_sync(0xffffffffu, wait(&box_full[stage], q / ring, q == 0 ? first_wait : kWaitLimit))) break;
      float v[16];
      const unsigned char *rowp = boxes + (size_t)stage * 2 * kGBox + (size_t)(diag ? 0 : half) * kGBox + row * 128;
#pragma unroll
      for (int c4 = 0; c4 < 4; ++c4) {
        const int k4 = 4 * h + c4;
        const float4 t = *reinterpret_cast<const float4 *>(rowp + ((k4 ^ (row & 7)) << 4));
        v[4 * c4] = ABS ? fabsf(t.x) : t.x;
        v[4 * c4 + 1] = ABS ? fabsf(t.y) : t.y;
        v[4 * c4 + 2] = ABS ? fabsf(t.z) : t.z;
        v[4 * c4 + 3] = ABS ? fabsf(t.w) : t.w;
      }
      // the bf16 hi/lo words first, then the wait for the operand buffer (its MMAs from nops
      // K-steps ago), then the stores
      uint4 hi[2], lo[2];
#pragma unroll
      for (int c8 = 0; c8 < 2; ++c8) {
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = v[8 * c8 + e];
        split8(x, hi[c8], lo[c8]);
      }
      if (q >= nops && !__all_sync(0xffffffffu, wait(&op_empty[b], q / nops - 1, kWaitLimit))) break;
      unsigned char *ob = ops + (size_t)b * 4 * TILE_BYTES + (size_t)half * 2 * TILE_BYTES;
#pragma unroll
      for (int c8 = 0; c8 < 2; ++c8) {
        const uint32_t off = tile_off(row, 16 * h + 8 * c8);
        *reinterpret_cast<uint4 *>(ob + off) = hi[c8];
        *reinterpret_cast<uint4 *>(ob + TILE_BYTES + off) = lo[c8];
      }
      fence_async_smem();  // the tiles are read by the tensor cores (async proxy)
      __syncwarp();
      // the box is released only now that every lane has used the values it loaded from it (a
      // release right after the loads let the next copy land in the box while reads were pending)
      if (lane == 0) {
        mbar_arrive(smem_u32(&box_empty[stage]));
        mbar_arrive(smem_u32(&op_full[b]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// G = scale * sum over the splits of partial[s] (FP64, fixed order); with `accumulate` the sum is
// added to G instead
__global__ void gram_splits_reduce_kernel(const double *__restrict__ partial, int splits, int ne, double scale,
                                          bool accumulate, double *__restrict__ G) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
#pragma unroll 8
  for (int k = 0; k < splits; ++k) s += partial[(long long)k * ne + e];
  G[e] = (accumulate ? G[e] : 0.0) + scale * s;
}

// ----------------------------------------------------------------------------------------
// Screen fed by TMA (section II: O_ij = dV sum_r |phi_i phi_j|, i <= j): FP32 on the CUDA cores.
//   - One CTA: a 64 x 64 tile (bi <= bj) of the upper triangle over one split of the columns.
//   - Boxes of 64 rows x 32 points of phi (128-byte swizzled) arrive by TMA through a ring; a
//     diagonal tile loads one box for both operands.
//   - Eight warps stage |phi| as (a, a) pairs (row block) and plain values (column block), then
//     each thread accumulates 4 x 4 outputs with packed f32x2 FMAs; 32-point FP32 partials are
//     added with Kahan compensation, and the tile's sums go to G with FP64 atomics.
// ----------------------------------------------------------------------------------------
constexpr int SC_B = 64;                      // rows per block
constexpr uint32_t kSBox = SC_B * BK * 4;     // 64 rows x 32 points

__global__ void __launch_bounds__(NT2, 2) screen_tma_kernel(const __grid_constant__ CUtensorMap tmX, int n,
                                                            long long c0, long long K, double scale, int ring,
                                                            double *__restrict__ G, int *__restrict__ err) {
  extern __shared__ unsigned char dyn[];
  unsigned char *base = align1024(dyn);
  unsigned char *boxes = base;  // ring x {row box, column box}
  float2 (*xs)[SC_B + 2] = reinterpret_cast<float2 (*)[SC_B + 2]>(boxes + (size_t)ring * 2 * kSBox);
  float (*ys)[SC_B + 4] = reinterpret_cast<float (*)[SC_B + 4]>(reinterpret_cast<unsigned char *>(xs) +
                                                                 sizeof(float2) * BK * (SC_B + 2));
  uint64_t *full = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(ys) + sizeof(float) * BK * (SC_B + 4));
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  int bi = 0, t = blockIdx.x;
  {
    const int nb = (n + SC_B - 1) / SC_B;
    while (t >= nb - bi) {
      t -= nb - bi;
      ++bi;
    }
  }
  const int bj = bi + t;
  const bool diag = bi == bj;
  const long long KS = K / BK;
  const long long ks_lo = (long long)blockIdx.y * KS / gridDim.y, ks_hi = (long long)(blockIdx.y + 1) * KS / gridDim.y;
  const int Q = (int)(ks_hi - ks_lo);
  if (tid == 0) {
    for (int r = 0; r < ring; ++r) mbar_init(smem_u32(&full[r]));
    mbar_init_fence();
  }
  __syncthreads();
  int p_stage = 0;
  long long p_ks = ks_lo;
  auto issue_next = [&]() {
    const uint32_t mb = smem_u32(&full[p_stage]);
    unsigned char *bx = boxes + (size_t)p_stage * 2 * kSBox;
    mbar_expect_tx(mb, diag ? kSBox : 2 * kSBox);
    tma_load_2d(smem_u32(bx), &tmX, (int)(c0 + p_ks * BK), bi * SC_B, mb);
    if (!diag) tma_load_2d(smem_u32(bx + kSBox), &tmX, (int)(c0 + p_ks * BK), bj * SC_B, mb);
    if (++p_stage == ring) p_stage = 0;
    ++p_ks;
  };
  int issued = Q < ring ? Q : ring;
  if (tid == 0)
    for (int k = 0; k < issued; ++k) issue_next();
  unsigned long long acc[4][2], comp[4][2];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = comp[a][b] = 0ull;
  bool ok = true;
  int q = 0, stage = 0;
  uint32_t fpar = 0;
  for (; q < Q; ++q) {
    const bool got = mbar_wait(smem_u32(&full[stage]), fpar);
    if (__syncthreads_or(!got)) {
      ok = false;
      break;
    }
    {
      // row `row` of a box: 16-byte chunk k4 at position k4 ^ (row & 7) (128-byte swizzle)
      const int row = tid & 63;
      const unsigned char *bx = boxes + (size_t)stage * 2 * kSBox;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k4 = (tid >> 6) + 4 * h;
        const float4 va = *reinterpret_cast<const float4 *>(bx + row * 128 + ((k4 ^ (row & 7)) << 4));
        const float4 vb = diag ? va : *reinterpret_cast<const float4 *>(bx + kSBox + row * 128 + ((k4 ^ (row & 7)) << 4));
        const float a4[4] = {fabsf(va.x), fabsf(va.y), fabsf(va.z), fabsf(va.w)};
        const float b4[4] = {fabsf(vb.x), fabsf(vb.y), fabsf(vb.z), fabsf(vb.w)};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          xs[4 * k4 + c][row] = make_float2(a4[c], a4[c]);
          ys[4 * k4 + c][row] = b4[c];
        }
      }
    }
    __syncthreads();  // the box is consumed; the staged operands are complete
    if (tid == 0) {
      if (issued < Q) {
        issue_next();
        ++issued;
      }
    } else if (issued < Q) {
      ++issued;
    }
    unsigned long long part[4][2];
#pragma unroll
    for (int a = 0; a < 4; ++a) part[a][0] = part[a][1] = 0ull;
#pragma unroll 8
    for (int k = 0; k < BK; ++k) {
      const ulonglong2 a01 = *reinterpret_cast<const ulonglong2 *>(&xs[k][ty * 4]);
      const ulonglong2 a23 = *reinterpret_cast<const ulonglong2 *>(&xs[k][ty * 4 + 2]);
      const ulonglong2 b = *reinterpret_cast<const ulonglong2 *>(&ys[k][tx * 4]);
      const unsigned long long av[4] = {a01.x, a01.y, a23.x, a23.y};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        part[r][0] = f2fma(av[r], b.x, part[r][0]);
        part[r][1] = f2fma(av[r], b.y, part[r][1]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const unsigned long long y = f2sub(part[r][c], comp[r][c]);
        const unsigned long long sm = f2add(acc[r][c], y);
        comp[r][c] = f2sub(f2sub(sm, acc[r][c]), y);
        acc[r][c] = sm;
      }
    if (++stage == ring) {
      stage = 0;
      fpar ^= 1u;
    }
    __syncthreads();  // the staged operands are read before the next step rewrites them
  }
  if (ok) {
    const int i0 = bi * SC_B, j0 = bj * SC_B;
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
  } else {
    for (int r = q; r < issued; ++r) mbar_wait(smem_u32(&full[r % ring]), (uint32_t)((r / ring) & 1));
    if (tid == 0) atomicExch(err, 1);
  }
}


// ----------------------------------------------------------------------------------------
// Screen on the CUDA cores, the default of the mixed form (section II: O_ij = dV sum_r
// |phi_i(r) phi_j(r)|, i <= j): FP32 products, FP32 partial sums over 64 grid points added into an
// FP32 running sum per K-split, FP64 across the K-splits in a fixed order.
//   - A 128 x 128 block pair (bi <= bj) of O is cut into 32 x 32 warp blocks.  A diagonal block
//     pair is one work unit of the 10 warp blocks on or above its diagonal; an off-diagonal pair is
//     two units (its row halves) of 8 warp blocks.  One CTA = one unit x one split of the points.
//   - Warp-specialised pipeline over a ring of shared-memory slots, handed on by mbarriers (no CTA
//     barrier per step): warp 10 issues the TMA boxes (128 rows x 32 points, 128-byte swizzle) into
//     a slot once the multiply warps have released it; warp 11 replaces each landed box by |phi| in
//     place; warps 0-9 multiply straight out of the slot and release it.
//   - Lane (ti, tj) = (lane / 8, lane % 8) owns rows ti + 4 rr (rr < 8) and columns tj + 8 cc
//     (cc < 4) of its warp block.  Per four grid points it loads one 16-byte run of each of its 8
//     rows and 4 columns (every such load of a warp touches distinct bank groups: its rows differ
//     in their low three bits, which select the swizzled position) and issues 64 packed f32x2 FMAs,
//     each multiplying two neighbouring grid points of one (row, column) pair.
//   - Every wait is bounded; a wait that gives up raises a shared flag that ends every role, and
//     the TMA warp waits (bounded) for its boxes in flight before it leaves.
// ----------------------------------------------------------------------------------------
constexpr int SY_MUL = 10;                  // multiply warps
constexpr int SY_NT = 32 * (SY_MUL + 2);    // + the TMA warp and the |phi| warp
constexpr int SY_RING = 5;
constexpr int SY_FOLD = 2;                  // K-steps per FP32 partial (64 points)
constexpr uint32_t kSyBox = 128 * BK * 4;   // 128 rows x 32 FP32 = 16 KB
constexpr size_t kSySmem = (size_t)SY_RING * 2 * kSyBox + 3 * SY_RING * 8 + 16 + 1024;

__global__ void __launch_bounds__(SY_NT, 1) screen_syrk_kernel(const __grid_constant__ CUtensorMap tmX, int n,
                                                               long long c0, long long K, int ndiag,
                                                               double *__restrict__ partial, int *__restrict__ err,
                                                               float *__restrict__ pmax, float *__restrict__ gmax,
                                                               long long npl, int n1) {
  extern __shared__ unsigned char dyn[];
  unsigned char *boxes = align1024(dyn);  // ring x {row box, column box}
  uint64_t *full = reinterpret_cast<uint64_t *>(boxes + (size_t)SY_RING * 2 * kSyBox);  // TMA landed
  uint64_t *ready = full + SY_RING;   // |phi| written (1 arrival)
  uint64_t *empty = ready + SY_RING;  // multiply warps done with the slot (SY_MUL arrivals)
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + SY_RING);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // work unit -> block pair (bi, bj), row half h (off-diagonal units)
  int bi, bj, h = 0;
  const int u = blockIdx.x;
  const bool diag = u < ndiag;
  if (diag) {
    bi = bj = u;
  } else {
    int t = (u - ndiag) >> 1;
    h = (u - ndiag) & 1;
    bi = 0;
    while (t >= ndiag - 1 - bi) {
      t -= ndiag - 1 - bi;
      ++bi;
    }
    bj = bi + 1 + t;
  }
  const long long KS = (K + BK - 1) / BK;
  const long long s_lo = (long long)blockIdx.y * KS / gridDim.y, s_hi = (long long)(blockIdx.y + 1) * KS / gridDim.y;
  const int Q = (int)(s_hi - s_lo);
  const int nbox = diag ? 1 : 2;
  if (tid == 0) {
    for (int r = 0; r < SY_RING; ++r) {
      mbar_init(smem_u32(&full[r]));
      mbar_init_n(smem_u32(&ready[r]), 1);
      mbar_init_n(smem_u32(&empty[r]), SY_MUL);
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  __syncthreads();
  // bounded wait that also leaves when another role has given up; false = leave
  auto wait = [&](uint64_t *bar, int q) -> bool {
    const uint32_t mb = smem_u32(bar), parity = (uint32_t)((q / SY_RING) & 1);
    for (uint32_t it = 0; it < kWaitLimit; it += 64) {
      if (mbar_wait(mb, parity, 64)) return true;
      if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
  };

  if (warp == SY_MUL) {
    // ---- TMA warp (one lane): box q into slot q % SY_RING once box q - SY_RING has been used ----
    if (lane == 0) {
      int issued = 0;
      for (int q = 0; q < Q; ++q) {
        const int slot = q % SY_RING;
        if (q >= SY_RING && !wait(&empty[slot], q - SY_RING)) break;
        const uint32_t mb = smem_u32(&full[slot]);
        unsigned char *bx = boxes + (size_t)slot * 2 * kSyBox;
        const int x = (int)(c0 + (s_lo + q) * BK);
        mbar_expect_tx(mb, nbox * kSyBox);
        tma_load_2d(smem_u32(bx), &tmX, x, bi * 128, mb);
        if (!diag) tma_load_2d(smem_u32(bx + kSyBox), &tmX, x, bj * 128, mb);
        issued = q + 1;
      }
      // no box may still be landing when the CTA ends (the other roles may leave early after a
      // give-up): wait (bounded) for the boxes whose slots were not refilled
      for (int q = issued > SY_RING ? issued - SY_RING : 0; q < issued; ++q)
        mbar_wait(smem_u32(&full[q % SY_RING]), (uint32_t)((q / SY_RING) & 1));
    }
    return;
  }
  if (warp == SY_MUL + 1) {
    // ---- |phi| warp: each landed box becomes |phi| in place; points at or past K (only in a
    // ragged last step) read as zero.  Row r holds its logical 16-byte run k4 at position k4 ^ (r & 7).
    // Lane l walks rows l, l + 32, l + 64, l + 96 of each box, a row's eight runs in turn.  With
    // pmax, a diagonal unit also keeps each row's running maximum of |phi| over the current plane i1
    // in registers (a box lies in one plane: c0 and the plane size are multiples of 32) and adds it
    // to pmax[row][i1] and gmax[row] by atomic maxima when the plane changes and at the end.
    const bool maxima = pmax != nullptr && diag;
    long long cur = -1;
    float rm[4] = {0.f, 0.f, 0.f, 0.f};
    auto flush = [&]() {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int row = bi * 128 + lane + 32 * g;
        if (row < n && cur >= 0) {
          atomicMax(reinterpret_cast<int *>(pmax) + (long long)row * n1 + cur, __float_as_int(rm[g]));
          atomicMax(reinterpret_cast<int *>(gmax) + row, __float_as_int(rm[g]));
        }
        rm[g] = 0.f;
      }
    };
    for (int q = 0; q < Q; ++q) {
      const int slot = q % SY_RING;
      if (!wait(&full[slot], q)) return;
      unsigned char *bx = boxes + (size_t)slot * 2 * kSyBox;
      const long long k0 = (s_lo + q) * BK;
      const bool ragged = k0 + BK > K;
      if (maxima) {
        const long long pl = (c0 + k0) / npl;
        if (pl != cur) {
          flush();
          cur = pl;
        }
      }
      for (int b = 0; b < nbox; ++b) {
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int row = lane + 32 * g;
          const uint32_t rbase = smem_u32(bx + (size_t)b * kSyBox) + (uint32_t)row * 128u;
          // the row's eight runs: all loads first, then the stores (logical run cl sits at position
          // cl ^ (row & 7), so lanes 8 apart share a bank group); volatile keeps the loads after the
          // wait on the landed box and in order with the stores
          uint4 v[8];
#pragma unroll
          for (int cl = 0; cl < 8; ++cl)
            asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                : "=r"(v[cl].x), "=r"(v[cl].y), "=r"(v[cl].z), "=r"(v[cl].w)
                : "r"(rbase + ((uint32_t)(cl ^ (lane & 7)) << 4)));
          float m = 0.f;
#pragma unroll
          for (int cl = 0; cl < 8; ++cl) {
            v[cl].x &= 0x7fffffffu;
            v[cl].y &= 0x7fffffffu;
            v[cl].z &= 0x7fffffffu;
            v[cl].w &= 0x7fffffffu;
            if (ragged) {
              const long long k = k0 + 4 * cl;
              if (k >= K) v[cl].x = 0u;
              if (k + 1 >= K) v[cl].y = 0u;
              if (k + 2 >= K) v[cl].z = 0u;
              if (k + 3 >= K) v[cl].w = 0u;
            }
            asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(rbase + ((uint32_t)(cl ^ (lane & 7)) << 4)),
                         "r"(v[cl].x), "r"(v[cl].y), "r"(v[cl].z), "r"(v[cl].w)
                         : "memory");
            m = fmaxf(m, fmaxf(fmaxf(__uint_as_float(v[cl].x), __uint_as_float(v[cl].y)),
                               fmaxf(__uint_as_float(v[cl].z), __uint_as_float(v[cl].w))));
          }
          if (maxima && b == 0) rm[g] = fmaxf(rm[g], m);
        }
      }
      fence_async_smem();  // these generic writes come before the TMA that refills the slot
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(&ready[slot]));
    }
    if (maxima) flush();
    return;
  }
  // ---- multiply warps: warp block (I, J); warps 8, 9 of an off-diagonal unit only release slots ----
  int I, J;
  bool computes = true;
  if (diag) {
    // (0,0) (0,1) (0,2) (0,3) (1,1) (1,2) (1,3) (2,2) (2,3) (3,3)
    I = warp < 4 ? 0 : (warp < 7 ? 1 : (warp < 9 ? 2 : 3));
    J = warp < 4 ? warp : (warp < 7 ? warp - 3 : (warp < 9 ? warp - 5 : 3));
  } else {
    I = 2 * h + ((warp >> 2) & 1);
    J = warp & 3;
    computes = warp < 8;
  }
  const int ti = lane >> 3, tj = lane & 7;
  unsigned long long part[8][4];
  float acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      part[r][c] = 0ull;
      acc[r][c] = 0.f;
    }
  // byte offsets inside a box: the thread's rows ti + 4 p + 8 s (p = rr & 1, s = rr >> 1) and
  // columns tj + 8 cc; the low three row bits (ti + 4 p, tj) pick the swizzled 16-byte position
  const uint32_t arow0 = (uint32_t)(32 * I + ti) * 128u, arow1 = arow0 + 4u * 128u;
  const uint32_t asw0 = (uint32_t)ti, asw1 = (uint32_t)(ti + 4);
  const uint32_t brow = (uint32_t)(32 * J + tj) * 128u + (diag ? 0u : kSyBox), bsw = (uint32_t)tj;
  for (int q = 0; q < Q; ++q) {
    const int slot = q % SY_RING;
    if (!wait(&ready[slot], q)) return;
    if (computes) {
      const unsigned char *bx = boxes + (size_t)slot * 2 * kSyBox;
#pragma unroll 2
      for (int k4 = 0; k4 < 8; ++k4) {
        const unsigned char *pa0 = bx + arow0 + (((uint32_t)k4 ^ asw0) << 4);
        const unsigned char *pa1 = bx + arow1 + (((uint32_t)k4 ^ asw1) << 4);
        const unsigned char *pb = bx + brow + (((uint32_t)k4 ^ bsw) << 4);
        ulonglong2 b[4], a[8];
#pragma unroll
        for (int c = 0; c < 4; ++c) b[c] = *reinterpret_cast<const ulonglong2 *>(pb + c * 1024);
#pragma unroll
        for (int r = 0; r < 8; ++r)
          a[r] = *reinterpret_cast<const ulonglong2 *>(((r & 1) ? pa1 : pa0) + (r >> 1) * 1024);
        // points (k, k + 1) of every (row, column) pair, then (k + 2, k + 3): 32 independent FMAs
        // between two updates of one accumulator
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) part[r][c] = f2fma(a[r].x, b[c].x, part[r][c]);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) part[r][c] = f2fma(a[r].y, b[c].y, part[r][c]);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&empty[slot]));
    if (computes && ((q + 1) % SY_FOLD == 0 || q + 1 == Q)) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float2 v = f2up(part[r][c]);
          acc[r][c] += v.x + v.y;
          part[r][c] = 0ull;
        }
    }
  }
  if (computes) {
    double *dst = partial + (long long)blockIdx.y * n * n;
    const int i0 = bi * 128 + 32 * I + ti, j0 = bj * 128 + 32 * J + tj;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = i0 + 4 * r;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j = j0 + 8 * c;
        if (i < n && j < n && j >= i) dst[(long long)i * n + j] = (double)acc[r][c];
      }
    }
  }
}

// O_ij += scale * sum over the splits of partial[s]_ij for i <= j (FP64, fixed order)
__global__ void screen_splits_reduce_kernel(const double *__restrict__ partial, int splits, int n, double scale,
                                            double *__restrict__ O) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n || e % n < e / n) return;
  const long long ne = (long long)n * n;
  double s = 0.0;
#pragma unroll 8
  for (int k = 0; k < splits; ++k) s += partial[(long long)k * ne + e];
  O[e] += scale * s;
}

}  // namespace tc

bool tc_shapes_ok(long long K) { return K % tc::BN == 0 && K % tc::BK == 0; }
bool tc_gram_shape_ok(long long K) { return K % tc::BK == 0; }

// FP32 accumulation length of the tensor-core Gram (a multiple of 32; ACE_TC_CHUNK overrides)
static int tc_chunk() {
  static int c = [] {
    const char *v = std::getenv("ACE_TC_CHUNK");
    int x = (v && *v) ? std::atoi(v) : tc::kGramChunkDefault;
    if (x < tc::BK) x = tc::BK;
    return (x / tc::BK) * tc::BK;
  }();
  return c;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link against libcuda)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// 2D map of a row-major FP32 matrix [rows][cols] with boxes of box_rows x box_cols; false when
// the encoder is unavailable or refuses the layout (base 16-byte aligned, cols % 4 == 0)
static bool make_map_f32(CUtensorMap *map, const float *ptr, long long rows, long long cols, int box_rows,
                         int box_cols, bool swizzle128, long long ld = 0) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (ld == 0) ld = cols;  // row stride in elements
  if (!enc || (reinterpret_cast<uintptr_t>(ptr) & 15) || (cols & 3) || (ld & 3) || ld < cols) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool use_tma() {
  static const bool on = [] {
    const char *v = std::getenv("ACE_NO_TMA");
    return !(v && *v && *v != '0');
  }();
  return on;
}

// Chunk-partial Gram (each CTA one chunk, FP32 partials, two-level FP64 reduction): the path
// for operands the TMA Gram cannot map.
static cudaError_t launch_tc_gram_chunks(const float *X, int nx, const float *Y, int ny, long long K, double scale,
                                        double *G, float *partial_ws, int *err, cudaStream_t st) {
  const int tx = (nx + tc::BM - 1) / tc::BM, ty = (ny + tc::BN - 1) / tc::BN;
  const int chunk = tc_chunk();
  const long long chunks = (K + chunk - 1) / chunk;
  if (K % tc::BK != 0 || chunks > 65535) return cudaErrorInvalidValue;
  const int smem = (int)tc::SmemLayout::kBytes;
  cudaError_t e = cudaFuncSetAttribute(tc::tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  tc::tc_gram_kernel<<<dim3(tx * ty, (unsigned)chunks), tc::NT, smem, st>>>(X, nx, Y, ny, K, chunk, tx, partial_ws,
                                                                             err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n = nx * ny;
  const size_t part2_off = ((sizeof(float) * (size_t)chunks * n + 255) / 256) * 256;  // aligned, after the partials
  double *part2 = reinterpret_cast<double *>(reinterpret_cast<char *>(partial_ws) + part2_off);
  tc::gram_reduce_kernel<<<dim3((n + 255) / 256, tc::kReduceGroups), 256, 0, st>>>(partial_ws, (int)chunks, n,
                                                                                   part2);
  tc::gram_reduce2_kernel<<<(n + 255) / 256, 256, 0, st>>>(part2, n, scale, G);
  return cudaGetLastError();
}

static size_t gram_chunks_workspace_bytes(int nx, int ny, long long K) {
  const long long chunks = (K + tc_chunk() - 1) / tc_chunk();
  // FP32 chunk partials, then (256-byte aligned) the FP64 group sums of the reduction
  const size_t part2_off = ((sizeof(float) * (size_t)chunks * nx * ny + 255) / 256) * 256;
  return part2_off + sizeof(double) * tc::kReduceGroups * (size_t)nx * ny;
}

// TMA Gram plan: splits of the K range (whole chunks) and ring depth; false when TMA cannot be
// used for these operands (disabled, encoder missing, misaligned base, K not a multiple of 32).
struct GramPlan {
  int splits, ring, nops, tiles_x, tiles;
};
static bool gram_tma_plan(const float *X, int nx, const float *Y, int ny, long long K, GramPlan *p) {
  if (!use_tma() || !tensor_map_encoder() || (reinterpret_cast<uintptr_t>(X) & 15) ||
      (reinterpret_cast<uintptr_t>(Y) & 15) || K % tc::BK != 0 || K / tc::BK > (1LL << 30))
    return false;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  p->tiles_x = (nx + tc::BM - 1) / tc::BM;
  p->tiles = p->tiles_x * ((ny + tc::BN - 1) / tc::BN);
  const int cs = tc_chunk() / tc::BK;
  const long long chunks = (K / tc::BK + cs - 1) / cs;
  p->splits = (int)std::max(1LL, std::min(chunks, (long long)std::max(1, sms / p->tiles)));
  // three operand buffers, the rest of shared memory for box stages (4); measured at 96^3, the
  // split of 2-4 buffers and 2-5 stages changes nothing
  p->nops = tc::GW_OPS;
  const size_t fixed = (size_t)p->nops * 4 * tc::TILE_BYTES + 1024 + 256;
  p->ring = (int)std::min<size_t>(4, (227 * 1024 - fixed) / (2 * tc::kGBox));
  return p->ring >= 2;
}

size_t tc_gram_workspace_bytes(const float *X, int nx, const float *Y, int ny, long long K) {
  GramPlan p;
  if (gram_tma_plan(X, nx, Y, ny, K, &p)) return sizeof(double) * (size_t)p.splits * nx * ny;
  return gram_chunks_workspace_bytes(nx, ny, K);
}

// The TMA Gram over the columns [c0, c0 + K) of X and Y (rows of ld elements): G = scale X Y^T,
// or G += scale |X| |Y|^T with ABS; false (nothing launched) when the plan or the maps fail.
template <bool ABS>
static bool launch_gram_tma(const float *X, int nx, const float *Y, int ny, long long ld, long long c0, long long K,
                            double scale, double *G, void *ws, int *err, cudaStream_t st, long *launches,
                            cudaError_t *e) {
  GramPlan p;
  CUtensorMap mx, my;
  if (c0 % 4 != 0 || !gram_tma_plan(X, nx, Y, ny, K, &p) || !make_map_f32(&mx, X, nx, ld, tc::BM, tc::BK, true) ||
      !make_map_f32(&my, Y, ny, ld, tc::BN, tc::BK, true))
    return false;
  const int smem = (int)((size_t)p.nops * 4 * tc::TILE_BYTES + (size_t)p.ring * 2 * tc::kGBox + 1024 + 256);
  *e = cudaFuncSetAttribute(tc::tc_gram_tma_kernel<ABS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (*e != cudaSuccess) return true;
  double *partial = static_cast<double *>(ws);
  // ACE_TC_FIRST_WAIT_POLLS: polls of the kernel's first wait on a TMA box (test knob; 0 makes
  // the kernel give up at once and report ACE_ERR_TIMEOUT after draining its copies)
  const char *fw = std::getenv("ACE_TC_FIRST_WAIT_POLLS");
  const uint32_t first_wait = (fw && *fw) ? (uint32_t)std::strtoul(fw, nullptr, 10) : tc::kWaitLimit;
  tc::tc_gram_tma_kernel<ABS><<<dim3(p.tiles, p.splits), tc::GW_NT, smem, st>>>(
      mx, my, nx, ny, c0, K, tc_chunk() / tc::BK, p.tiles_x, p.ring, p.nops, partial, err, first_wait);
  *e = cudaGetLastError();
  if (*e != cudaSuccess) return true;
  const int n = nx * ny;
  // 64-thread blocks spread the FP64 adds (splits x n elements) over most SMs
  tc::gram_splits_reduce_kernel<<<(n + 63) / 64, 64, 0, st>>>(partial, p.splits, n, scale, ABS, G);
  *launches += 2;
  *e = cudaGetLastError();
  return true;
}

cudaError_t launch_tc_gram(const float *X, int nx, const float *Y, int ny, long long K, double scale, double *G,
                           void *ws, int *err, cudaStream_t st, long *launches) {
  cudaError_t e = cudaSuccess;
  if (launch_gram_tma<false>(X, nx, Y, ny, K, 0, K, scale, G, ws, err, st, launches, &e)) return e;
  *launches += 3;
  return launch_tc_gram_chunks(X, nx, Y, ny, K, scale, G, static_cast<float *>(ws), err, st);
}

size_t tc_screen_workspace_bytes(const float *X, int n, long long K) {
  GramPlan p;
  return gram_tma_plan(X, n, X, n, K, &p) ? sizeof(double) * (size_t)p.splits * n * n : 0;
}

bool launch_tc_screen(const float *X, int n, long long ld, long long c0, long long K, double scale, double *G,
                      void *ws, int *err, cudaStream_t st, long *launches, cudaError_t *e) {
  return launch_gram_tma<true>(X, n, X, n, ld, c0, K, scale, G, ws, err, st, launches, e);
}

// Screen contribution of the columns [c0, c0 + K) of phi (n rows of ld points) through TMA; false
// (nothing launched) when TMA cannot map phi or the columns are not whole 32-point steps.
bool launch_screen_tma(const float *X, int n, long long ld, long long c0, long long K, double scale, double *G,
                       int *err, cudaStream_t st) {
  if (!use_tma() || K % tc::BK != 0 || c0 % 4 != 0) return false;
  CUtensorMap map;
  if (!make_map_f32(&map, X, n, ld, tc::SC_B, tc::BK, true)) return false;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int nb = (n + tc::SC_B - 1) / tc::SC_B, tiles = nb * (nb + 1) / 2;
  const long long ks = K / tc::BK;
  const int splits = (int)std::max(1LL, std::min(ks, (long long)std::max(1, 2 * sms / tiles)));
  const int ring = 4;
  const size_t smem = (size_t)ring * 2 * tc::kSBox + sizeof(float2) * tc::BK * (tc::SC_B + 2) +
                      sizeof(float) * tc::BK * (tc::SC_B + 4) + 1024 + 128;
  if (cudaFuncSetAttribute(tc::screen_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  tc::screen_tma_kernel<<<dim3(tiles, splits), tc::NT2, smem, st>>>(map, n, c0, K, scale, ring, G, err);
  return true;
}

// Plan of the CUDA-core screen: work units (diagonal block pairs, then two per off-diagonal
// pair) and K-splits so that units x splits fill the SMs once.
static void screen_syrk_plan(int n, long long K, int *ndiag, int *units, int *splits) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  *ndiag = (n + 127) / 128;
  *units = *ndiag + (*ndiag) * (*ndiag - 1);
  const long long ks = std::max(1LL, (K + tc::BK - 1) / tc::BK);
  *splits = (int)std::max(1LL, std::min(ks, (long long)std::max(1, sms / *units)));
}

size_t screen_syrk_workspace_bytes(int n, long long K) {
  int nd, un, sp;
  screen_syrk_plan(n, K, &nd, &un, &sp);
  return sizeof(double) * (size_t)sp * n * n;
}

bool launch_screen_syrk(const float *X, int n, long long ld, long long c0, long long K, double scale, double *G,
                        void *ws, int *err, cudaStream_t st, long *launches, cudaError_t *e, const PlaneMaxOut *pm) {
  if (!use_tma() || c0 % 4 != 0 || K <= 0 || !ws) return false;
  CUtensorMap map;
  if (!make_map_f32(&map, X, n, ld, 128, tc::BK, true)) return false;
  int ndiag, units, splits;
  screen_syrk_plan(n, K, &ndiag, &units, &splits);
  // the shared-memory limit is a per-device attribute of the kernel: set once per device
  static unsigned long long attr_done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(__atomic_load_n(&attr_done, __ATOMIC_ACQUIRE) & bit)) {
    *e = cudaFuncSetAttribute(tc::screen_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::kSySmem);
    if (*e != cudaSuccess) return true;
    __atomic_fetch_or(&attr_done, bit, __ATOMIC_RELEASE);
  }
  double *partial = static_cast<double *>(ws);
  // plane maxima along the way when every box lies in one plane
  const bool with_max = pm && pm->pmax && pm->npl % tc::BK == 0 && c0 % tc::BK == 0;
  tc::screen_syrk_kernel<<<dim3(units, splits), tc::SY_NT, tc::kSySmem, st>>>(
      map, n, c0, K, ndiag, partial, err, with_max ? pm->pmax : nullptr, with_max ? pm->gmax : nullptr,
      with_max ? pm->npl : 1, with_max ? pm->n1 : 1);
  if (pm && pm->done) *pm->done = *pm->done && with_max;
  *e = cudaGetLastError();
  if (*e != cudaSuccess) return true;
  tc::screen_splits_reduce_kernel<<<(n * n + 63) / 64, 64, 0, st>>>(partial, splits, n, scale, G);
  *launches += 2;
  *e = cudaGetLastError();
  return true;
}

cudaError_t launch_tc_left_mul(const float *A, int m, int n, const float *Y, long long K, float *Z, int *err,
                               cudaStream_t st) {
  if (K % 4 != 0) return cudaErrorNotSupported;
  if (use_tma()) {
    const int nsteps = (n + tc::BK - 1) / tc::BK;
    const size_t fixed = ((size_t)nsteps * 2 + 4) * tc::TILE_BYTES + 2 * tc::kEpiBox + 1024 + 256;
    const size_t cap = 227 * 1024;
    const int ring = fixed + 2 * tc::kLmBox <= cap ? (int)std::min<size_t>(8, (cap - fixed) / tc::kLmBox) : 0;
    CUtensorMap map, zmap;
    if (ring >= 2 && make_map_f32(&map, Y, n, K, tc::BK, tc::BN, false) &&
        make_map_f32(&zmap, Z, m, K, tc::BM, 32, true)) {
      const int smem = (int)(fixed + (size_t)ring * tc::kLmBox);
      cudaError_t e =
          cudaFuncSetAttribute(tc::tc_left_mul_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      int dev = 0, sms = 152;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const long long tiles = (K + tc::BN - 1) / tc::BN;
      const int rows = (m + tc::BM - 1) / tc::BM;
      const unsigned gx = (unsigned)std::max(1LL, std::min(tiles, (long long)std::max(1, sms / rows)));
      tc::tc_left_mul_tma_kernel<<<dim3(gx, rows), tc::NT2, smem, st>>>(A, m, n, map, zmap, K, ring, err);
      return cudaGetLastError();
    }
  }
  if (K % tc::BN != 0) return cudaErrorNotSupported;  // the register-staged kernel stores whole tiles
  const int nsteps = (n + tc::BK - 1) / tc::BK;
  const int smem = (int)(((size_t)nsteps * 2 + 4) * tc::TILE_BYTES + 2048);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(tc::tc_left_mul_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = K / tc::BN;
  const int rows = (m + tc::BM - 1) / tc::BM;
  const int per_sm = smem <= 110 * 1024 ? 2 : 1;
  const long long want = (long long)sms * per_sm / rows;
  const unsigned gx = (unsigned)std::max(1LL, std::min(tiles, want));
  tc::tc_left_mul_kernel<<<dim3(gx, rows), tc::NT, smem, st>>>(A, m, n, Y, K, Z, err);
  return cudaGetLastError();
}

}  // namespace ace
