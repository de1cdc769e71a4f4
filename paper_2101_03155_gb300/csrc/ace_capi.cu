// ace_capi.cu -- the C ABI declared in include/ace.h: argument checks, host-made tables, device
// workspaces and the order of the build steps (screen, pair chain, M, Cholesky, xi) and of the
// ACE application.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/ace.h"
#include "ace_internal.h"
#include "fft.cuh"

using ace::cpx;

namespace {

thread_local std::string g_last_error;

ace_status fail(ace_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

ace_status cuda_fail(cudaError_t e, const char *what) {
  if (e == cudaErrorMemoryAllocation) return fail(ACE_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(ACE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define ACE_CUDA(call, what)                 \
  do {                                       \
    cudaError_t _e = (call);                 \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

// Keep freed stream-ordered allocations cached in the device's default pool (once per device).
std::mutex g_pool_mu;
std::vector<int> g_pool_ready;

cudaError_t prepare_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (std::find(g_pool_ready.begin(), g_pool_ready.end(), dev) != g_pool_ready.end()) return cudaSuccess;
  cudaMemPool_t pool;
  cudaError_t e = cudaDeviceGetDefaultMemPool(&pool, dev);
  if (e != cudaSuccess) return e;
  unsigned long long thr = ~0ull;
  e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  if (e != cudaSuccess) return e;
  g_pool_ready.push_back(dev);
  return cudaSuccess;
}

bool is_device_pointer(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Reciprocal basis b_k = 2 pi (row k of A^-T) of the lattice rows A.
void reciprocal_basis(const ace_desc &d, double B[3][3]) {
  const double *A = &d.lattice[0][0];
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  // row k of A^-T = column k of A^-1; A^-1 = adj(A) / det
  const double adj[9] = {A[4] * A[8] - A[5] * A[7], A[2] * A[7] - A[1] * A[8], A[1] * A[5] - A[2] * A[4],
                         A[5] * A[6] - A[3] * A[8], A[0] * A[8] - A[2] * A[6], A[2] * A[3] - A[0] * A[5],
                         A[3] * A[7] - A[4] * A[6], A[1] * A[6] - A[0] * A[7], A[0] * A[4] - A[1] * A[3]};
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) B[k][c] = 2.0 * ace::kPi * adj[c * 3 + k] / det;
}

// Cut-off radius of the truncated kernel: r_cut, or when r_cut <= 0 the radius of the largest
// sphere inside the cell (half the smallest distance between lattice planes, min_k pi / |b_k|).
double cutoff_radius(const ace_desc &d) {
  if (d.r_cut > 0.0) return d.r_cut;
  double B[3][3];
  reciprocal_basis(d, B);
  double r = HUGE_VAL;
  for (int k = 0; k < 3; ++k)
    r = std::min(r, ace::kPi / std::sqrt(B[k][0] * B[k][0] + B[k][1] * B[k][1] + B[k][2] * B[k][2]));
  return r;
}

// Kernel table on the FFT box, divided by N (the 1/N of the forward transform), mean over the
// +-N_k/2 choices at Nyquist indices:
//   ACE_COULOMB_PERIODIC  4 pi / |G|^2, G = 0 -> 0 (Eq. e:vij in reciprocal space);
//   ACE_COULOMB_TRUNCATED 4 pi (1 - cos(|G| rc)) / |G|^2 (the interaction 1/r for r < rc), whose
//                         G = 0 limit 2 pi rc^2 is kept.
void coulomb_table(const ace_desc &d, std::vector<double> &K) {
  const int n1 = d.n[0], n2 = d.n[1], n3 = d.n[2];
  double B[3][3];
  reciprocal_basis(d, B);
  const bool trunc = d.coulomb == ACE_COULOMB_TRUNCATED;
  const double rc = trunc ? cutoff_radius(d) : 0.0;
  // Gram matrix of the reciprocal basis: |G|^2 = sum_kl m_k m_l (b_k . b_l)
  double g[3][3];
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) g[k][l] = B[k][0] * B[l][0] + B[k][1] * B[l][1] + B[k][2] * B[l][2];
  const long long N = (long long)n1 * n2 * n3;
  K.assign((size_t)N, 0.0);
  const int nn[3] = {n1, n2, n3};
  const double fourpi_over_N = 4.0 * ace::kPi / (double)N;
  for (int i1 = 0; i1 < n1; ++i1)
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i3 = 0; i3 < n3; ++i3) {
        const int idx[3] = {i1, i2, i3};
        int m[3];
        bool nyq[3];
        for (int k = 0; k < 3; ++k) {
          m[k] = (2 * idx[k] < nn[k]) ? idx[k] : idx[k] - nn[k];
          nyq[k] = (nn[k] % 2 == 0) && (2 * idx[k] == nn[k]);
        }
        const long long lin = ((long long)i1 * n2 + i2) * n3 + i3;
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) {
          if (trunc) K[(size_t)lin] = fourpi_over_N * 0.5 * rc * rc;
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
            for (int l = 0; l < 3; ++l) q += mm[k] * mm[l] * g[k][l];
          acc += trunc ? (1.0 - std::cos(std::sqrt(q) * rc)) / q : 1.0 / q;
          ++cnt;
        }
        K[(size_t)lin] = fourpi_over_N * acc / cnt;
      }
}


// Device copies of the Coulomb kernel table and the per-axis twiddles, made once per
// (device, grid, lattice, precision) and kept until the process exits.
struct DeviceTables {
  int dev;
  int n[3];
  double lattice[9];
  int coulomb;
  double rc;
  size_t esz;
  void *K;
  void *Kperm;  // K[m1][k2(p2)][k3(p3)]: axes 2 and 3 in the plane passes' output positions
  void *tw[3];
};
std::mutex g_tab_mu;
std::deque<DeviceTables> g_tables;  // deque: references stay valid on push_back

template <typename T>
cudaError_t get_tables(int dev, const ace_desc &d, cudaStream_t st, const DeviceTables **out) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  for (const DeviceTables &t : g_tables) {
    if (t.dev == dev && t.esz == sizeof(T) && t.n[0] == d.n[0] && t.n[1] == d.n[1] && t.n[2] == d.n[2] &&
        std::memcmp(t.lattice, &d.lattice[0][0], sizeof(t.lattice)) == 0 && t.coulomb == (int)d.coulomb &&
        (d.coulomb != ACE_COULOMB_TRUNCATED || t.rc == cutoff_radius(d))) {
      *out = &t;
      return cudaSuccess;
    }
  }
  DeviceTables t{};
  t.dev = dev;
  t.esz = sizeof(T);
  for (int k = 0; k < 3; ++k) t.n[k] = d.n[k];
  std::memcpy(t.lattice, &d.lattice[0][0], sizeof(t.lattice));
  t.coulomb = (int)d.coulomb;
  t.rc = d.coulomb == ACE_COULOMB_TRUNCATED ? cutoff_radius(d) : 0.0;
  std::vector<double> Kh;
  coulomb_table(d, Kh);
  std::vector<T> Kt(Kh.begin(), Kh.end());
  cudaError_t e = cudaMalloc(&t.K, sizeof(T) * Kt.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(t.K, Kt.data(), sizeof(T) * Kt.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  std::vector<T> Kp(Kt.size());
  {
    int a2, b2, a3, b3;
    ace::axis_factors(d.n[1], &a2, &b2);
    ace::axis_factors(d.n[2], &a3, &b3);
    const int n2 = d.n[1], n3 = d.n[2];
    for (int m1 = 0; m1 < d.n[0]; ++m1)
      for (int p2 = 0; p2 < n2; ++p2) {
        const int k2 = p2 / b2 + a2 * (p2 % b2);
        for (int p3 = 0; p3 < n3; ++p3) {
          const int k3 = p3 / b3 + a3 * (p3 % b3);
          Kp[((size_t)m1 * n2 + p2) * n3 + p3] = Kt[((size_t)m1 * n2 + k2) * n3 + k3];
        }
      }
  }
  e = cudaMalloc(&t.Kperm, sizeof(T) * Kp.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(t.Kperm, Kp.data(), sizeof(T) * Kp.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  std::vector<cpx<T>> twh[3];
  for (int a = 0; a < 3; ++a) {
    const int L = d.n[a];
    twh[a].resize(L);
    for (int k = 0; k < L; ++k) {
      const double ang = 2.0 * ace::kPi * (double)k / (double)L;
      twh[a][k] = cpx<T>{(T)std::cos(ang), (T)(-std::sin(ang))};
    }
    e = cudaMalloc(&t.tw[a], sizeof(cpx<T>) * L);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(t.tw[a], twh[a].data(), sizeof(cpx<T>) * L, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  e = cudaStreamSynchronize(st);  // host vectors must outlive the copies
  if (e != cudaSuccess) return e;
  g_tables.push_back(t);
  *out = &g_tables.back();
  return cudaSuccess;
}

}  // namespace

struct ace_op {
  int dev = 0;
  cudaStream_t stream = nullptr;
  ace_desc desc{};
  int n = 0;
  long long N = 0;
  double dV = 0.0;
  bool fp64 = false;
  size_t esz = 4;
  void *W = nullptr, *xi = nullptr;
  double *O = nullptr, *O_sym = nullptr, *M_raw = nullptr, *M = nullptr, *L = nullptr, *Linv = nullptr;
  double *energy_d = nullptr;
  int *status_d = nullptr, *count_d = nullptr;
  int *tc_err = nullptr;  // set by a tensor-core kernel whose bounded wait gave up
  int2 *pairs = nullptr;
  int4 *packs = nullptr;
  long npairs = 0;
  double energy = 0.0;
  int status = 0;
  cudaEvent_t ev[6] = {};
  float stage_ms[6] = {};
  long launches = 0;          // kernels of this library launched by the build
  std::vector<void *> owned;  // stream-ordered allocations freed by ace_destroy
  std::vector<int2> pairs_h;  // host copy of the kept pairs
  std::vector<int2> given;    // ace_build_pairs: the caller's pair list (sorted, unique); skips the screen
  bool use_given = false;
  std::vector<void *> temps;  // build workspaces released in stream order at the end of the build
  const void *phi_work = nullptr;
  const DeviceTables *tab = nullptr;
  void *readback = nullptr;   // pinned host area for the asynchronous readbacks of a build
  size_t readback_bytes = 0;
  int lane = 0;               // stream lane of a batched build (selects its side streams)
  cudaStream_t tail = nullptr;  // batched builds: stream of the steps after the pair chain
  float *pmax = nullptr;      // plane maxima of the working orbitals [n][N1] for the plane skip
  float *gmax = nullptr;      // and the orbitals' maxima [n]
  bool queued = false;        // screened build whose chain ran in a device pack queue
  bool graph = false;         // recorded into a CUDA graph: no host waits, no timing events,
                              // uploads from pinned buffers that live as long as the handle
  std::vector<std::pair<void *, size_t>> staged;  // those pinned upload buffers
};

namespace {

// Buffers the handle owns (results and pair lists).  A handle recorded into a graph takes them
// from cudaMalloc, outside the graph, so that they keep their addresses over every launch.
template <typename P>
cudaError_t op_alloc(ace_op *op, P **p, size_t bytes) {
  void *v = nullptr;
  cudaError_t e = op->graph ? cudaMalloc(&v, bytes > 0 ? bytes : 16)
                            : cudaMallocAsync(&v, bytes > 0 ? bytes : 16, op->stream);
  if (e != cudaSuccess) return e;
  op->owned.push_back(v);
  *p = static_cast<P *>(v);
  return cudaSuccess;
}

void op_free_all(ace_op *op) {
  for (void *p : op->owned) op->graph ? cudaFree(p) : cudaFreeAsync(p, op->stream);
  op->owned.clear();
}

void destroy_op(ace_op *op);

// Host-to-device copy of a host temporary: directly (the call returns once the pageable source
// has been read) or, when the op is recorded into a graph, through a pinned buffer kept with the
// handle, since the graph reads its source again at every launch.
cudaError_t host_upload(ace_op *op, void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if (!op->graph) return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
  void *pin = nullptr;
  cudaError_t e = cudaHostAlloc(&pin, bytes, cudaHostAllocDefault);
  if (e != cudaSuccess) return e;
  std::memcpy(pin, src, bytes);
  op->staged.emplace_back(pin, bytes);
  return cudaMemcpyAsync(dst, pin, bytes, cudaMemcpyHostToDevice, st);
}

// Default plane-skip fraction of the mixed form (see plane_skip_rel).
constexpr float kPlaneSkipDefault = 1e-7f;

// Fraction of an orbital's maximum below which its planes count as negligible for the plane skip of
// the mixed form's chain (ACE_PLANE_SKIP; 0 turns the skip off).  The FP64 form never skips.
float plane_skip_rel(bool fp64) {
  if (fp64) return 0.f;
  const char *v = std::getenv("ACE_PLANE_SKIP");
  const float r = (v && *v) ? (float)std::atof(v) : kPlaneSkipDefault;
  return r > 0.f ? r : 0.f;
}

// The plane-maxima table of the op's working orbitals (computed once per build, on st).
cudaError_t plane_max_table(ace_op *op, const float *phi, cudaStream_t st) {
  if (op->pmax) return cudaSuccess;
  cudaError_t e = op_alloc(op, &op->pmax, sizeof(float) * (size_t)op->n * op->desc.n[0]);
  if (e == cudaSuccess) e = op_alloc(op, &op->gmax, sizeof(float) * (size_t)op->n);
  if (e == cudaSuccess) e = cudaMemsetAsync(op->gmax, 0, sizeof(float) * (size_t)op->n, st);
  if (e == cudaSuccess)
    e = ace::launch_plane_max(phi, op->n, op->desc.n[0], (long long)op->desc.n[1] * op->desc.n[2], op->pmax, op->gmax,
                              st);
  if (e == cudaSuccess) ++op->launches;
  return e;
}

// Stage-timing event i of a build (not recorded inside a graph)
cudaError_t mark(ace_op *op, int i, cudaStream_t st) {
  return op->graph ? cudaSuccess : cudaEventRecord(op->ev[i], st);
}

ace_status check_desc(const ace_desc *d) {
  if (!d) return fail(ACE_ERR_ARG, "desc is NULL");
  if (d->norb < 1 || d->norb > 1024) return fail(ACE_ERR_ARG, "norb = %d outside [1, 1024]", d->norb);
  for (int k = 0; k < 3; ++k)
    if (d->n[k] < 1) return fail(ACE_ERR_ARG, "grid axis %d has length %d", k, d->n[k]);
  for (int k = 0; k < 3; ++k)
    if (!ace::pass_length_supported(d->n[k]))
      return fail(ACE_ERR_UNSUPPORTED_GRID, "grid axis %d length %d has no compiled FFT plan", k, d->n[k]);
  const double *A = &d->lattice[0][0];
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(A[i])) return fail(ACE_ERR_ARG, "lattice has a non-finite entry");
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  if (!(std::fabs(det) > 0.0)) return fail(ACE_ERR_ARG, "lattice is singular");
  if (d->prec != ACE_FP64 && d->prec != ACE_MIXED) return fail(ACE_ERR_ARG, "unknown precision %d", (int)d->prec);
  if (!std::isfinite(d->spin_factor) || !std::isfinite(d->rho_cut)) return fail(ACE_ERR_ARG, "non-finite scalar");
  if (d->coulomb != ACE_COULOMB_PERIODIC && d->coulomb != ACE_COULOMB_TRUNCATED)
    return fail(ACE_ERR_ARG, "unknown Coulomb kernel %d", (int)d->coulomb);
  if (d->coulomb == ACE_COULOMB_TRUNCATED && !std::isfinite(d->r_cut)) return fail(ACE_ERR_ARG, "non-finite r_cut");
  return ACE_OK;
}

int env_int(const char *name, int dflt) {
  const char *v = std::getenv(name);
  if (!v || !*v) return dflt;
  return std::atoi(v);
}

// Bring `src` (host or device, dtype `dt`) to a device array of T; returns the device pointer
// (either src itself or an op-owned or caller-supplied staging copy).
template <typename T>
ace_status stage_input(ace_op *op, const void *src, ace_dtype dt, long long count, const T **out,
                       std::vector<void *> *temps) {
  // a conversion kernel (if any) is counted in op->launches
  const bool dev = is_device_pointer(src);
  const bool same = (dt == ACE_F64) == (sizeof(T) == 8);
  const size_t in_bytes = (size_t)count * (dt == ACE_F64 ? 8 : 4);
  const void *d_in = src;
  // host memory, and device memory off a 16-byte boundary when no conversion follows (the
  // kernels read operands in 16-byte vectors and by TMA), go through an aligned device copy
  const bool misaligned = (reinterpret_cast<uintptr_t>(src) & 15) != 0;
  if (!dev || (same && misaligned)) {
    void *tmp = nullptr;
    ACE_CUDA(cudaMallocAsync(&tmp, in_bytes, op->stream), "staging allocation");
    temps->push_back(tmp);
    ACE_CUDA(cudaMemcpyAsync(tmp, src, in_bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, op->stream),
             "staging copy");
    d_in = tmp;
  }
  if (same) {
    *out = static_cast<const T *>(d_in);
    return ACE_OK;
  }
  void *conv = nullptr;
  ACE_CUDA(cudaMallocAsync(&conv, (size_t)count * sizeof(T), op->stream), "conversion allocation");
  temps->push_back(conv);
  if (dt == ACE_F64)
    ACE_CUDA((ace::launch_convert<double, T>(static_cast<const double *>(d_in), static_cast<T *>(conv), count, 1.0,
                                             op->stream)),
             "convert");
  else
    ACE_CUDA((ace::launch_convert<float, T>(static_cast<const float *>(d_in), static_cast<T *>(conv), count, 1.0,
                                            op->stream)),
             "convert");
  ++op->launches;
  *out = static_cast<const T *>(conv);
  return ACE_OK;
}

// Small pinned host buffers for the asynchronous readbacks of builds, reused across builds.
std::mutex g_pin_mu;
std::vector<std::pair<size_t, void *>> g_pinned;

cudaError_t pinned_get(size_t bytes, void **out) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pinned.size(); ++i)
      if (g_pinned[i].first >= bytes) {
        *out = g_pinned[i].second;
        g_pinned.erase(g_pinned.begin() + i);
        return cudaSuccess;
      }
  }
  return cudaHostAlloc(out, bytes < 4096 ? 4096 : bytes, cudaHostAllocDefault);
}

void pinned_put(void *p, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  if (g_pinned.size() < 64) {
    g_pinned.emplace_back(bytes < 4096 ? 4096 : bytes, p);
  } else {
    cudaFreeHost(p);
  }
}

// Per-device side streams of the pair chain (created once, non-blocking, kept until exit).
std::mutex g_side_mu;
constexpr int kLanes = 4;           // concurrent builds of one batched call
constexpr int kSide = 8;            // pair-chain side streams per lane
// per lane: kSide chain side streams; then the lane streams; then one input-copy stream per lane;
// then one tail stream per lane (the steps after the pair chain of a batched build)
cudaStream_t g_side[64][(kSide + 3) * kLanes] = {};

cudaError_t get_side_stream(int dev, int k, cudaStream_t *out) {
  if (dev < 0 || dev >= 64 || k < 0 || k >= (kSide + 3) * kLanes) return cudaErrorInvalidValue;
  std::lock_guard<std::mutex> lk(g_side_mu);
  if (!g_side[dev][k]) {
    cudaError_t e = cudaStreamCreateWithFlags(&g_side[dev][k], cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  *out = g_side[dev][k];
  return cudaSuccess;
}

template <typename T>
bool find_persist_ops(int n1, int n2, int n3, ace::PersistOps<T> *out);
template <>
bool find_persist_ops<float>(int n1, int n2, int n3, ace::PersistOps<float> *out) {
  return ace::persist_ops_f32_small(n1, n2, n3, out) || ace::persist_ops_f32_large(n1, n2, n3, out);
}
template <>
bool find_persist_ops<double>(int, int, int, ace::PersistOps<double> *) {
  return false;
}

template <typename T>
bool find_plane_ops(int n2, int n3, ace::PlaneOps<T> *out);
template <>
bool find_plane_ops<float>(int n2, int n3, ace::PlaneOps<float> *out) {
  return ace::plane_ops_f32_small(n2, n3, out) || ace::plane_ops_f32_large(n2, n3, out);
}
template <>
bool find_plane_ops<double>(int n2, int n3, ace::PlaneOps<double> *out) {
  return ace::plane_ops_f64(n2, n3, out);
}

// Run-time parameters of the plane chain: packs per CTA group (G), packs per batch (B), side
// streams, and the L2 set-aside for the scratch window (MB).  Defaults, or values found by
// ace_autotune for the grid and precision; ACE_* environment variables override both.
struct ChainParams {
  int G = 1, B = 2, streams = 4, persist_mb = 60;
  int RB = 4;          // rows per block of the pack order
  int persistent = 0;  // 1: the persistent chain (one launch, device task queue)
  int lag = 3;         // its queue lag (rounds between the stages of one pack)
  int conv = 0;        // pencil tile of the axis-1 pass (PairPassArgs::conv_tile)
};

struct TuneKey {
  int n1, n2, n3, fp64;
  bool operator==(const TuneKey &o) const {
    return n1 == o.n1 && n2 == o.n2 && n3 == o.n3 && fp64 == o.fp64;
  }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, ChainParams>> g_tuned;
bool g_tune_file_read = false;

void tune_file_load_locked() {
  if (g_tune_file_read) return;
  g_tune_file_read = true;
  const char *path = std::getenv("ACE_TUNE_FILE");
  if (!path || !*path) return;
  FILE *f = std::fopen(path, "r");
  if (!f) return;
  // one line per grid; the twelfth field (pencil tile) may be absent (files of eleven fields)
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    TuneKey k;
    ChainParams c;
    const int got = std::sscanf(line, "%d %d %d %d %d %d %d %d %d %d %d %d", &k.n1, &k.n2, &k.n3, &k.fp64, &c.G, &c.B,
                                &c.streams, &c.persist_mb, &c.RB, &c.persistent, &c.lag, &c.conv);
    if (got < 11) continue;
    if (got == 11) c.conv = 0;
    g_tuned.emplace_back(k, c);
  }
  std::fclose(f);
}

void tune_store(const TuneKey &k, const ChainParams &c) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_file_load_locked();
  bool found = false;
  for (auto &e : g_tuned)
    if (e.first == k) {
      e.second = c;
      found = true;
    }
  if (!found) g_tuned.emplace_back(k, c);
  const char *path = std::getenv("ACE_TUNE_FILE");
  if (path && *path) {
    FILE *f = std::fopen(path, "w");
    if (f) {
      for (const auto &e : g_tuned)
        std::fprintf(f, "%d %d %d %d %d %d %d %d %d %d %d %d\n", e.first.n1, e.first.n2, e.first.n3, e.first.fp64,
                     e.second.G, e.second.B, e.second.streams, e.second.persist_mb, e.second.RB, e.second.persistent,
                     e.second.lag, e.second.conv);
      std::fclose(f);
    }
  }
}

ChainParams chain_params(const ace_desc &d, bool fp64) {
  ChainParams c;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_file_load_locked();
    const TuneKey k{d.n[0], d.n[1], d.n[2], fp64 ? 1 : 0};
    for (const auto &e : g_tuned)
      if (e.first == k) c = e.second;
  }
  c.G = std::max(1, env_int("ACE_GROUP", c.G));
  c.B = std::max(c.G, env_int("ACE_PLANE_BATCH", c.B));
  c.streams = std::min(kSide, std::max(1, env_int("ACE_STREAMS", c.streams)));
  c.persist_mb = std::max(0, env_int("ACE_L2_PERSIST_MB", c.persist_mb));
  c.RB = std::max(1, env_int("ACE_ROW_BLOCK", c.RB));
  c.persistent = env_int("ACE_PERSISTENT", c.persistent) != 0;
  c.lag = std::max(1, env_int("ACE_PERSIST_LAG", c.lag));
  c.conv = std::min(2, std::max(0, env_int("ACE_CONV_TILE", c.conv)));
  if (fp64) c.conv = 0;
  return c;
}

// Five pencil passes per batch of packs (any compiled grid).
int form_packs(const std::vector<int2> &pr, int RB, std::vector<int4> &packs);
std::vector<int> form_rounds(std::vector<int4> &packs, int norb);

// Five pencil passes per batch of packs, one stream.  The FP64 form takes its packs in rounds on
// disjoint orbitals (batches never span two rounds), so that W repeats bit for bit.
template <typename T>
ace_status run_chain_pencil(ace_op *op, const T *phi, const T *Kd, const cpx<T> *const *twd, int count,
                            std::vector<void *> &temps) {
  const ace_desc &d = op->desc;
  const long long N = op->N;
  cudaStream_t st = op->stream;
  const int npacks = (count + 1) / 2;
  const double scratch_budget = (double)env_int("ACE_SCRATCH_MB", 64) * 1048576.0;
  int batch = (int)std::max(1.0, std::floor(scratch_budget / (double)(sizeof(cpx<T>) * N)));
  batch = std::min(batch, std::max(npacks, 1));
  batch = std::min(batch, 65535);
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(cpx<T>) * (size_t)N * batch, st), "alloc scratch");
  temps.push_back(tmp);
  ace::PairPassArgs<T> a{};
  a.phi = phi;
  a.W = static_cast<T *>(op->W);
  a.scratch = static_cast<cpx<T> *>(tmp);
  a.packs = op->packs;
  a.kernel = Kd;
  a.N = N;
  a.n1 = d.n[0];
  a.n2 = d.n[1];
  a.n3 = d.n[2];
  std::vector<int> rb = {0, npacks};
  if (op->fp64) {
    std::vector<int4> packs;
    form_packs(op->pairs_h, 1, packs);
    rb = form_rounds(packs, op->n);
    ACE_CUDA(cudaMallocAsync(&tmp, sizeof(int4) * packs.size(), st), "alloc packs");
    temps.push_back(tmp);
    ACE_CUDA(host_upload(op, tmp, packs.data(), sizeof(int4) * packs.size(), st), "pack upload");
    a.packs = static_cast<const int4 *>(tmp);
  }
  for (size_t r = 0; r + 1 < rb.size(); ++r)
    for (int p0 = rb[r]; p0 < rb[r + 1]; p0 += batch) {
      const int nb = std::min(batch, rb[r + 1] - p0);
      a.pack0 = p0;
      const int modes[5] = {ace::PASS_FWD3_PAIR, ace::PASS_FWD2, ace::PASS_CONV1, ace::PASS_INV2,
                            ace::PASS_INV3_ACC};
      const int axis[5] = {2, 1, 0, 1, 2};
      for (int k = 0; k < 5; ++k) {
        a.tw = twd[axis[k]];
        ACE_CUDA(ace::launch_pair_pass<T>(modes[k], a, nb, st), "pair pass");
        ++op->launches;
      }
    }
  return ACE_OK;
}

// The per-context L2 set-aside for persisting lines, raised to mb MB (clamped to the device's
// maximum) if it is smaller; returns the set-aside in bytes (0: none possible).
size_t l2_set_aside(int dev, int mb) {
  int max_persist = 0;
  cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
  const size_t limit = std::min((size_t)mb << 20, (size_t)std::max(0, max_persist));
  if (limit == 0) return 0;
  size_t now = 0;
  cudaDeviceGetLimit(&now, cudaLimitPersistingL2CacheSize);
  if (now < limit) cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, limit);
  cudaGetLastError();
  return limit;
}

// Marks [base, base + bytes) as persisting in L2 for work on stream st (a per-context set-aside of
// at most mb MB, clamped to the device's limits); bytes = 0 turns the window off.  Failures only
// lose the hint: their error state is cleared.  Inside a stream capture the window is copied into
// the recorded kernels; the set-aside must then exist already (l2_set_aside before the capture).
void l2_window(cudaStream_t st, int dev, void *base, size_t bytes, int mb) {
  cudaStreamAttrValue v{};
  if (bytes > 0 && mb > 0) {
    int max_window = 0;
    cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev);
    const size_t limit = l2_set_aside(dev, mb);
    if (limit == 0 || max_window <= 0) return;
    v.accessPolicyWindow.base_ptr = base;
    v.accessPolicyWindow.num_bytes = std::min({bytes, limit, (size_t)max_window});
    v.accessPolicyWindow.hitRatio = 1.0f;
    v.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    v.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
  }
  cudaStreamSetAttribute(st, cudaStreamAttributeAccessPolicyWindow, &v);
  cudaGetLastError();
}

// Packs of a sorted pair list: two pairs that share an orbital s, written (s, i1, s, i2), so that
// both plane passes read three planes and the W_s terms of the pack go out with one atomic.  The
// list is taken in blocks of RB consecutive rows; inside a block, pairs with the same partner j are
// packed together first (phi_j and W_j are then reused while they are in L2, and the block's own
// rows stay in L2 for the whole block), then the block's remaining pairs by common row (RB = 1 gives
// the row packs (i, j1), (i, j2) only).  Single pairs left over are packed together at the end as
// mixed packs.  Returns the number of packs that share their first orbital (they come first).
int form_packs(const std::vector<int2> &pr, int RB, std::vector<int4> &packs) {
  RB = std::max(1, RB);
  packs.clear();
  std::vector<int2> left;
  std::vector<int2> bp, rest;
  size_t r0 = 0;
  while (r0 < pr.size()) {
    const int blk = pr[r0].x / RB;
    size_t r1 = r0;
    while (r1 < pr.size() && pr[r1].x / RB == blk) ++r1;
    bp.assign(pr.begin() + r0, pr.begin() + r1);
    rest.clear();
    if (RB > 1) {
      std::stable_sort(bp.begin(), bp.end(), [](int2 u, int2 v) { return u.y < v.y; });
      for (size_t k = 0; k < bp.size();) {
        size_t k1 = k;
        while (k1 < bp.size() && bp[k1].y == bp[k].y) ++k1;
        const int j = bp[k].y;
        size_t m = k;
        for (; m + 1 < k1; m += 2) packs.push_back(make_int4(j, bp[m].x, j, bp[m + 1].x));
        if (m < k1) rest.push_back(bp[m]);
        k = k1;
      }
      std::sort(rest.begin(), rest.end(), [](int2 u, int2 v) { return u.x < v.x || (u.x == v.x && u.y < v.y); });
    } else {
      rest.swap(bp);
    }
    for (size_t k = 0; k < rest.size();) {
      size_t k1 = k;
      while (k1 < rest.size() && rest[k1].x == rest[k].x) ++k1;
      const int row = rest[k].x;
      size_t m = k;
      for (; m + 1 < k1; m += 2) packs.push_back(make_int4(row, rest[m].y, row, rest[m + 1].y));
      if (m < k1) left.push_back(rest[m]);
      k = k1;
    }
    r0 = r1;
  }
  const int nshared = (int)packs.size();
  for (size_t k = 0; k < left.size(); k += 2) {
    const int2 p = left[k];
    const int2 q = (k + 1 < left.size()) ? left[k + 1] : make_int2(-1, -1);
    packs.push_back(make_int4(p.x, p.y, q.x, q.y));
  }
  return nshared;
}

// Reorders packs into rounds whose packs touch disjoint orbitals (first fit in pack order) and
// returns the start of every round in the new order, followed by the end.  Inside a round each W
// element receives at most one addition, so a chain run round after round adds the terms of every
// element in one fixed order: the FP64 form repeats bit for bit.
std::vector<int> form_rounds(std::vector<int4> &packs, int norb) {
  std::vector<std::vector<int4>> rounds;
  std::vector<std::vector<unsigned char>> used;
  for (const int4 &p : packs) {
    const int rows[4] = {p.x, p.y, p.z, p.w};
    size_t r = 0;
    for (; r < rounds.size(); ++r) {
      bool free_ = true;
      for (int k = 0; k < 4 && free_; ++k)
        if (rows[k] >= 0 && used[r][rows[k]]) free_ = false;
      if (free_) break;
    }
    if (r == rounds.size()) {
      rounds.emplace_back();
      used.emplace_back((size_t)norb, (unsigned char)0);
    }
    for (int k = 0; k < 4; ++k)
      if (rows[k] >= 0) used[r][rows[k]] = 1;
    rounds[r].push_back(p);
  }
  std::vector<int> bounds;
  packs.clear();
  for (const auto &rd : rounds) {
    bounds.push_back((int)packs.size());
    packs.insert(packs.end(), rd.begin(), rd.end());
  }
  bounds.push_back((int)packs.size());
  return bounds;
}

// Persistent chain of one or more builds on one grid: every pack of every build in one launch
// (persistent_chain.cuh) on stream st.  The packs are either on the host (packs, with pack_build the
// build of each pack, empty for one build), or, with packs empty, the builds' device lists `dev`,
// concatenated on the device (their counts are read there; maxnp bounds the total).  builds[b]
// holds the device pointers of build b; a wait that gives up sets op->tc_err.
template <typename T>
ace_status run_chain_persistent(ace_op *op, cudaStream_t st, const DeviceTables *tab, const ace::PersistOps<T> &po,
                                const std::vector<int4> &packs, const std::vector<int> &pack_build,
                                const std::vector<ace::QueueSrc> &dev, int maxnp,
                                const std::vector<ace::ChainBuild<T>> &builds, std::vector<void *> &temps,
                                const ChainParams &cp) {
  const long long N = op->N;
  const bool on_device = packs.empty() && !dev.empty();
  const int np = on_device ? maxnp : (int)packs.size();
  if (np == 0) return ACE_OK;
  const int lag = std::max(1, cp.lag);
  const int nslots = on_device ? 2 * lag + 2 : std::min(2 * lag + 2, np);
  // one allocation: packs, builds, pack_build, device list sources, counters (3 np) with the ticket,
  // the stall word and the device pack count; then the scratch slots
  const size_t b_packs = sizeof(int4) * np, b_builds = sizeof(ace::ChainBuild<T>) * builds.size();
  const size_t b_pb = sizeof(int) * (on_device ? (size_t)np : pack_build.size());
  const size_t b_src = on_device ? sizeof(ace::QueueSrc) * dev.size() : 0;
  const size_t b_cnt = sizeof(int) * (3 * (size_t)np + 4);
  auto up16 = [](size_t x) { return (x + 15) / 16 * 16; };
  const size_t o_builds = up16(b_packs), o_pb = o_builds + up16(b_builds), o_src = o_pb + up16(b_pb);
  const size_t o_cnt = o_src + up16(b_src);
  const size_t meta = o_cnt + up16(b_cnt);
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, meta, st), "alloc pack queue");
  temps.push_back(tmp);
  char *m = static_cast<char *>(tmp);
  int *cnt = reinterpret_cast<int *>(m + o_cnt);
  ACE_CUDA(cudaMemsetAsync(cnt, 0, b_cnt, st), "zero counters");
  if (on_device) {
    ACE_CUDA(host_upload(op, m + o_builds, builds.data(), b_builds, st), "queue upload");
    ACE_CUDA(host_upload(op, m + o_src, dev.data(), b_src, st), "queue upload");
    ACE_CUDA(ace::launch_queue_assemble(reinterpret_cast<const ace::QueueSrc *>(m + o_src), (int)dev.size(),
                                        reinterpret_cast<int4 *>(m), reinterpret_cast<int *>(m + o_pb),
                                        cnt + 3 * (size_t)np + 2, st),
             "queue assembly");
    ++op->launches;
  } else {
    std::vector<char> hm(o_src, 0);
    std::memcpy(hm.data(), packs.data(), b_packs);
    std::memcpy(hm.data() + o_builds, builds.data(), b_builds);
    if (b_pb) std::memcpy(hm.data() + o_pb, pack_build.data(), b_pb);
    ACE_CUDA(host_upload(op, m, hm.data(), o_src, st), "pack queue upload");
  }
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(cpx<T>) * (size_t)N * nslots, st), "alloc scratch");
  temps.push_back(tmp);
  ace::PersistArgs<T> a{};
  a.builds = reinterpret_cast<const ace::ChainBuild<T> *>(m + o_builds);
  a.pack_build = b_pb ? reinterpret_cast<const int *>(m + o_pb) : nullptr;
  a.packs = reinterpret_cast<const int4 *>(m);
  a.npacks = np;
  a.npacks_d = on_device ? cnt + 3 * (size_t)np + 2 : nullptr;
  a.scratch = static_cast<cpx<T> *>(tmp);
  a.nslots = nslots;
  a.lag = lag;
  a.tw1 = static_cast<const cpx<T> *>(tab->tw[0]);
  a.tw2 = static_cast<const cpx<T> *>(tab->tw[1]);
  a.tw3 = static_cast<const cpx<T> *>(tab->tw[2]);
  a.counters = cnt;
  a.ticket = cnt + 3 * (size_t)np;
  a.err = op->tc_err;
  a.N = N;
  // ACE_PERSIST_WAIT_NS bounds each wait (default 2 s); ACE_PERSIST_TEST_STALL=1 makes the pencil
  // tasks wait for a word that nothing sets (a test of the give-up path)
  const char *wn = std::getenv("ACE_PERSIST_WAIT_NS");
  a.wait_ns = (wn && *wn) ? std::strtoull(wn, nullptr, 10) : 2000000000ull;
  a.stall = env_int("ACE_PERSIST_TEST_STALL", 0) ? cnt + 3 * (size_t)np + 1 : nullptr;
  a.hints = env_int("ACE_L2_HINTS", 1);
  a.skip_rel = plane_skip_rel(sizeof(T) == 8);
  // keep the scratch slots resident in L2 (a per-context set-aside of persisting lines)
  const int persist_mb = cp.persist_mb;
  if (persist_mb > 0) l2_window(st, op->dev, a.scratch, sizeof(cpx<T>) * (size_t)N * nslots, persist_mb);
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, op->dev);
  const int per_sm = po.blocks_per_sm();
  if (per_sm <= 0) return fail(ACE_ERR_CUDA, "persistent chain kernel does not fit on an SM");
  const long long tasks = (long long)po.tasks_per_pack * (np + 2 * lag);
  const int grid = (int)std::min<long long>((long long)per_sm * sms, tasks);
  cudaError_t e = po.launch(a, grid, st);
  if (persist_mb > 0) l2_window(st, op->dev, nullptr, 0, 0);  // window off again
  ACE_CUDA(e, "persistent chain");
  ++op->launches;
  return ACE_OK;
}

// Plane, pencil, plane per batch; packs grouped by their shared first orbital.
template <typename T>
ace_status run_chain_plane(ace_op *op, const T *phi, const DeviceTables *tab, const ace::PlaneOps<T> &pops,
                           int count, std::vector<void *> &temps, const ChainParams &cp, int max_packs = -1) {
  const ace_desc &d = op->desc;
  const long long N = op->N;
  cudaStream_t st = op->stream;
  const int G = cp.G;
  const int B = std::max(G, cp.B);
  const int nstreams = std::min(kSide, std::max(1, cp.streams));
  const bool acc = pops.acc_fits && G > 1;
  std::vector<int4> packs;
  std::vector<int4> groups;
  int nshared = form_packs(op->pairs_h, cp.RB, packs);
  // FP64 form: rounds of packs on disjoint orbitals, one pack per group, the side streams joined
  // between rounds (deterministic W)
  const bool rounds_on = op->fp64;
  std::vector<int> rb;
  if (rounds_on) {
    rb = form_rounds(packs, op->n);
    nshared = 0;
  }
  const bool acc_on = acc && !rounds_on;
  // groups: runs of at most G consecutive packs with the same shared orbital (accumulated in
  // shared memory by the inverse pass when acc); mixed packs are groups of their own
  for (int k = 0; k < (int)packs.size();) {
    int k1 = k + 1;
    if (k < nshared)
      while (k1 < nshared && k1 - k < G && packs[k1].x == packs[k].x) ++k1;
    groups.push_back(make_int4(k, k1 - k, (acc_on && k < nshared) ? packs[k].x : -1, 0));
    k = k1;
  }
  // batches of whole groups holding at most B packs (never across a round boundary); round_end[b]
  // marks the last batch of a round
  std::vector<int2> batches;  // (first group, end group)
  std::vector<char> round_end;
  {
    size_t ri = 1;
    int gb = 0, cnt = 0;
    for (int g = 0; g < (int)groups.size(); ++g) {
      const bool new_round = rounds_on && ri < rb.size() && groups[g].x == rb[ri];
      if ((cnt + groups[g].y > B || new_round) && g > gb) {
        batches.push_back(make_int2(gb, g));
        round_end.push_back(new_round ? 1 : 0);
        gb = g;
        cnt = 0;
      }
      if (new_round) ++ri;
      cnt += groups[g].y;
    }
    if (gb < (int)groups.size()) {
      batches.push_back(make_int2(gb, (int)groups.size()));
      round_end.push_back(1);
    }
  }
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(int4) * (packs.size() + groups.size()), st), "alloc packs");
  temps.push_back(tmp);
  int4 *packs_d = static_cast<int4 *>(tmp);
  int4 *groups_d = packs_d + packs.size();
  std::vector<int4> up(packs);
  up.insert(up.end(), groups.begin(), groups.end());
  ACE_CUDA(host_upload(op, packs_d, up.data(), sizeof(int4) * up.size(), st), "pack upload");
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(cpx<T>) * (size_t)N * B * nstreams, st), "alloc scratch");
  temps.push_back(tmp);
  cpx<T> *scratch_all = static_cast<cpx<T> *>(tmp);
  // plane maxima for the plane skip (mixed form), on st before the side streams fork from it
  float skip_rel = 0.f;
  if constexpr (sizeof(T) == 4) {
    skip_rel = plane_skip_rel(false);
    if (skip_rel > 0.f) ACE_CUDA(plane_max_table(op, phi, st), "plane maxima");
  }
  // consecutive batches alternate between side streams (own scratch each) so that one batch's
  // kernels fill the tail of the previous one; W is only touched by atomic adds
  cudaStream_t side[kSide];
  for (int k = 0; k < kSide; ++k) side[k] = st;
  cudaEvent_t fork = nullptr;
  cudaEvent_t rev[kSide] = {};
  if (nstreams > 1 && rounds_on)
    for (int k = 0; k < nstreams; ++k) ACE_CUDA(cudaEventCreateWithFlags(&rev[k], cudaEventDisableTiming), "event");
  if (nstreams > 1) {
    ACE_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event");
    ACE_CUDA(cudaEventRecord(fork, st), "event");
    for (int k = 0; k < nstreams; ++k) {
      ACE_CUDA(get_side_stream(op->dev, kSide * op->lane + k, &side[k]), "side stream");
      ACE_CUDA(cudaStreamWaitEvent(side[k], fork, 0), "wait");
    }
  }
  // ask L2 to keep each stream's FFT scratch resident between the three passes (a per-context
  // set-aside of the L2 for persisting lines; ACE_L2_PERSIST_MB=0 turns it off)
  const int persist_mb = cp.persist_mb;
  if (persist_mb > 0 && nstreams > 1) {
    for (int k = 0; k < nstreams; ++k)
      l2_window(side[k], op->dev, scratch_all + (size_t)k * B * N,
                std::min<size_t>(((size_t)persist_mb << 20) / (size_t)nstreams, sizeof(cpx<T>) * (size_t)B * (size_t)N),
                persist_mb);
  }

  ace::PlaneArgs<T> pa;
  pa.phi = phi;
  pa.W = static_cast<T *>(op->W);
  pa.scratch = scratch_all;
  pa.packs = packs_d;
  pa.groups = groups_d;
  pa.tw2 = static_cast<const cpx<T> *>(tab->tw[1]);
  pa.tw3 = static_cast<const cpx<T> *>(tab->tw[2]);
  pa.N = N;
  pa.n1 = d.n[0];
  pa.hints = env_int("ACE_L2_HINTS", 1);
  pa.pmax = skip_rel > 0.f ? op->pmax : nullptr;
  pa.gmax = skip_rel > 0.f ? op->gmax : nullptr;
  pa.skip_rel = skip_rel;
  ace::PairPassArgs<T> ca;
  ca.phi = phi;
  ca.W = static_cast<T *>(op->W);
  ca.scratch = scratch_all;
  ca.packs = packs_d;
  ca.kernel = static_cast<const T *>(tab->Kperm);
  ca.tw = static_cast<const cpx<T> *>(tab->tw[0]);
  ca.N = N;
  ca.n1 = d.n[0];
  ca.n2 = d.n[1];
  ca.n3 = d.n[2];
  ca.conv_tile = cp.conv;
  for (size_t bi = 0; bi < batches.size(); ++bi) {
    const int2 b = batches[bi];
    if (max_packs >= 0 && groups[b.x].x >= max_packs) break;  // autotuning sample
    const int k = (int)(bi % nstreams);
    const int p0 = groups[b.x].x;
    const int p1 = groups[b.y - 1].x + groups[b.y - 1].y;
    pa.scratch = scratch_all + (size_t)k * B * N;
    ca.scratch = pa.scratch;
    pa.pack0 = p0;
    pa.batch0 = p0;
    pa.group0 = b.x;
    ca.pack0 = p0;
    ACE_CUDA(pops.fwd(pa, p1 - p0, side[k]), "plane forward");
    ACE_CUDA(ace::launch_conv_pass<T>(ca, p1 - p0, side[k]), "pencil pass");
    ACE_CUDA(pops.inv(pa, b.y - b.x, acc_on, side[k]), "plane inverse");
    op->launches += 3;
    if (rounds_on && nstreams > 1 && round_end[bi]) {
      // every stream waits for every other one: the next round starts after this one ends
      for (int j = 0; j < nstreams; ++j) ACE_CUDA(cudaEventRecord(rev[j], side[j]), "event");
      for (int j = 0; j < nstreams; ++j)
        for (int q = 0; q < nstreams; ++q)
          if (q != j) ACE_CUDA(cudaStreamWaitEvent(side[j], rev[q], 0), "round join");
    }
  }
  if (nstreams > 1) {
    for (int k = 0; k < nstreams; ++k) {
      if (persist_mb > 0) l2_window(side[k], op->dev, nullptr, 0, 0);  // window off again
      ACE_CUDA(cudaEventRecord(fork, side[k]), "event");
      ACE_CUDA(cudaStreamWaitEvent(st, fork, 0), "join");
    }
    cudaEventDestroy(fork);
    for (int k = 0; k < nstreams; ++k)
      if (rev[k]) cudaEventDestroy(rev[k]);
  }
  return ACE_OK;
}

bool use_tc() { return env_int("ACE_NO_TC", 0) == 0; }

// G = scale * X Y^T (FP64 result)
template <typename T>
cudaError_t dense_gram(const T *X, int nx, const T *Y, int ny, long long K, double scale, double *G, int *err,
                       std::vector<void *> &temps, cudaStream_t st, long *launches) {
  if constexpr (sizeof(T) == 4) {
    if (use_tc() && ace::tc_gram_shape_ok(K)) {
      void *ws = nullptr;
      cudaError_t e = cudaMallocAsync(&ws, ace::tc_gram_workspace_bytes(X, nx, Y, ny, K), st);
      if (e != cudaSuccess) return e;
      temps.push_back(ws);
      return ace::launch_tc_gram(X, nx, Y, ny, K, scale, G, ws, err, st, launches);
    }
  }
  *launches += 1;
  double *partial = nullptr;
  if constexpr (sizeof(T) == 8) {
    // FP64 form: chunk sums added in a fixed order, so that the result repeats bit for bit
    void *ws = nullptr;
    cudaError_t e = cudaMallocAsync(&ws, ace::gram_chunks_bytes(nx, ny, K), st);
    if (e != cudaSuccess) return e;
    temps.push_back(ws);
    partial = static_cast<double *>(ws);
    *launches += 1;
  }
  return ace::launch_gram<T>(X, nx, Y, ny, K, scale, false, false, G, st, partial);
}

// Z = A Y, A (m x n) in T
template <typename T>
cudaError_t dense_left_mul(const T *A, int m, int n, const T *Y, long long K, T *Z, int *err, cudaStream_t st,
                           long *launches) {
  *launches += 1;
  if constexpr (sizeof(T) == 4) {
    if (use_tc()) {
      const cudaError_t e = ace::launch_tc_left_mul(A, m, n, Y, K, Z, err, st);
      if (e != cudaErrorNotSupported) return e;  // else the CUDA-core kernel below takes the shape
    }
  }
  return ace::launch_left_mul<T>(A, m, n, Y, K, Z, st);
}

// Relative distance from rho_cut within which screen values are recomputed (twice the BF16x3
// tensor-core bound of 3 * 2^-16 per product, the opt-in tensor-core screen).
constexpr double kScreenRefineBand = 1e-4;

// The screen runs on the CUDA cores (FP32 products, FP64 across K-splits) unless ACE_TC_SCREEN=1
// asks for the BF16x3 tensor-core Gram of |phi|.
bool tc_screen_requested() { return use_tc() && env_int("ACE_TC_SCREEN", 0) != 0; }

// Workspace of the FP32 screen of n orbitals over N points (0: none needed)
size_t screen_workspace_bytes(const float *phi, int n, long long N) {
  if (tc_screen_requested()) return ace::tc_screen_workspace_bytes(phi, n, N - N % 32);
  return ace::screen_syrk_workspace_bytes(n, N);
}

// Screen contribution of the columns [c0, c0 + K) of phi into O (accumulating; O zeroed by the
// caller; only the upper triangle is used): the CUDA-core kernel of FP32 products and FP64 split
// sums (ws of screen_workspace_bytes), or the tensor-core Gram of |phi| when requested; else the
// TMA-fed 64 x 64 tile kernel, else the register-staged kernels.  With pm, the CUDA-core kernel
// also fills the plane-maxima table; *pm->done is cleared when this call did not.
template <typename T>
cudaError_t screen_cols(const T *phi, int n, long long ld, long long c0, long long K, double dV, double *O, int *err,
                        void *ws, cudaStream_t st, long *launches, const ace::PlaneMaxOut *pm = nullptr) {
  if constexpr (sizeof(T) == 4) {
    cudaError_t e = cudaSuccess;
    if (ws && tc_screen_requested()) {
      if (pm) *pm->done = false;
      if (ace::launch_tc_screen(phi, n, ld, c0, K, dV, O, ws, err, st, launches, &e)) return e;
    } else if (ws && env_int("ACE_SCREEN_TILES", 0) == 0 &&
               ace::launch_screen_syrk(phi, n, ld, c0, K, dV, O, ws, err, st, launches, &e, pm)) {
      return e;
    }
    if (pm) *pm->done = false;
    ++*launches;
    if (ace::launch_screen_tma(phi, n, ld, c0, K, dV, O, err, st)) return cudaGetLastError();
    if (K % 4 != 0 || ld % 4 != 0 || c0 % 4 != 0) {
      // point counts off the 16-byte grid (odd axis lengths): the general Gram kernel (clears O;
      // such inputs are never split into column chunks)
      if (c0 != 0 || K != ld) return cudaErrorInvalidValue;
      return ace::launch_gram<T>(phi, n, phi, n, K, dV, true, true, O, st);
    }
    return ace::launch_screen_cols(phi + c0, n, ld, K, dV, O, st);
  } else {
    *launches += ws ? 2 : 1;
    if (c0 != 0 || K != ld) return cudaErrorInvalidValue;
    // clears O itself; with ws the chunk sums are added in a fixed order
    return ace::launch_gram<T>(phi, n, phi, n, K, dV, true, true, O, st, static_cast<double *>(ws));
  }
}

// Phase 1 of a build: inputs, tables, screen and compaction; the pair count and list are copied
// to pinned host memory asynchronously (read after the stream reaches them).
template <typename T>
ace_status build_begin(ace_op *op, const void *phi_in, ace_dtype dtype) {
  const ace_desc &d = op->desc;
  const int n = op->n;
  const long long N = op->N;
  cudaStream_t st = op->stream;
  for (int i = 0; i < 6; ++i) ACE_CUDA(cudaEventCreate(&op->ev[i]), "event create");
  ACE_CUDA(mark(op, 0, st), "event record");
  // FP32 host input of a screened build: copied in column chunks on a copy stream while the
  // screen adds each chunk's contribution on the build stream (the transfer hides the screen)
  const bool same = (dtype == ACE_F64) == (sizeof(T) == 8);
  const bool pipelined = sizeof(T) == 4 && same && d.rho_cut > 0.0 && !op->use_given && N % 4 == 0 &&
                         !is_device_pointer(phi_in) &&
                         env_int("ACE_PIPELINED_INPUT", 1) != 0;
  const T *phi = nullptr;
  if (pipelined) {
    void *tmp = nullptr;
    ACE_CUDA(cudaMallocAsync(&tmp, sizeof(T) * (size_t)n * N, st), "staging allocation");
    op->temps.push_back(tmp);
    phi = static_cast<const T *>(tmp);
  } else {
    ace_status s = stage_input<T>(op, phi_in, dtype, (long long)n * N, &phi, &op->temps);
    if (s != ACE_OK) return s;
  }
  op->phi_work = phi;
  cudaError_t e = get_tables<T>(op->dev, d, st, &op->tab);
  if (e != cudaSuccess) return cuda_fail(e, "kernel and twiddle tables");

  // ---- screen (section II): O_ij = dV sum |phi_i phi_j|, pair list ----
  const size_t maxpairs = (size_t)n * (n + 1) / 2;
  ACE_CUDA(op_alloc(op, &op->O, sizeof(double) * n * n), "alloc O");
  ACE_CUDA(op_alloc(op, &op->O_sym, sizeof(double) * n * n), "alloc O_sym");
  ACE_CUDA(op_alloc(op, &op->pairs, sizeof(int2) * (maxpairs + 2)), "alloc pairs");
  ACE_CUDA(op_alloc(op, &op->packs, sizeof(int4) * (maxpairs / 2 + 2)), "alloc packs");
  ACE_CUDA(op_alloc(op, &op->count_d, sizeof(int) * 4), "alloc count");
  ACE_CUDA(op_alloc(op, &op->status_d, sizeof(int) * 4), "alloc status");
  op->tc_err = op->status_d + 1;
  ACE_CUDA(cudaMemsetAsync(op->status_d, 0, sizeof(int) * 4, st), "zero status");
  ACE_CUDA(op_alloc(op, &op->energy_d, sizeof(double) * 2), "alloc energy");
  if (op->use_given) {
    // the caller's pair list: no screen (O stays zero); pairs and packs uploaded, count and pairs
    // written straight into the host readback area
    const size_t np = op->given.size();
    std::vector<int4> pk((np + 1) / 2);
    for (size_t p = 0; p < pk.size(); ++p) {
      const int2 a = op->given[2 * p];
      const int2 b = 2 * p + 1 < np ? op->given[2 * p + 1] : make_int2(-1, -1);
      pk[p] = make_int4(a.x, a.y, b.x, b.y);
    }
    ACE_CUDA(cudaMemsetAsync(op->O, 0, sizeof(double) * n * n, st), "zero O");
    ACE_CUDA(cudaMemsetAsync(op->O_sym, 0, sizeof(double) * n * n, st), "zero O");
    const size_t rb_bytes = 32 + sizeof(int2) * maxpairs;
    ACE_CUDA(pinned_get(rb_bytes, &op->readback), "pinned readback");
    op->readback_bytes = rb_bytes;
    *static_cast<int *>(op->readback) = (int)np;
    int2 *rp = reinterpret_cast<int2 *>(static_cast<char *>(op->readback) + 32);
    std::copy(op->given.begin(), op->given.end(), rp);
    // uploads from the pinned area, so that they stay asynchronous (the area lives until destroy)
    ACE_CUDA(cudaMemcpyAsync(op->pairs, rp, sizeof(int2) * np, cudaMemcpyHostToDevice, st), "pair upload");
    ACE_CUDA(cudaMemcpyAsync(op->count_d, op->readback, sizeof(int), cudaMemcpyHostToDevice, st), "count upload");
    if (!pk.empty()) ACE_CUDA(host_upload(op, op->packs, pk.data(), sizeof(int4) * pk.size(), st), "pack upload");
    ACE_CUDA(mark(op, 1, st), "event record");
    return ACE_OK;
  }
  // workspace of the tensor-core screen (FP64 partial sums of its K-splits; sized for the whole N)
  void *screen_ws = nullptr;
  if constexpr (sizeof(T) == 4) {
    const size_t wsb = d.rho_cut > 0.0 ? screen_workspace_bytes(phi, n, N) : 0;
    if (wsb) ACE_CUDA(op_alloc(op, &screen_ws, wsb), "alloc screen workspace");
  } else if (d.rho_cut > 0.0) {
    ACE_CUDA(cudaMallocAsync(&screen_ws, ace::gram_chunks_bytes(n, n, N), st), "alloc screen workspace");
    op->temps.push_back(screen_ws);
  }
  // the plane-maxima table of the mixed form's plane skip, taken by the screen on its way through phi
  // when it can (else the chain computes it with its own pass)
  bool pm_done = false;
  ace::PlaneMaxOut pmo{nullptr, nullptr, (long long)d.n[1] * d.n[2], d.n[0], &pm_done};
  if (sizeof(T) == 4 && d.rho_cut > 0.0 && plane_skip_rel(false) > 0.f && !op->pmax) {
    ACE_CUDA(op_alloc(op, &pmo.pmax, sizeof(float) * (size_t)n * d.n[0]), "alloc plane maxima");
    ACE_CUDA(op_alloc(op, &pmo.gmax, sizeof(float) * (size_t)n), "alloc orbital maxima");
    ACE_CUDA(cudaMemsetAsync(pmo.pmax, 0, sizeof(float) * (size_t)n * d.n[0], st), "zero plane maxima");
    ACE_CUDA(cudaMemsetAsync(pmo.gmax, 0, sizeof(float) * (size_t)n, st), "zero orbital maxima");
    pm_done = true;
  }
  const ace::PlaneMaxOut *pm = pmo.pmax ? &pmo : nullptr;
  if (pipelined) {
    ACE_CUDA(cudaMemsetAsync(op->O, 0, sizeof(double) * n * n, st), "zero O");
    cudaStream_t cs;
    ACE_CUDA(get_side_stream(op->dev, (kSide + 1) * kLanes + op->lane, &cs), "copy stream");
    cudaEvent_t ev;
    ACE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    ACE_CUDA(cudaEventRecord(ev, st), "event");  // the staging buffer is allocated on st
    ACE_CUDA(cudaStreamWaitEvent(cs, ev, 0), "wait");
    cudaEventDestroy(ev);
    const long long w = ((N + 7) / 8 + 2047) / 2048 * 2048;  // about 8 chunks, 2048-point aligned
    for (long long c0 = 0; c0 < N; c0 += w) {
      const long long wc = std::min(w, N - c0);
      ACE_CUDA(cudaMemcpy2DAsync(const_cast<T *>(phi) + c0, sizeof(T) * N, static_cast<const T *>(phi_in) + c0,
                                 sizeof(T) * N, sizeof(T) * wc, n, cudaMemcpyHostToDevice, cs),
               "host-to-device copy");
      ACE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
      ACE_CUDA(cudaEventRecord(ev, cs), "event");
      ACE_CUDA(cudaStreamWaitEvent(st, ev, 0), "wait");
      cudaEventDestroy(ev);
      ACE_CUDA(screen_cols<T>(phi, n, N, c0, wc, op->dV, op->O, op->tc_err, screen_ws, st, &op->launches, pm),
               "screen");
    }
  } else if (d.rho_cut > 0.0) {
    ACE_CUDA(cudaMemsetAsync(op->O, 0, sizeof(double) * n * n, st), "zero O");
    ACE_CUDA(screen_cols<T>(phi, n, N, 0, N, op->dV, op->O, op->tc_err, screen_ws, st, &op->launches, pm),
             "screen");
  } else {
    ACE_CUDA(cudaMemsetAsync(op->O, 0, sizeof(double) * n * n, st), "screen skip");
  }
  if (pm && pm_done) {
    // every screen launch filled the table: the chain uses it instead of its own pass
    op->pmax = pmo.pmax;
    op->gmax = pmo.gmax;
  }
  if constexpr (sizeof(T) == 4) {
    // pair decisions within the tensor-core products' error of rho_cut are taken on recomputed values
    if (d.rho_cut > 0.0) {
      ACE_CUDA(ace::launch_screen_refine(phi, n, N, op->dV, d.rho_cut, kScreenRefineBand, op->O, st), "refine");
      ++op->launches;
    }
  }
  ACE_CUDA(ace::launch_screen_compact(op->O, n, d.rho_cut, op->pairs, op->packs, op->count_d, op->O_sym, st),
           "compact");
  ++op->launches;
  // pinned readback area: [count, flags0, flags1, pad] [energy] [pairs]
  const size_t rb_bytes = 32 + sizeof(int2) * maxpairs;
  ACE_CUDA(pinned_get(rb_bytes, &op->readback), "pinned readback");
  op->readback_bytes = rb_bytes;
  ACE_CUDA(cudaMemcpyAsync(op->readback, op->count_d, sizeof(int), cudaMemcpyDeviceToHost, st), "count readback");
  ACE_CUDA(cudaMemcpyAsync(static_cast<char *>(op->readback) + 32, op->pairs, sizeof(int2) * maxpairs,
                           cudaMemcpyDeviceToHost, st),
           "pair readback");
  ACE_CUDA(mark(op, 1, st), "event record");
  return ACE_OK;
}

// Phase 2: with the pair list on the host, the pair chain, M, Cholesky and xi; status and E_x are
// copied back asynchronously.  Call after op->ev[1] has completed.
// W = sum over the listed pairs op->pairs_h of the Eq. (vx) terms, into op->W (zeroed here): the
// persistent chain when requested, else the plane chain where the plane shape is compiled, else
// the five pencil passes.
template <typename T>
ace_status run_chain(ace_op *op, const T *phi, int count) {
  const ace_desc &d = op->desc;
  const DeviceTables *tab = op->tab;
  std::vector<void *> &temps = op->temps;
  ACE_CUDA(cudaMemsetAsync(op->W, 0, op->esz * (size_t)op->n * op->N, op->stream), "zero W");
  ace::PlaneOps<T> pops{};
  ace::PersistOps<T> qops{};
  const bool plane = find_plane_ops<T>(d.n[1], d.n[2], &pops) && ace::conv_length_supported(d.n[0]) &&
                     env_int("ACE_FORCE_PENCIL", 0) == 0;
  const ChainParams cp = chain_params(d, op->fp64);
  const bool persistent = plane && cp.persistent && find_persist_ops<T>(d.n[0], d.n[1], d.n[2], &qops);
  if (count > 0 && persistent) {
    std::vector<int4> packs;
    form_packs(op->pairs_h, cp.RB, packs);
    const float *pm = nullptr, *gm = nullptr;
    if (sizeof(T) == 4 && plane_skip_rel(false) > 0.f) {
      ACE_CUDA(plane_max_table(op, reinterpret_cast<const float *>(phi), op->stream), "plane maxima");
      pm = op->pmax;
      gm = op->gmax;
    }
    const std::vector<ace::ChainBuild<T>> one{
        {phi, static_cast<T *>(op->W), static_cast<const T *>(tab->Kperm), pm, gm}};
    return run_chain_persistent<T>(op, op->stream, tab, qops, packs, {}, {}, 0, one, temps, cp);
  }
  if (count > 0 && plane) return run_chain_plane<T>(op, phi, tab, pops, count, temps, cp);
  if (count > 0) {
    const cpx<T> *twd[3] = {static_cast<const cpx<T> *>(tab->tw[0]), static_cast<const cpx<T> *>(tab->tw[1]),
                            static_cast<const cpx<T> *>(tab->tw[2])};
    return run_chain_pencil<T>(op, phi, static_cast<const T *>(tab->K), twd, count, temps);
  }
  return ACE_OK;
}

template <typename T>
ace_status factor_and_project(ace_op *op, const T *W);
template <typename T>
ace_status build_dense(ace_op *op);

template <typename T>
ace_status build_finish(ace_op *op) {
  const int n = op->n;
  const long long N = op->N;
  cudaStream_t st = op->stream;
  const T *phi = static_cast<const T *>(op->phi_work);
  const int count = *static_cast<const int *>(op->readback);
  op->npairs = count;
  const int2 *ph = reinterpret_cast<const int2 *>(static_cast<const char *>(op->readback) + 32);
  op->pairs_h.assign(ph, ph + count);
  ace_status s = ACE_OK;

  // ---- pair chain (Eq. vx, Eq. e:vij): W_i = sum_j v_ij phi_j ----
  ACE_CUDA(op_alloc(op, &op->W, op->esz * (size_t)n * N), "alloc W");
  s = run_chain<T>(op, phi, count);
  if (s != ACE_OK) return s;
  ACE_CUDA(mark(op, 2, st), "event record");
  if (op->tail) {
    // M, the Cholesky and xi on the lane's tail stream, so that the next build's pair chain starts
    // on the lane stream meanwhile; the handle keeps the tail stream (its last work) from here on
    cudaEvent_t ev;
    ACE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    ACE_CUDA(cudaEventRecord(ev, st), "event");
    ACE_CUDA(cudaStreamWaitEvent(op->tail, ev, 0), "wait");
    cudaEventDestroy(ev);
    op->stream = op->tail;
  }
  return build_dense<T>(op);
}

// The steps after the pair chain (op->W complete on op->stream): M = -dV Phi^T W, then
// factor_and_project.
template <typename T>
ace_status build_dense(ace_op *op) {
  const int n = op->n;
  const long long N = op->N;
  cudaStream_t st = op->stream;
  const T *phi = static_cast<const T *>(op->phi_work);
  std::vector<void *> &temps = op->temps;

  // ---- M = -dV Phi^T W (App. A) ----
  ACE_CUDA(op_alloc(op, &op->M_raw, sizeof(double) * n * n), "alloc M_raw");
  ACE_CUDA(op_alloc(op, &op->M, sizeof(double) * n * n), "alloc M");
  ACE_CUDA(op_alloc(op, &op->L, sizeof(double) * n * n), "alloc L");
  ACE_CUDA(op_alloc(op, &op->Linv, sizeof(double) * n * n), "alloc Linv");
  ACE_CUDA(dense_gram<T>(phi, n, static_cast<const T *>(op->W), n, N, -op->dV, op->M_raw, op->tc_err, temps, st,
                         &op->launches),
           "M");
  ACE_CUDA(mark(op, 3, st), "event record");

  return factor_and_project<T>(op, static_cast<const T *>(op->W));
}

// App. A from M_raw (filled, op->M_raw): -M = L L^T with M symmetrised, L^-1 and E_x = (f/2) tr M
// (one kernel), then xi = W L^-T stored as rows xi = L^-1 W for the op->N points of W; status and
// E_x are copied to the readback area; the build's workspaces are released in stream order.
template <typename T>
ace_status factor_and_project(ace_op *op, const T *W) {
  const int n = op->n;
  const long long N = op->N;
  cudaStream_t st = op->stream;
  std::vector<void *> &temps = op->temps;
  void *tmp = nullptr;
  double *chol_work = nullptr;
  if (n > 128) {
    ACE_CUDA(cudaMallocAsync(&tmp, sizeof(double) * ((size_t)n * n + 4 * n), st), "alloc cholesky workspace");
    temps.push_back(tmp);
    chol_work = static_cast<double *>(tmp);
  }
  ACE_CUDA(ace::launch_cholesky(op->M_raw, n, op->desc.spin_factor, op->M, op->L, op->Linv, op->energy_d,
                                op->status_d, chol_work, st),
           "cholesky");
  ++op->launches;
  ACE_CUDA(mark(op, 4, st), "event record");

  // ---- xi = W L^-T, stored as rows: xi_rows = L^-1 W_rows ----
  ACE_CUDA(op_alloc(op, &op->xi, op->esz * (size_t)n * N), "alloc xi");
  const T *Linv_T = nullptr;
  if (sizeof(T) == 8) {
    Linv_T = reinterpret_cast<const T *>(op->Linv);
  } else {
    ACE_CUDA(cudaMallocAsync(&tmp, sizeof(T) * n * n, st), "alloc Linv32");
    temps.push_back(tmp);
    ACE_CUDA((ace::launch_convert<double, T>(op->Linv, static_cast<T *>(tmp), (long long)n * n, 1.0, st)), "Linv32");
    ++op->launches;
    Linv_T = static_cast<const T *>(tmp);
  }
  ACE_CUDA(dense_left_mul<T>(Linv_T, n, n, W, N, static_cast<T *>(op->xi), op->tc_err, st, &op->launches), "xi");
  ACE_CUDA(mark(op, 5, st), "event record");
  char *rb = static_cast<char *>(op->readback);
  ACE_CUDA(cudaMemcpyAsync(rb + 4, op->status_d, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "status readback");
  ACE_CUDA(cudaMemcpyAsync(rb + 16, op->energy_d, sizeof(double), cudaMemcpyDeviceToHost, st), "energy readback");
  // workspaces of the build are released in stream order after their last use
  for (void *p : temps) cudaFreeAsync(p, st);
  temps.clear();
  op->phi_work = nullptr;
  return ACE_OK;
}

// The pair chains of `group` (builds begun on one grid, screened on the device, pair counts not
// read on the host) as one persistent launch on st over their concatenated device pack lists; the
// W of every build is allocated and zeroed here.  The caller has joined every build's stream into
// st.  A wait that gives up marks every build of the group.
template <typename T>
ace_status run_queue_chain(const std::vector<ace_op *> &group, cudaStream_t st) {
  ace_op *op0 = group[0];
  const ace_desc &d = op0->desc;
  ace::PersistOps<T> qops{};
  if (!find_persist_ops<T>(d.n[0], d.n[1], d.n[2], &qops))
    return fail(ACE_ERR_UNSUPPORTED_GRID, "no persistent chain for the %dx%dx%d grid", d.n[0], d.n[1], d.n[2]);
  std::vector<ace::ChainBuild<T>> builds;
  std::vector<ace::QueueSrc> src;
  std::vector<int *> flags;
  long long maxnp = 0;
  for (ace_op *op : group) {
    const size_t bytes = op->esz * (size_t)op->n * op->N;
    ACE_CUDA(op_alloc(op, &op->W, bytes), "alloc W");
    ACE_CUDA(cudaMemsetAsync(op->W, 0, bytes, st), "zero W");
    const float *pm = nullptr, *gm = nullptr;
    if (sizeof(T) == 4 && plane_skip_rel(false) > 0.f) {
      ACE_CUDA(plane_max_table(op, reinterpret_cast<const float *>(op->phi_work), st), "plane maxima");
      pm = op->pmax;
      gm = op->gmax;
    }
    builds.push_back({static_cast<const T *>(op->phi_work), static_cast<T *>(op->W),
                      static_cast<const T *>(op->tab->Kperm), pm, gm});
    src.push_back({op->packs, op->count_d});
    flags.push_back(op->tc_err);
    maxnp += ((long long)op->n * (op->n + 1) / 2 + 1) / 2;
  }
  if (maxnp > (1ll << 28)) return fail(ACE_ERR_ARG, "%lld packs in one queue", maxnp);
  std::vector<void *> temps;
  const ChainParams cp = chain_params(d, sizeof(T) == 8);
  ace_status s = run_chain_persistent<T>(op0, st, op0->tab, qops, {}, {}, src, (int)maxnp, builds, temps, cp);
  if (s == ACE_OK && group.size() > 1) {
    void *tmp = nullptr;
    cudaError_t e = cudaMallocAsync(&tmp, sizeof(int *) * flags.size(), st);
    if (e == cudaSuccess) {
      temps.push_back(tmp);
      e = host_upload(op0, tmp, flags.data(), sizeof(int *) * flags.size(), st);
    }
    if (e == cudaSuccess) e = ace::launch_flag_fanout(op0->tc_err, static_cast<int *const *>(tmp), (int)flags.size(), st);
    if (e != cudaSuccess) s = cuda_fail(e, "queue give-up flags");
    ++op0->launches;
  }
  for (void *p : temps) cudaFreeAsync(p, st);
  return s;
}

// Whether builds can run with their chains in device pack queues: the mixed form on grids with a
// persistent chain plan.
bool queue_eligible(int k, const ace_desc *desc) {
  for (int i = 0; i < k; ++i) {
    ace::PersistOps<float> q{};
    if (desc[i].prec == ACE_FP64 || !find_persist_ops<float>(desc[i].n[0], desc[i].n[1], desc[i].n[2], &q))
      return false;
  }
  return true;
}

// Builds screened on the device with their pair chains as one persistent launch per grid (no host
// wait between the screen and the chain): every build's screen on its lane, then per grid the
// queue chain on lane 0 once every build of that grid is screened, then each build's dense steps
// on its lane.  ops[i] is new (lane stream set, working type FP32, no given pairs); phi[i] device.
ace_status run_queued_builds(const std::vector<ace_op *> &ops, const void *const *phi, ace_dtype dtype,
                             cudaStream_t gs) {
  for (size_t i = 0; i < ops.size(); ++i) {
    ops[i]->queued = true;
    ace_status s = build_begin<float>(ops[i], phi[i], dtype);
    if (s != ACE_OK) return fail(s, "build %zu of %zu: %s", i, ops.size(), g_last_error.c_str());
  }
  std::vector<std::vector<ace_op *>> groups;
  for (ace_op *op : ops) {
    auto same = [&](const std::vector<ace_op *> &g) {
      return g[0]->desc.n[0] == op->desc.n[0] && g[0]->desc.n[1] == op->desc.n[1] && g[0]->desc.n[2] == op->desc.n[2];
    };
    auto it = std::find_if(groups.begin(), groups.end(), same);
    if (it == groups.end())
      groups.push_back({op});
    else
      it->push_back(op);
  }
  cudaEvent_t ev = nullptr;
  ACE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  struct EvGuard {
    cudaEvent_t e;
    ~EvGuard() { cudaEventDestroy(e); }
  } guard{ev};
  for (auto &g : groups) {
    for (ace_op *op : g)
      if (op->stream != gs) {
        ACE_CUDA(cudaEventRecord(ev, op->stream), "event");
        ACE_CUDA(cudaStreamWaitEvent(gs, ev, 0), "join");
      }
    ace_status s = run_queue_chain<float>(g, gs);
    if (s != ACE_OK) return s;
    ACE_CUDA(cudaEventRecord(ev, gs), "event");
    for (ace_op *op : g) {
      if (op->stream != gs) ACE_CUDA(cudaStreamWaitEvent(op->stream, ev, 0), "fork");
      ACE_CUDA(mark(op, 2, op->stream), "event record");
      s = build_dense<float>(op);
      if (s != ACE_OK) return s;
    }
  }
  return ACE_OK;
}

// Phase 3: after the stream has completed the build.
ace_status build_collect(ace_op *op) {
  const char *rb = static_cast<const char *>(op->readback);
  int flags[2];
  std::memcpy(flags, rb + 4, sizeof flags);
  std::memcpy(&op->energy, rb + 16, sizeof(double));
  op->status = flags[0];
  if (op->queued) op->npairs = *reinterpret_cast<const int *>(rb);  // the pair count, read back
  if (!op->graph) {
    for (int i = 0; i < 5; ++i) cudaEventElapsedTime(&op->stage_ms[i], op->ev[i], op->ev[i + 1]);
    cudaEventElapsedTime(&op->stage_ms[5], op->ev[0], op->ev[5]);
    pinned_put(op->readback, op->readback_bytes);
    op->readback = nullptr;
  }
  if (flags[1]) return fail(ACE_ERR_TIMEOUT, "a kernel gave up waiting (tensor-core pipeline, TMA copy or pair-chain task queue)");
  if (op->status >= 2000000) return fail(ACE_ERR_NONFINITE, "M has a non-finite entry");
  if (op->status >= 1000000)
    return fail(ACE_ERR_NOT_POSDEF, "-M is not positive definite: Cholesky pivot %d", op->status - 1000000);
  return ACE_OK;
}

// Buffer that a result of `count` T elements for the caller's `out` (dtype `dtype`, host or device)
// is computed into: `out` itself when it is 16-byte aligned device memory of type T, else a
// temporary that deliver_result passes on.
template <typename T>
ace_status result_target(void *out, ace_dtype dtype, long long count, cudaStream_t st, std::vector<void *> &temps,
                         T **res) {
  const bool same = (dtype == ACE_F64) == (sizeof(T) == 8);
  if (same && is_device_pointer(out) && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    *res = static_cast<T *>(out);
    return ACE_OK;
  }
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(T) * (size_t)count, st), "alloc out");
  temps.push_back(tmp);
  *res = static_cast<T *>(tmp);
  return ACE_OK;
}

// Pass a result from result_target's buffer to `out`: conversion to `dtype`, copy to the host, or
// copy to a misaligned device buffer, as needed (stream-ordered on st).
template <typename T>
ace_status deliver_result(T *res, void *out, ace_dtype dtype, long long count, cudaStream_t st,
                          std::vector<void *> &temps) {
  if (res == out) return ACE_OK;
  const bool same = (dtype == ACE_F64) == (sizeof(T) == 8);
  const bool host_out = !is_device_pointer(out);
  void *final_dev = res;
  const size_t out_bytes = (size_t)count * (dtype == ACE_F64 ? 8 : 4);
  if (!same) {
    void *conv = nullptr;
    if (!host_out) {
      conv = out;
    } else {
      ACE_CUDA(cudaMallocAsync(&conv, out_bytes, st), "alloc out conv");
      temps.push_back(conv);
    }
    if (dtype == ACE_F64)
      ACE_CUDA((ace::launch_convert<T, double>(res, static_cast<double *>(conv), count, 1.0, st)), "conv");
    else
      ACE_CUDA((ace::launch_convert<T, float>(res, static_cast<float *>(conv), count, 1.0, st)), "conv");
    final_dev = conv;
  }
  if (host_out)
    ACE_CUDA(cudaMemcpyAsync(out, final_dev, out_bytes, cudaMemcpyDeviceToHost, st), "device-to-host copy");
  else if (final_dev != out)
    ACE_CUDA(cudaMemcpyAsync(out, final_dev, out_bytes, cudaMemcpyDeviceToDevice, st), "unaligned output copy");
  return ACE_OK;
}

// C = dV xi^T psi (n x m FP64, device) for psi of m rows of op->N points (staged from any side)
template <typename T>
ace_status apply_coeffs_impl(const ace_op *op, const void *psi_in, ace_dtype dtype, int m, double *C, int *err_d,
                             cudaStream_t st, std::vector<void *> &temps) {
  ace_op tmpop;  // only for staging on `st`
  tmpop.stream = st;
  const T *psi = nullptr;
  ace_status s = stage_input<T>(&tmpop, psi_in, dtype, (long long)m * op->N, &psi, &temps);
  if (s != ACE_OK) return s;
  long nl = 0;
  ACE_CUDA(dense_gram<T>(static_cast<const T *>(op->xi), op->n, psi, m, op->N, op->dV, C, err_d, temps, st, &nl),
           "xi^T psi");
  return ACE_OK;
}

// out = -xi C (m rows of op->N points, any side) from C (n x m FP64, device)
template <typename T>
ace_status apply_finish_impl(const ace_op *op, const double *C, ace_dtype dtype, int m, void *out, int *err_d,
                             cudaStream_t st, std::vector<void *> &temps) {
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(T) * op->n * m, st), "alloc A");
  temps.push_back(tmp);
  T *A = static_cast<T *>(tmp);
  ACE_CUDA(ace::launch_transpose_scale<T>(C, op->n, m, -1.0, A, st), "transpose");
  T *res = nullptr;
  ace_status s = result_target<T>(out, dtype, (long long)m * op->N, st, temps, &res);
  if (s != ACE_OK) return s;
  long nl = 0;
  ACE_CUDA(dense_left_mul<T>(A, m, op->n, static_cast<const T *>(op->xi), op->N, res, err_d, st, &nl), "xi C");
  return deliver_result<T>(res, out, dtype, (long long)m * op->N, st, temps);
}

// Frees the temporaries of a call in stream order when it leaves.
struct TempGuard {
  std::vector<void *> *v;
  cudaStream_t s;
  ~TempGuard() {
    for (void *p : *v) cudaFreeAsync(p, s);
  }
};

// Reads the give-up flag of the call's kernels after the stream has finished them.
ace_status finish_flag(int *err_d, cudaStream_t st, const char *what) {
  int err_h = 0;
  ACE_CUDA(cudaMemcpyAsync(&err_h, err_d, sizeof(int), cudaMemcpyDeviceToHost, st), "flag readback");
  ACE_CUDA(cudaStreamSynchronize(st), what);
  if (err_h) return fail(ACE_ERR_TIMEOUT, "a kernel gave up waiting (tensor-core pipeline or TMA copy)");
  return ACE_OK;
}

template <typename T>
ace_status apply_impl(const ace_op *op, const void *psi_in, ace_dtype dtype, int m, void *out, cudaStream_t st) {
  const int n = op->n;
  std::vector<void *> temps;
  TempGuard guard{&temps, st};
  void *tmp = nullptr;
  // C = dV xi psi^T  (n x m, FP64 across chunks)
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(double) * n * m, st), "alloc C");
  temps.push_back(tmp);
  double *C = static_cast<double *>(tmp);
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(int), st), "alloc flag");
  temps.push_back(tmp);
  int *err_d = static_cast<int *>(tmp);
  ACE_CUDA(cudaMemsetAsync(err_d, 0, sizeof(int), st), "zero flag");
  ace_status s = apply_coeffs_impl<T>(op, psi_in, dtype, m, C, err_d, st, temps);
  if (s != ACE_OK) return s;
  s = apply_finish_impl<T>(op, C, dtype, m, out, err_d, st, temps);
  if (s != ACE_OK) return s;
  return finish_flag(err_d, st, "apply");
}

// SCDM localisation of n orbitals of N points: pivots and Loewdin factor (scdm.cu), then
// Phi = U^T Psi by the dense left multiply of the working type.
template <typename T>
ace_status scdm_impl(int n, long long N, const void *psi_in, ace_dtype dtype, void *phi_out, int *piv_host,
                     double *u_host, cudaStream_t st, long *launches) {
  std::vector<void *> temps;
  struct TempGuard {
    std::vector<void *> *v;
    cudaStream_t s;
    ~TempGuard() {
      for (void *p : *v) cudaFreeAsync(p, s);
    }
  } guard{&temps, st};
  ace_op tmpop;  // only for staging on `st`
  tmpop.stream = st;
  const T *psi = nullptr;
  ace_status s = stage_input<T>(&tmpop, psi_in, dtype, (long long)n * N, &psi, &temps);
  if (s != ACE_OK) return s;
  *launches += tmpop.launches;
  void *ws = nullptr;
  ACE_CUDA(cudaMallocAsync(&ws, ace::scdm_workspace_bytes(n, N, sizeof(T)) + 256, st), "alloc SCDM workspace");
  temps.push_back(ws);
  int *err_d = reinterpret_cast<int *>(static_cast<char *>(ws) + ace::scdm_workspace_bytes(n, N, sizeof(T)));
  ACE_CUDA(cudaMemsetAsync(err_d, 0, sizeof(int), st), "zero flag");
  ace::ScdmResult r{};
  ACE_CUDA(ace::launch_scdm<T>(psi, n, N, ws, st, launches, &r), "SCDM selection");
  T *res = nullptr;
  s = result_target<T>(phi_out, dtype, (long long)n * N, st, temps, &res);
  if (s != ACE_OK) return s;
  ACE_CUDA(dense_left_mul<T>(static_cast<const T *>(r.Ut), n, n, psi, N, res, err_d, st, launches), "U^T Psi");
  s = deliver_result<T>(res, phi_out, dtype, (long long)n * N, st, temps);
  if (s != ACE_OK) return s;
  if ((dtype == ACE_F64) != (sizeof(T) == 8)) ++*launches;  // the conversion to the caller's dtype
  const int nit = ace::scdm_max_iterations();
  std::vector<double> dev(nit);
  std::vector<int> piv(n);
  int err_h = 0, dep_h = 0;
  ACE_CUDA(cudaMemcpyAsync(&dep_h, r.dependent, sizeof(int), cudaMemcpyDeviceToHost, st), "readback");
  ACE_CUDA(cudaMemcpyAsync(dev.data(), r.dev, sizeof(double) * nit, cudaMemcpyDeviceToHost, st), "readback");
  ACE_CUDA(cudaMemcpyAsync(piv.data(), r.piv, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "readback");
  if (u_host) ACE_CUDA(cudaMemcpyAsync(u_host, r.U, sizeof(double) * n * n, cudaMemcpyDeviceToHost, st), "readback");
  ACE_CUDA(cudaMemcpyAsync(&err_h, err_d, sizeof(int), cudaMemcpyDeviceToHost, st), "flag readback");
  ACE_CUDA(cudaStreamSynchronize(st), "SCDM");
  if (err_h) return fail(ACE_ERR_TIMEOUT, "a tensor-core kernel gave up waiting for its MMAs");
  if (piv_host) std::copy(piv.begin(), piv.end(), piv_host);
  // the last Newton-Schulz iteration that ran decides convergence
  double last = dev[0];
  for (int it = 1; it < nit && dev[it] != 0.0; ++it) last = dev[it];
  if (dep_h) return fail(ACE_ERR_NOT_POSDEF, "psi has rank < norb: a selected column lies in the span of the others");
  if (!(last < 1e-8))
    return fail(ACE_ERR_NOT_POSDEF, "the selected columns are linearly dependent (Newton-Schulz residual %.3g)", last);
  return ACE_OK;
}

size_t item_bytes(const ace_op *op, int what) {
  const size_t nn = (size_t)op->n * op->n;
  switch (what) {
    case ACE_GET_XI:
    case ACE_GET_W: return op->esz * (size_t)op->n * op->N;
    case ACE_GET_M:
    case ACE_GET_M_RAW:
    case ACE_GET_L:
    case ACE_GET_OVERLAP: return sizeof(double) * nn;
    case ACE_GET_PAIRS: return sizeof(int2) * (size_t)op->npairs;
    default: return 0;
  }
}

}  // namespace

namespace ace {
void set_last_error(const char *msg) { g_last_error = msg; }
}  // namespace ace

namespace {
// Sorted, checked copy of a caller's pair list: i <= j, 0 <= i, j < norb, each pair once.
ace_status checked_pairs(const ace_desc *desc, const int *pairs_host, long npairs, std::vector<int2> &given) {
  if (npairs < 0 || (npairs > 0 && !pairs_host)) return fail(ACE_ERR_ARG, "bad pair list");
  const long maxp = (long)desc->norb * (desc->norb + 1) / 2;
  if (npairs > maxp) return fail(ACE_ERR_ARG, "%ld pairs for %d orbitals", npairs, desc->norb);
  given.assign((size_t)npairs, make_int2(0, 0));
  for (long p = 0; p < npairs; ++p) {
    int i = pairs_host[2 * p], j = pairs_host[2 * p + 1];
    if (i > j) std::swap(i, j);
    if (i < 0 || j >= desc->norb) return fail(ACE_ERR_ARG, "pair %ld = (%d, %d) outside [0, %d)", p, i, j, desc->norb);
    given[(size_t)p] = make_int2(i, j);
  }
  std::sort(given.begin(), given.end(), [](int2 a, int2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); });
  for (size_t p = 1; p < given.size(); ++p)
    if (given[p].x == given[p - 1].x && given[p].y == given[p - 1].y)
      return fail(ACE_ERR_ARG, "pair (%d, %d) listed twice", given[p].x, given[p].y);
  return ACE_OK;
}

// The pair chain of a begun build with a given pair list, into W_out (the caller's buffer when it
// is device memory, else through a device buffer and a copy); no M, no Cholesky.
template <typename T>
ace_status exchange_w_impl(ace_op *op, void *W_out) {
  const int count = *static_cast<const int *>(op->readback);
  op->npairs = count;
  const int2 *ph = reinterpret_cast<const int2 *>(static_cast<const char *>(op->readback) + 32);
  op->pairs_h.assign(ph, ph + count);
  const size_t bytes = op->esz * (size_t)op->n * op->N;
  const bool direct = is_device_pointer(W_out);
  if (direct)
    op->W = W_out;
  else
    ACE_CUDA(op_alloc(op, &op->W, bytes), "alloc W");
  ace_status s = run_chain<T>(op, static_cast<const T *>(op->phi_work), count);
  if (s == ACE_OK && !direct)
    ACE_CUDA(cudaMemcpyAsync(W_out, op->W, bytes, cudaMemcpyDefault, op->stream), "W copy");
  for (void *p : op->temps) cudaFreeAsync(p, op->stream);
  op->temps.clear();
  if (direct) op->W = nullptr;  // the caller's buffer
  if (s != ACE_OK) return s;
  return finish_flag(op->tc_err, op->stream, "exchange W");
}

ace_status working_dtype(const ace_desc *desc, ace_dtype dtype) {
  if ((desc->prec == ACE_FP64) != (dtype == ACE_F64))
    return fail(ACE_ERR_ARG, "dtype %d is not the working type of precision %d", (int)dtype, (int)desc->prec);
  return ACE_OK;
}
}  // namespace

extern "C" {

const char *ace_last_error(void) { return g_last_error.c_str(); }

int ace_grid_supported(int n_axis, ace_precision prec) {
  (void)prec;
  return ace::pass_length_supported(n_axis) ? 1 : 0;
}

}  // extern "C"

namespace {

ace_op *new_op(const ace_desc *desc, cudaStream_t st, ace_status *status) {
  ace_op *op = new (std::nothrow) ace_op();
  if (!op) {
    *status = fail(ACE_ERR_OOM, "host allocation failed");
    return nullptr;
  }
  op->stream = st;
  op->desc = *desc;
  op->n = desc->norb;
  op->N = (long long)desc->n[0] * desc->n[1] * desc->n[2];
  const double *A = &desc->lattice[0][0];
  const double vol = std::fabs(A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                               A[2] * (A[3] * A[7] - A[4] * A[6]));
  op->dV = vol / (double)op->N;
  op->fp64 = desc->prec == ACE_FP64;
  op->esz = op->fp64 ? 8 : 4;
  cudaError_t e = cudaGetDevice(&op->dev);
  if (e == cudaSuccess) e = prepare_pool(op->dev);
  if (e != cudaSuccess) {
    delete op;
    *status = cuda_fail(e, "device setup");
    return nullptr;
  }
  *status = ACE_OK;
  return op;
}

ace_status begin_any(ace_op *op, const void *phi, ace_dtype dt) {
  return op->fp64 ? build_begin<double>(op, phi, dt) : build_begin<float>(op, phi, dt);
}
ace_status finish_any(ace_op *op) { return op->fp64 ? build_finish<double>(op) : build_finish<float>(op); }

bool keeps_handle(ace_status s) { return s == ACE_OK || s == ACE_ERR_NOT_POSDEF || s == ACE_ERR_NONFINITE; }

}  // namespace

extern "C" {

ace_status ace_build(const ace_desc *desc, const void *phi, ace_dtype dtype, void *cuda_stream, ace_op **out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  ace_status s = check_desc(desc);
  if (s != ACE_OK) return s;
  if (!phi) return fail(ACE_ERR_ARG, "phi is NULL");
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  ace_op *op = new_op(desc, static_cast<cudaStream_t>(cuda_stream), &s);
  if (!op) return s;
  s = begin_any(op, phi, dtype);
  if (s == ACE_OK) {
    cudaError_t e = cudaEventSynchronize(op->ev[1]);
    s = e == cudaSuccess ? finish_any(op) : cuda_fail(e, "pair list readback");
  }
  if (s == ACE_OK) {
    cudaError_t e = cudaStreamSynchronize(op->stream);
    s = e == cudaSuccess ? build_collect(op) : cuda_fail(e, "build");
  }
  if (keeps_handle(s)) {
    *out = op;
    return s;
  }
  cudaStreamSynchronize(op->stream);
  ace_destroy(op);
  return s;
}

ace_status ace_exchange_w(const ace_desc *desc, const void *phi, ace_dtype dtype, const int *pairs_host, long npairs,
                          void *W, void *cuda_stream) {
  ace_status s = check_desc(desc);
  if (s != ACE_OK) return s;
  if (!phi || !W) return fail(ACE_ERR_ARG, "NULL argument");
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  std::vector<int2> given;
  s = checked_pairs(desc, pairs_host, npairs, given);
  if (s != ACE_OK) return s;
  ace_op *op = new_op(desc, static_cast<cudaStream_t>(cuda_stream), &s);
  if (!op) return s;
  op->given.swap(given);
  op->use_given = true;
  s = begin_any(op, phi, dtype);
  if (s == ACE_OK) {
    cudaError_t e = cudaEventSynchronize(op->ev[1]);
    if (e != cudaSuccess)
      s = cuda_fail(e, "pair upload");
    else
      s = op->fp64 ? exchange_w_impl<double>(op, W) : exchange_w_impl<float>(op, W);
  }
  cudaStreamSynchronize(op->stream);
  ace_destroy(op);
  return s;
}

ace_status ace_m_partial(const ace_desc *desc, const void *phi_slab, const void *W_slab, ace_dtype dtype,
                         long long npts, double *M, void *cuda_stream) {
  ace_status s = check_desc(desc);
  if (s != ACE_OK) return s;
  if (!phi_slab || !W_slab || !M) return fail(ACE_ERR_ARG, "NULL argument");
  if (npts < 1) return fail(ACE_ERR_ARG, "npts = %lld < 1", npts);
  if ((s = working_dtype(desc, dtype)) != ACE_OK) return s;
  if (!is_device_pointer(phi_slab) || !is_device_pointer(W_slab) || !is_device_pointer(M))
    return fail(ACE_ERR_ARG, "phi_slab, W_slab and M must be device memory");
  ace_op *op = new_op(desc, static_cast<cudaStream_t>(cuda_stream), &s);  // dV of the whole grid
  if (!op) return s;
  const double dV = op->dV;
  const int n = op->n;
  ace_destroy(op);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<void *> temps;
  TempGuard guard{&temps, st};
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(int), st), "alloc flag");
  temps.push_back(tmp);
  int *err_d = static_cast<int *>(tmp);
  ACE_CUDA(cudaMemsetAsync(err_d, 0, sizeof(int), st), "zero flag");
  long nl = 0;
  if (dtype == ACE_F64)
    ACE_CUDA(dense_gram<double>(static_cast<const double *>(phi_slab), n, static_cast<const double *>(W_slab), n, npts,
                                -dV, M, err_d, temps, st, &nl),
             "M partial");
  else
    ACE_CUDA(dense_gram<float>(static_cast<const float *>(phi_slab), n, static_cast<const float *>(W_slab), n, npts,
                               -dV, M, err_d, temps, st, &nl),
             "M partial");
  return finish_flag(err_d, st, "M partial");
}

ace_status ace_build_from_m(const ace_desc *desc, const double *M, const void *W_slab, ace_dtype dtype, long long npts,
                            void *cuda_stream, ace_op **out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  ace_status s = check_desc(desc);
  if (s != ACE_OK) return s;
  if (!M || !W_slab) return fail(ACE_ERR_ARG, "NULL argument");
  if (npts < 1) return fail(ACE_ERR_ARG, "npts = %lld < 1", npts);
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  ace_op *op = new_op(desc, static_cast<cudaStream_t>(cuda_stream), &s);
  if (!op) return s;
  op->N = npts;  // the slab's points; dV stays that of the whole grid
  const int n = op->n;
  cudaStream_t st = op->stream;
  auto run = [&]() -> ace_status {
    for (int i = 0; i < 6; ++i) ACE_CUDA(cudaEventCreate(&op->ev[i]), "event create");
    for (int i = 0; i < 4; ++i) ACE_CUDA(mark(op, i, st), "event record");
    ACE_CUDA(op_alloc(op, &op->status_d, sizeof(int) * 4), "alloc status");
    op->tc_err = op->status_d + 1;
    ACE_CUDA(cudaMemsetAsync(op->status_d, 0, sizeof(int) * 4, st), "zero status");
    ACE_CUDA(op_alloc(op, &op->energy_d, sizeof(double) * 2), "alloc energy");
    ACE_CUDA(op_alloc(op, &op->M_raw, sizeof(double) * n * n), "alloc M_raw");
    ACE_CUDA(op_alloc(op, &op->M, sizeof(double) * n * n), "alloc M");
    ACE_CUDA(op_alloc(op, &op->L, sizeof(double) * n * n), "alloc L");
    ACE_CUDA(op_alloc(op, &op->Linv, sizeof(double) * n * n), "alloc Linv");
    ACE_CUDA(pinned_get(32, &op->readback), "pinned readback");
    op->readback_bytes = 32;
    ACE_CUDA(cudaMemcpyAsync(op->M_raw, M, sizeof(double) * n * n, cudaMemcpyDefault, st), "M copy");
    if (op->fp64) {
      const double *W = nullptr;
      ace_status r = stage_input<double>(op, W_slab, dtype, (long long)n * npts, &W, &op->temps);
      return r != ACE_OK ? r : factor_and_project<double>(op, W);
    }
    const float *W = nullptr;
    ace_status r = stage_input<float>(op, W_slab, dtype, (long long)n * npts, &W, &op->temps);
    return r != ACE_OK ? r : factor_and_project<float>(op, W);
  };
  s = run();
  if (s == ACE_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    s = e == cudaSuccess ? build_collect(op) : cuda_fail(e, "build from M");
  }
  if (keeps_handle(s)) {
    *out = op;
    return s;
  }
  cudaStreamSynchronize(st);
  ace_destroy(op);
  return s;
}

ace_status ace_apply_coeffs(const ace_op *op, const void *psi, ace_dtype dtype, int m, double *C, void *cuda_stream) {
  if (!op || !psi || !C) return fail(ACE_ERR_ARG, "NULL argument");
  if (m < 1) return fail(ACE_ERR_ARG, "m = %d < 1", m);
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (op->status != 0) return fail(ACE_ERR_NOT_POSDEF, "operator build did not complete (status %d)", op->status);
  if (!is_device_pointer(C)) return fail(ACE_ERR_ARG, "C must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<void *> temps;
  TempGuard guard{&temps, st};
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(int), st), "alloc flag");
  temps.push_back(tmp);
  int *err_d = static_cast<int *>(tmp);
  ACE_CUDA(cudaMemsetAsync(err_d, 0, sizeof(int), st), "zero flag");
  ace_status s = op->fp64 ? apply_coeffs_impl<double>(op, psi, dtype, m, C, err_d, st, temps)
                          : apply_coeffs_impl<float>(op, psi, dtype, m, C, err_d, st, temps);
  return s != ACE_OK ? s : finish_flag(err_d, st, "apply coefficients");
}

ace_status ace_apply_finish(const ace_op *op, const double *C, ace_dtype dtype, int m, void *out, void *cuda_stream) {
  if (!op || !C || !out) return fail(ACE_ERR_ARG, "NULL argument");
  if (m < 1) return fail(ACE_ERR_ARG, "m = %d < 1", m);
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (op->status != 0) return fail(ACE_ERR_NOT_POSDEF, "operator build did not complete (status %d)", op->status);
  if (!is_device_pointer(C)) return fail(ACE_ERR_ARG, "C must be device memory");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  std::vector<void *> temps;
  TempGuard guard{&temps, st};
  void *tmp = nullptr;
  ACE_CUDA(cudaMallocAsync(&tmp, sizeof(int), st), "alloc flag");
  temps.push_back(tmp);
  int *err_d = static_cast<int *>(tmp);
  ACE_CUDA(cudaMemsetAsync(err_d, 0, sizeof(int), st), "zero flag");
  ace_status s = op->fp64 ? apply_finish_impl<double>(op, C, dtype, m, out, err_d, st, temps)
                          : apply_finish_impl<float>(op, C, dtype, m, out, err_d, st, temps);
  return s != ACE_OK ? s : finish_flag(err_d, st, "apply finish");
}

ace_status ace_build_pairs(const ace_desc *desc, const void *phi, ace_dtype dtype, const int *pairs_host, long npairs,
                           void *cuda_stream, ace_op **out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  ace_status s = check_desc(desc);
  if (s != ACE_OK) return s;
  if (!phi) return fail(ACE_ERR_ARG, "phi is NULL");
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  std::vector<int2> given;
  s = checked_pairs(desc, pairs_host, npairs, given);
  if (s != ACE_OK) return s;
  ace_op *op = new_op(desc, static_cast<cudaStream_t>(cuda_stream), &s);
  if (!op) return s;
  op->given.swap(given);
  op->use_given = true;
  s = begin_any(op, phi, dtype);
  if (s == ACE_OK) {
    cudaError_t e = cudaEventSynchronize(op->ev[1]);
    s = e == cudaSuccess ? finish_any(op) : cuda_fail(e, "pair upload");
  }
  if (s == ACE_OK) {
    cudaError_t e = cudaStreamSynchronize(op->stream);
    s = e == cudaSuccess ? build_collect(op) : cuda_fail(e, "build");
  }
  if (keeps_handle(s)) {
    *out = op;
    return s;
  }
  cudaStreamSynchronize(op->stream);
  ace_destroy(op);
  return s;
}

// Builds go on stream lanes forked from `cuda_stream` (one by default, up to four): all screens
// first, one wait for the pair lists, then every build's chain on its lane and its dense steps on
// the lane's tail stream (so that they run beside the next build's chain; ACE_BATCH_TAIL=0 keeps
// them on the lane), then one join back into `cuda_stream`.
ace_status ace_build_batched(int k, const ace_desc *desc, const void *const *phi, ace_dtype dtype, void *cuda_stream,
                             ace_op **out) {
  if (k < 0 || (k > 0 && (!desc || !phi || !out))) return fail(ACE_ERR_ARG, "bad batched arguments");
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  for (int i = 0; i < k; ++i) out[i] = nullptr;
  for (int i = 0; i < k; ++i) {
    ace_status s = check_desc(&desc[i]);
    if (s != ACE_OK) return fail(s, "build %d of %d: %s", i, k, g_last_error.c_str());
    if (!phi[i]) return fail(ACE_ERR_ARG, "build %d of %d: phi is NULL", i, k);
  }
  if (k == 0) return ACE_OK;
  cudaStream_t user = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  ACE_CUDA(cudaGetDevice(&dev), "device");
  // one lane by default: each build's chain fills the GPU through its side streams, and concurrent
  // builds only share the L2 (measured on the 24 uneven builds: 37.5 builds/s on one lane, 35.5 on
  // four)
  const int lanes = std::min(kLanes, std::max(1, std::min(k, env_int("ACE_BATCH_LANES", 1))));
  cudaStream_t lane_st[kLanes], tail_st[kLanes];
  const bool queue = env_int("ACE_BATCH_QUEUE", 0) != 0 && queue_eligible(k, desc);
  const bool tail = !queue && env_int("ACE_BATCH_TAIL", 1) != 0;
  cudaEvent_t fork = nullptr;
  ACE_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "event");
  ACE_CUDA(cudaEventRecord(fork, user), "event");
  for (int l = 0; l < lanes; ++l) {
    ACE_CUDA(get_side_stream(dev, kSide * kLanes + l, &lane_st[l]), "lane stream");
    ACE_CUDA(cudaStreamWaitEvent(lane_st[l], fork, 0), "fork");
    if (tail) {
      ACE_CUDA(get_side_stream(dev, (kSide + 2) * kLanes + l, &tail_st[l]), "tail stream");
      ACE_CUDA(cudaStreamWaitEvent(tail_st[l], fork, 0), "fork");
    }
  }
  ace_status s = ACE_OK;
  int failed = -1;
  for (int i = 0; i < k && s == ACE_OK; ++i) {
    ace_op *op = new_op(&desc[i], lane_st[i % lanes], &s);
    if (!op) {
      failed = i;
      break;
    }
    op->lane = i % lanes;
    if (tail) op->tail = tail_st[i % lanes];
    out[i] = op;
    if (!queue) {
      s = begin_any(op, phi[i], dtype);
      if (s != ACE_OK) failed = i;
    }
  }
  if (queue && s == ACE_OK) {
    // one persistent chain launch per grid over the builds' device pack lists, no host wait
    std::vector<ace_op *> ops(out, out + k);
    s = run_queued_builds(ops, phi, dtype, lane_st[0]);
    if (s != ACE_OK) failed = 0;
  }
  for (int i = 0; i < k && s == ACE_OK && !queue; ++i) {
    cudaError_t e = cudaEventSynchronize(out[i]->ev[1]);
    s = e == cudaSuccess ? finish_any(out[i]) : cuda_fail(e, "pair list readback");
    if (s != ACE_OK) failed = i;
  }
  for (int l = 0; l < lanes; ++l) {
    cudaEventRecord(fork, lane_st[l]);
    cudaStreamWaitEvent(user, fork, 0);
    if (tail) {
      cudaEventRecord(fork, tail_st[l]);
      cudaStreamWaitEvent(user, fork, 0);
    }
  }
  for (int i = 0; i < k; ++i)
    if (out[i]) cudaStreamSynchronize(out[i]->stream);
  cudaEventDestroy(fork);
  for (int i = 0; i < k && s == ACE_OK; ++i) {
    s = build_collect(out[i]);
    if (s != ACE_OK) failed = i;
  }
  if (s != ACE_OK) {
    std::string msg = g_last_error;
    for (int j = 0; j < k; ++j) {
      if (out[j]) ace_destroy(out[j]);
      out[j] = nullptr;
    }
    return fail(s, "build %d of %d: %s", failed, k, msg.c_str());
  }
  // the handles keep their lane stream for ace_destroy; later calls take a stream argument
  return ACE_OK;
}

ace_status ace_apply(const ace_op *op, const void *psi, ace_dtype dtype, int m, void *out, void *cuda_stream) {
  if (!op || !psi || !out) return fail(ACE_ERR_ARG, "NULL argument");
  if (m < 1) return fail(ACE_ERR_ARG, "m = %d < 1", m);
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (op->status != 0) return fail(ACE_ERR_NOT_POSDEF, "operator build did not complete (status %d)", op->status);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  return op->fp64 ? apply_impl<double>(op, psi, dtype, m, out, st) : apply_impl<float>(op, psi, dtype, m, out, st);
}

ace_status ace_scdm(int norb, long long npts, ace_precision prec, const void *psi, ace_dtype dtype, void *phi,
                    int *piv_host, double *u_host, void *cuda_stream, long *launches) {
  if (!psi || !phi) return fail(ACE_ERR_ARG, "NULL argument");
  if (norb < 1 || norb > 1024) return fail(ACE_ERR_ARG, "norb = %d outside [1, 1024]", norb);
  if (npts < norb || npts > 0x7fffffffLL) return fail(ACE_ERR_ARG, "npts = %lld outside [norb, 2^31 - 1]", npts);
  if (prec != ACE_FP64 && prec != ACE_MIXED) return fail(ACE_ERR_ARG, "unknown precision %d", (int)prec);
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  if (is_device_pointer(psi) != is_device_pointer(phi)) return fail(ACE_ERR_ARG, "psi and phi on different sides");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  long nl = 0;
  const ace_status s = prec == ACE_FP64 ? scdm_impl<double>(norb, npts, psi, dtype, phi, piv_host, u_host, st, &nl)
                                        : scdm_impl<float>(norb, npts, psi, dtype, phi, piv_host, u_host, st, &nl);
  if (launches) *launches = nl;
  return s;
}

ace_status exchange_energy(const ace_op *op, double *ex_hartree) {
  if (!op || !ex_hartree) return fail(ACE_ERR_ARG, "NULL argument");
  *ex_hartree = op->energy;
  return ACE_OK;
}

ace_status ace_get_size(const ace_op *op, int what, size_t *bytes) {
  if (!op || !bytes) return fail(ACE_ERR_ARG, "NULL argument");
  const size_t b = item_bytes(op, what);
  if (b == 0 && what != ACE_GET_PAIRS) return fail(ACE_ERR_ARG, "unknown item %d", what);
  *bytes = b;
  return ACE_OK;
}

ace_status ace_get(const ace_op *op, int what, void *dst, size_t bytes, void *cuda_stream) {
  if (!op || (!dst && bytes)) return fail(ACE_ERR_ARG, "NULL argument");
  const size_t want = item_bytes(op, what);
  if (want == 0 && what != ACE_GET_PAIRS) return fail(ACE_ERR_ARG, "unknown item %d", what);
  if (bytes != want) return fail(ACE_ERR_ARG, "item %d has %zu bytes, %zu given", what, want, bytes);
  if (bytes == 0) return ACE_OK;
  const void *src = nullptr;
  switch (what) {
    case ACE_GET_XI: src = op->xi; break;
    case ACE_GET_W: src = op->W; break;
    case ACE_GET_M: src = op->M; break;
    case ACE_GET_M_RAW: src = op->M_raw; break;
    case ACE_GET_L: src = op->L; break;
    case ACE_GET_PAIRS: src = op->pairs; break;
    case ACE_GET_OVERLAP: src = op->O_sym; break;
  }
  if (!src) return fail(ACE_ERR_ARG, "item %d is not available", what);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  ACE_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st), "ace_get copy");
  ACE_CUDA(cudaStreamSynchronize(st), "ace_get");
  return ACE_OK;
}

ace_status ace_pair_count(const ace_op *op, long *npairs) {
  if (!op || !npairs) return fail(ACE_ERR_ARG, "NULL argument");
  *npairs = op->npairs;
  return ACE_OK;
}

ace_status ace_kernel_launches(const ace_op *op, long *launches) {
  if (!op || !launches) return fail(ACE_ERR_ARG, "NULL argument");
  *launches = op->launches;
  return ACE_OK;
}

ace_status ace_stage_times(const ace_op *op, float ms[6]) {
  if (!op || !ms) return fail(ACE_ERR_ARG, "NULL argument");
  for (int i = 0; i < 6; ++i) ms[i] = op->stage_ms[i];
  return ACE_OK;
}

ace_status ace_autotune(const ace_desc *desc, const void *phi, ace_dtype dtype, void *cuda_stream, int *params) {
  ace_status s = check_desc(desc);
  if (s != ACE_OK) return s;
  if (!phi) return fail(ACE_ERR_ARG, "phi is NULL");
  if (dtype != ACE_F32 && dtype != ACE_F64) return fail(ACE_ERR_ARG, "unknown dtype %d", (int)dtype);
  ace_op *op = new_op(desc, static_cast<cudaStream_t>(cuda_stream), &s);
  if (!op) return s;
  struct Guard {
    ace_op *op;
    ~Guard() {
      cudaStreamSynchronize(op->stream);
      ace_destroy(op);
    }
  } guard{op};
  s = begin_any(op, phi, dtype);
  if (s != ACE_OK) return s;
  ACE_CUDA(cudaEventSynchronize(op->ev[1]), "pair list readback");
  const int count = *static_cast<const int *>(op->readback);
  op->npairs = count;
  const int2 *ph = reinterpret_cast<const int2 *>(static_cast<const char *>(op->readback) + 32);
  op->pairs_h.assign(ph, ph + count);
  ChainParams best = chain_params(*desc, op->fp64);
  auto run = [&](auto tag) -> ace_status {
    using T = decltype(tag);
    ace::PlaneOps<T> pops{};
    if (count == 0 || !find_plane_ops<T>(desc->n[1], desc->n[2], &pops) || !ace::conv_length_supported(desc->n[0]))
      return ACE_OK;  // nothing to tune
    ACE_CUDA(op_alloc(op, &op->W, op->esz * (size_t)op->n * op->N), "alloc W");
    const T *phi_w = static_cast<const T *>(op->phi_work);
    // a sample long enough (about 40% of a 128-orbital build on 96^3) for the L2 reuse of the
    // blocked pack order and of the persisting scratch window to show in the timing
    const int sample = std::min((count + 1) / 2, 480);
    cudaEvent_t e0, e1;
    ACE_CUDA(cudaEventCreate(&e0), "event");
    ACE_CUDA(cudaEventCreate(&e1), "event");
    float best_ms = 1e30f;
    const int Bs[5] = {1, 2, 3, 4, 6}, Ss[3] = {2, 4, 8}, Ps[2] = {0, 60}, Rs[4] = {1, 2, 4, 8};
    for (int ri = 0; ri < 4; ++ri)
    for (int bi = 0; bi < 5; ++bi)
      for (int si = 0; si < 3; ++si)
        for (int pi = 0; pi < 2; ++pi) {
          ChainParams c;
          c.G = 1;
          c.B = Bs[bi];
          c.streams = Ss[si];
          c.persist_mb = Ps[pi];
          c.RB = Rs[ri];
          float t[2];
          for (int rep = 0; rep < 2; ++rep) {
            std::vector<void *> tmp;
            ACE_CUDA(cudaEventRecord(e0, op->stream), "event");
            ace_status r = run_chain_plane<T>(op, phi_w, op->tab, pops, count, tmp, c, sample);
            ACE_CUDA(cudaEventRecord(e1, op->stream), "event");
            for (void *q : tmp) cudaFreeAsync(q, op->stream);
            if (r != ACE_OK) return r;
            ACE_CUDA(cudaEventSynchronize(e1), "tuning run");
            cudaEventElapsedTime(&t[rep], e0, e1);
          }
          const float ms = std::min(t[0], t[1]);
          if (ms < best_ms) {
            best_ms = ms;
            best = c;
          }
        }
    // the pencil tile of the axis-1 pass (three compiled for the FP32 form) on the best settings
    if (sizeof(T) == 4) {
      const ChainParams base = best;
      for (int v : {1, 2}) {
        ChainParams c = base;
        c.conv = v;
        float t[2];
        for (int rep = 0; rep < 2; ++rep) {
          std::vector<void *> tmp;
          ACE_CUDA(cudaEventRecord(e0, op->stream), "event");
          ace_status r = run_chain_plane<T>(op, phi_w, op->tab, pops, count, tmp, c, sample);
          ACE_CUDA(cudaEventRecord(e1, op->stream), "event");
          for (void *q : tmp) cudaFreeAsync(q, op->stream);
          if (r != ACE_OK) return r;
          ACE_CUDA(cudaEventSynchronize(e1), "tuning run");
          cudaEventElapsedTime(&t[rep], e0, e1);
        }
        const float ms = std::min(t[0], t[1]);
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    }
    // the persistent chain on the same sample, for a few queue lags
    ace::PersistOps<T> qops{};
    if (find_persist_ops<T>(desc->n[0], desc->n[1], desc->n[2], &qops)) {
      std::vector<int4> packs;
      form_packs(op->pairs_h, best.RB, packs);
      packs.resize(std::min<size_t>(packs.size(), (size_t)sample));
      const std::vector<ace::ChainBuild<T>> one{
          {phi_w, static_cast<T *>(op->W), static_cast<const T *>(op->tab->Kperm), op->pmax, op->gmax}};
      for (int lag : {2, 3, 4}) {
        ChainParams c = best;
        c.persistent = 1;
        c.lag = lag;
        float t[2];
        for (int rep = 0; rep < 2; ++rep) {
          std::vector<void *> tmp;
          ACE_CUDA(cudaEventRecord(e0, op->stream), "event");
          ace_status r = run_chain_persistent<T>(op, op->stream, op->tab, qops, packs, {}, {}, 0, one, tmp, c);
          ACE_CUDA(cudaEventRecord(e1, op->stream), "event");
          for (void *q : tmp) cudaFreeAsync(q, op->stream);
          if (r != ACE_OK) return r;
          ACE_CUDA(cudaEventSynchronize(e1), "tuning run");
          cudaEventElapsedTime(&t[rep], e0, e1);
        }
        const float ms = std::min(t[0], t[1]);
        if (ms < best_ms) {
          best_ms = ms;
          best = c;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tune_store(TuneKey{desc->n[0], desc->n[1], desc->n[2], op->fp64 ? 1 : 0}, best);
    return ACE_OK;
  };
  s = op->fp64 ? run(double{}) : run(float{});
  if (s != ACE_OK) return s;
  if (params) {
    params[0] = best.G;
    params[1] = best.B;
    params[2] = best.streams;
    params[3] = best.persist_mb;
    params[4] = best.RB;
    params[5] = best.persistent ? best.lag : 0;
    params[6] = best.conv;
  }
  return ACE_OK;
}

void ace_destroy(ace_op *op) {
  if (!op || op->graph) return;  // handles of a graph belong to it (ace_graph_destroy)
  destroy_op(op);
}

}  // extern "C"

namespace {

void destroy_op(ace_op *op) {
  for (void *p : op->temps) cudaFreeAsync(p, op->stream);
  op->temps.clear();
  op_free_all(op);
  if (op->readback) {
    cudaStreamSynchronize(op->stream);  // an unfinished build may still copy into it
    pinned_put(op->readback, op->readback_bytes);
  }
  for (int i = 0; i < 6; ++i)
    if (op->ev[i]) cudaEventDestroy(op->ev[i]);
  for (auto &b : op->staged) cudaFreeHost(b.first);
  delete op;
}

}  // namespace

// ---- many builds on given pair lists as one CUDA graph ----

struct ace_graph {
  std::vector<ace_op *> ops;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;  // private stream the builds were recorded from
  cudaEvent_t done = nullptr;  // recorded after each launch
  bool launched = false;
  bool screened = false;       // builds screen on the device; chains in device pack queues
};

namespace {

void graph_free(ace_graph *g) {
  if (g->launched) cudaEventSynchronize(g->done);
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  for (ace_op *op : g->ops) destroy_op(op);
  if (g->done) cudaEventDestroy(g->done);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}

// Records the builds of g->ops (already created, graph mode) from g->cap.  Each build is
// build_begin + build_finish with no host wait in between (the pair count is the caller's); builds
// are spread over stream lanes forked from g->cap and joined back.
ace_status record_builds(ace_graph *g, const void *const *phi, ace_dtype dtype, int lanes, cudaStream_t *lane_st) {
  cudaEvent_t ev = nullptr;
  ACE_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
  struct EvGuard {
    cudaEvent_t e;
    ~EvGuard() { cudaEventDestroy(e); }
  } guard{ev};
  ACE_CUDA(cudaEventRecord(ev, g->cap), "event");
  for (int l = 0; l < lanes; ++l) ACE_CUDA(cudaStreamWaitEvent(lane_st[l], ev, 0), "fork");
  if (g->screened) {
    ace_status s = run_queued_builds(g->ops, phi, dtype, lane_st[0]);
    if (s != ACE_OK) return s;
  }
  for (size_t i = 0; i < g->ops.size() && !g->screened; ++i) {
    ace_status s = begin_any(g->ops[i], phi[i], dtype);
    if (s == ACE_OK) s = finish_any(g->ops[i]);
    if (s != ACE_OK) return fail(s, "build %zu of %zu: %s", i, g->ops.size(), g_last_error.c_str());
  }
  for (int l = 0; l < lanes; ++l) {
    ACE_CUDA(cudaEventRecord(ev, lane_st[l]), "event");
    ACE_CUDA(cudaStreamWaitEvent(g->cap, ev, 0), "join");
  }
  return ACE_OK;
}

}  // namespace

extern "C" {

ace_status ace_graph_create(int k, const ace_desc *desc, const void *const *phi, ace_dtype dtype,
                            const int *const *pairs_host, const long *npairs, void *cuda_stream, ace_graph **out) {
  if (!out) return fail(ACE_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (k < 1 || k > ace::kQueueMaxBuilds || !desc || !phi || (pairs_host && !npairs))
    return fail(ACE_ERR_ARG, "bad graph arguments");
  const bool screened = pairs_host == nullptr;
  std::vector<std::vector<int2>> given(k);
  for (int i = 0; i < k; ++i) {
    ace_status s = check_desc(&desc[i]);
    if (s == ACE_OK) s = working_dtype(&desc[i], dtype);
    if (s == ACE_OK && (!phi[i] || !is_device_pointer(phi[i])))
      s = fail(ACE_ERR_ARG, "phi is not device memory");
    if (s == ACE_OK && reinterpret_cast<uintptr_t>(phi[i]) % 16 != 0) s = fail(ACE_ERR_ARG, "phi is not 16-byte aligned");
    if (s == ACE_OK && !screened) s = checked_pairs(&desc[i], pairs_host[i], npairs[i], given[i]);
    if (s == ACE_OK && screened && desc[i].prec == ACE_FP64)
      s = fail(ACE_ERR_ARG, "screened builds in a graph run in the mixed form only");
    if (s == ACE_OK && screened && !queue_eligible(1, &desc[i]))
      s = fail(ACE_ERR_UNSUPPORTED_GRID, "no persistent chain for the %dx%dx%d grid", desc[i].n[0], desc[i].n[1],
               desc[i].n[2]);
    if (s != ACE_OK) return fail(s, "build %d of %d: %s", i, k, g_last_error.c_str());
  }
  cudaStream_t user = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  ACE_CUDA(cudaStreamIsCapturing(user, &cs), "stream state");
  if (cs != cudaStreamCaptureStatusNone) return fail(ACE_ERR_ARG, "cuda_stream is being captured");
  int dev = 0;
  ACE_CUDA(cudaGetDevice(&dev), "device");
  // the kernel and twiddle tables are made (uploaded, then waited for) before the recording
  for (int i = 0; i < k; ++i) {
    const DeviceTables *tab = nullptr;
    cudaError_t e = dtype == ACE_F64 ? get_tables<double>(dev, desc[i], user, &tab)
                                     : get_tables<float>(dev, desc[i], user, &tab);
    if (e != cudaSuccess) return cuda_fail(e, "kernel and twiddle tables");
  }
  // the L2 set-aside for the chain's scratch windows is a context limit: made before the recording,
  // which then only sets the windows (stream attributes, copied into the recorded kernels)
  for (int i = 0; i < k; ++i) {
    const int mb = chain_params(desc[i], desc[i].prec == ACE_FP64).persist_mb;
    if (mb > 0) l2_set_aside(dev, mb);
  }
  ace_graph *g = new ace_graph;
  g->screened = screened;
  cudaError_t e = cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming);
  // one lane by default: a build's chain already fills the GPU through its side streams, and
  // concurrent builds only share the L2 (measured: 4 lanes 25% slower on 8 builds at 96^3)
  const int lanes = std::min(kLanes, std::max(1, std::min(k, env_int("ACE_GRAPH_LANES", 1))));
  cudaStream_t lane_st[kLanes];
  for (int l = 0; l < lanes && e == cudaSuccess; ++l) e = get_side_stream(dev, kSide * kLanes + l, &lane_st[l]);
  ace_status s = e == cudaSuccess ? ACE_OK : cuda_fail(e, "graph setup");
  for (int i = 0; i < k && s == ACE_OK; ++i) {
    ace_op *op = new_op(&desc[i], lane_st[i % lanes], &s);
    if (!op) break;
    op->graph = true;
    op->lane = i % lanes;
    op->use_given = !screened;
    op->given.swap(given[i]);
    g->ops.push_back(op);
  }
  if (s == ACE_OK) {
    // relaxed mode: the handles' buffers come from cudaMalloc while the builds are recorded
    e = cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "begin capture");
    } else {
      s = record_builds(g, phi, dtype, lanes, lane_st);
      const std::string msg = g_last_error;
      cudaGraph_t graph = nullptr;
      e = cudaStreamEndCapture(g->cap, &graph);
      g->graph = graph;
      if (s != ACE_OK) {
        cudaGetLastError();
        s = fail(s, "%s", msg.c_str());
      } else if (e != cudaSuccess) {
        s = cuda_fail(e, "end capture");
      }
    }
    if (s != ACE_OK) {
      // workspaces taken inside the recording belong to the discarded graph
      for (ace_op *op : g->ops) op->temps.clear();
    }
  }
  if (s == ACE_OK) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e == cudaSuccess) e = cudaGraphUpload(g->exec, user);
    if (e != cudaSuccess) s = cuda_fail(e, "graph instantiate");
  }
  if (s != ACE_OK) {
    const std::string msg = g_last_error;
    graph_free(g);
    return fail(s, "%s", msg.c_str());
  }
  *out = g;
  return ACE_OK;
}

ace_status ace_graph_launch(ace_graph *g, void *cuda_stream) {
  if (!g) return fail(ACE_ERR_ARG, "graph is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  ACE_CUDA(cudaGraphLaunch(g->exec, st), "graph launch");
  ACE_CUDA(cudaEventRecord(g->done, st), "event");
  g->launched = true;
  return ACE_OK;
}

ace_status ace_graph_sync(ace_graph *g) {
  if (!g) return fail(ACE_ERR_ARG, "graph is NULL");
  if (!g->launched) return fail(ACE_ERR_ARG, "the graph has not been launched");
  ACE_CUDA(cudaEventSynchronize(g->done), "graph");
  ace_status first = ACE_OK;
  std::string msg;
  for (size_t i = 0; i < g->ops.size(); ++i) {
    ace_status s = build_collect(g->ops[i]);
    if (s != ACE_OK && first == ACE_OK) {
      first = s;
      msg = "build " + std::to_string(i) + " of " + std::to_string(g->ops.size()) + ": " + g_last_error;
    }
  }
  return first == ACE_OK ? ACE_OK : fail(first, "%s", msg.c_str());
}

int ace_graph_size(const ace_graph *g) { return g ? (int)g->ops.size() : 0; }

ace_status ace_graph_op(const ace_graph *g, int i, ace_op **op) {
  if (!g || !op) return fail(ACE_ERR_ARG, "NULL argument");
  if (i < 0 || i >= (int)g->ops.size()) return fail(ACE_ERR_ARG, "build %d of %zu", i, g->ops.size());
  *op = g->ops[i];
  return ACE_OK;
}

void ace_graph_destroy(ace_graph *g) {
  if (g) graph_free(g);
}

}  // extern "C"
