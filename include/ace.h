/*
 * ace.h -- C ABI of the GB300 (sm_103a) screened adaptively-compressed-exchange (s-ACE) library.
 *
 * Method: arXiv:2101.03155 (s-MTACE).  The library builds the ACE operator from a set of real,
 * Gamma-point, orthonormal (typically localized) orbitals on a periodic grid and applies it:
 *
 *   pair screen (section II, display after Eq. unit): keep pair (i,j) iff int |phi_i phi_j| >= rho_cut
 *   pair potential (Eq. e:vij): v_ij = <phi_j | 1/r12 | phi_i>, by FFT with the 4 pi/|G|^2 kernel
 *                              (or the isolated-cell kernel, see Conventions)
 *   exchange action (Eq. vx):  W_i = sum_j v_ij phi_j            (W = -V_X phi)
 *   Appendix A:                M = -dV Phi^T W, -M = L L^T, xi = W L^-T   (xi = -P of App. A)
 *   ACE application (section II): K psi = -xi (dV xi^T psi) = V_X^ACE psi
 *   exchange energy:           E_x = (f/2) tr M
 *
 * Conventions (all entry points):
 *   - grid index r = (i1, i2, i3), i3 fastest; point x_r = sum_k (i_k/N_k) a_k; N = N1 N2 N3;
 *     dV = Omega / N with Omega = |det(lattice)|.
 *   - orbital arrays are [count][N1][N2][N3] in the stated dtype, rows contiguous; the input set
 *     is orthonormal under dV (dV sum_r phi_i phi_j = delta_ij); this is not checked.
 *   - Fourier convention: rho~(m) = (1/N) sum_r rho(r) e^{-i G_m . x_r}; G_m = sum_k m_k b_k,
 *     b = 2 pi A^-T, m_k wrapped to [-N_k/2, N_k/2); full FFT box; G = 0 term dropped; at a Nyquist
 *     index the kernel is the mean of 4 pi/|G|^2 over the +-N_k/2 choices.
 *   - isolated cell (ace_desc.coulomb = ACE_COULOMB_TRUNCATED; the QM box of the paper's enzyme
 *     application in section III, for which the paper names no Poisson solver): the interaction is
 *     1/r cut off at r = r_cut, i.e. the kernel 4 pi (1 - cos(|G| r_cut))/|G|^2 with its G = 0 limit
 *     2 pi r_cut^2 kept (same Nyquist mean).  For a pair density of diameter D with D <= r_cut and
 *     D + r_cut <= the distance to its nearest periodic image it is the open-boundary Coulomb
 *     interaction exactly.
 *   - pointers named *_dev are CUDA device pointers; pointers that the comments say "host or
 *     device" may be either (host memory, pageable or pinned, is copied inside the call on the
 *     given stream; device memory that does not start on a 16-byte boundary is likewise read
 *     through, or written through, an aligned copy).  `cuda_stream` is a cudaStream_t (NULL =
 *     legacy default stream).
 *   - every entry point returns an ace_status and never throws; on failure the message is
 *     available from ace_last_error() on the calling thread.
 *   - ownership: the caller owns every buffer it passes and must keep it valid and unchanged
 *     until the stream work of the call completes.  The library owns everything inside an
 *     ace_op; ace_destroy frees it and must not race with stream work that uses the handle.
 *   - thread safety: distinct handles may be used concurrently on distinct streams.
 */
#ifndef ACE_GB300_H
#define ACE_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ACE_OK = 0,
  ACE_ERR_ARG = 1,              /* invalid argument (null pointer, bad size, bad lattice)        */
  ACE_ERR_CUDA = 2,             /* a CUDA runtime call failed; see ace_last_error()              */
  ACE_ERR_OOM = 3,              /* device allocation failed                                      */
  ACE_ERR_NOT_POSDEF = 4,       /* -M is not positive definite (Cholesky pivot in the message)   */
  ACE_ERR_NONFINITE = 5,        /* NaN/Inf reached M                                             */
  ACE_ERR_UNSUPPORTED_GRID = 6, /* an axis length has no compiled FFT plan (see ace_grid_supported) */
  ACE_ERR_TIMEOUT = 7           /* a bounded device-side wait gave up                            */
} ace_status;

typedef enum {
  ACE_FP64 = 0,  /* plain form: every step in double precision                                 */
  ACE_MIXED = 1  /* mixed form: FP32 pair densities/FFTs/kernel multiply/accumulation,
                    screen |Phi| |Phi|^T as FP32 products on the CUDA cores (FP64 across
                    K-splits), BF16x3 split products on the tensor cores (FP32 accumulate within
                    256-point chunks, FP64 across) for Phi^T W, xi^T psi and xi C; M, Cholesky,
                    L^-1 and E_x in FP64                                                          */
} ace_precision;

typedef enum { ACE_F32 = 0, ACE_F64 = 1 } ace_dtype;

typedef enum {
  ACE_COULOMB_PERIODIC = 0,  /* 4 pi/|G|^2, G = 0 dropped (Eq. e:vij in reciprocal space)        */
  ACE_COULOMB_TRUNCATED = 1  /* isolated cell: 1/r cut off at r_cut (see Conventions)           */
} ace_coulomb;

typedef struct {
  int n[3];              /* N1, N2, N3 (each must satisfy ace_grid_supported)                  */
  double lattice[3][3];  /* rows a1, a2, a3 in bohr; det != 0                                    */
  int norb;              /* n, 1 <= n <= 1024                                                    */
  double rho_cut;        /* keep (i,j) iff dV sum_r |phi_i phi_j| >= rho_cut; <= 0 keeps all     */
  double spin_factor;    /* f in E_x = (f/2) tr M: 2 closed shell, 1 one spin channel            */
  ace_precision prec;
  ace_coulomb coulomb;   /* kernel of step a4; a zeroed field is the periodic kernel             */
  double r_cut;          /* ACE_COULOMB_TRUNCATED: cut-off radius in bohr; <= 0 selects the
                            radius of the largest sphere inside the cell, min_k pi/|b_k|         */
} ace_desc;

typedef struct ace_op ace_op; /* opaque: owns xi, W, M, L, L^-1, the pair list and workspaces  */

/* Build the s-ACE operator (Appendix A with the screen of section II).
 *   phi:   orbitals [norb][N1][N2][N3], host or device, dtype as given (converted internally to
 *          the working precision of desc->prec).
 *   out:   receives a new handle, also on ACE_ERR_NOT_POSDEF / ACE_ERR_NONFINITE (so that M can be
 *          inspected); NULL on every other error.
 * The call returns after the build has completed on `cuda_stream` (it reads the pair count and
 * the Cholesky status back to the host).  Errors: ACE_ERR_ARG, ACE_ERR_UNSUPPORTED_GRID,
 * ACE_ERR_OOM, ACE_ERR_CUDA, ACE_ERR_NOT_POSDEF, ACE_ERR_NONFINITE. */
ace_status ace_build(const ace_desc *desc, const void *phi, ace_dtype dtype, void *cuda_stream,
                     ace_op **out);

/* Build the ACE operator on a given pair list instead of the screen: the reuse step of a
 * multiple-time-step run (section III: an outer step every n steps, many snapshots in between that
 * move each centre by ~0.05 bohr), where the pair list of an earlier snapshot (ace_get(...,
 * ACE_GET_PAIRS)) serves the next ones.  W, M, L, xi and E_x are those of Appendix A with Eq. (vx)
 * summed over exactly the listed pairs (desc->rho_cut is not used; ACE_GET_OVERLAP returns zeros).
 *   pairs_host: host int32 [npairs][2], 0 <= i, j < norb; (i, j) and (j, i) are the same pair, each
 *               pair at most once (ACE_ERR_ARG otherwise); the diagonal pairs (i, i) are not added.
 * Synchronous like ace_build; the same errors. */
ace_status ace_build_pairs(const ace_desc *desc, const void *phi, ace_dtype dtype, const int *pairs_host,
                           long npairs, void *cuda_stream, ace_op **out);

/* ---- One build over several GPUs (Eq. vx split by pairs, App. A split by grid points) ----
 * The pairs of Eq. (vx) are independent terms, and App. A's M_kl = -dV sum_r phi_k(r) W_l(r) and
 * xi = W L^-T (row-wise xi = L^-1 W, pointwise in r) split over disjoint slabs of grid points.  On
 * R ranks (one GPU each, one process each):
 *   1. rank r: ace_exchange_w on its share of the pair list       -> partial W^(r) [norb][N]
 *   2. caller: reduce-scatter of the W^(r) over point slabs         -> W_slab [norb][N_r] on rank r
 *   3. rank r: ace_m_partial on its slab of phi and W               -> M^(r) [norb][norb] FP64
 *   4. caller: all-reduce of the M^(r) (sum)                        -> M on every rank
 *   5. rank r: ace_build_from_m(M, W_slab)                          -> handle holding xi_slab, L, E_x
 *   6. apply: ace_apply_coeffs on psi_slab, caller all-reduce of C, ace_apply_finish -> (K psi)_slab
 * The collectives (steps 2, 4, 6) are the caller's (NCCL, or any other); the library computes.
 * Every slab array is [norb][npts] (or [m][npts]) with rows contiguous. */

/* Step 1: W = sum of the Eq. (vx) terms of the listed pairs only, W_i += v_ij phi_j and
 * W_j += v_ij phi_i (i = j once).  pairs_host as in ace_build_pairs (no diagonal pair is added).
 *   phi: [norb][N] host or device, dtype as given (converted to the working precision).
 *   W:   [norb][N] in the working dtype of desc->prec (F32 mixed, F64 plain), host or device;
 *        overwritten.
 * Synchronous; errors as ace_build_pairs. */
ace_status ace_exchange_w(const ace_desc *desc, const void *phi, ace_dtype dtype, const int *pairs_host,
                          long npairs, void *W, void *cuda_stream);

/* Step 3: M_partial = -dV Phi_slab^T W_slab over the npts points of a slab (App. A, M_kl summed
 * over the slab's points), dV = Omega / N of the whole grid of desc.
 *   phi_slab, W_slab: device [norb][npts] in the working dtype (ACE_ERR_ARG otherwise).
 *   M: device FP64 [norb][norb], overwritten.
 * Synchronous (reads back the tensor-core kernels' give-up flag). */
ace_status ace_m_partial(const ace_desc *desc, const void *phi_slab, const void *W_slab, ace_dtype dtype,
                         long long npts, double *M, void *cuda_stream);

/* Step 5: the operator on a slab from the summed M (App. A): M <- (M + M^T)/2, -M = L L^T, L^-1,
 * E_x = (f/2) tr M, and xi_slab = L^-1 W_slab (rows).  The handle behaves as one from ace_build
 * on a grid of npts points: exchange_energy, ace_get(ACE_GET_XI / M / M_RAW / L) with
 * [norb][npts] for xi, ace_apply_coeffs / ace_apply_finish; it holds no W and no pair list.
 *   M: FP64 [norb][norb], host or device.  W_slab: [norb][npts], host or device, dtype as given.
 * Synchronous; out as in ace_build (also on ACE_ERR_NOT_POSDEF / ACE_ERR_NONFINITE). */
ace_status ace_build_from_m(const ace_desc *desc, const double *M, const void *W_slab, ace_dtype dtype,
                            long long npts, void *cuda_stream, ace_op **out);

/* Step 6, the two halves of ace_apply around the caller's all-reduce (section II, ACE
 * application): ace_apply_coeffs writes C = dV xi^T psi (device FP64 [norb][m]) for psi of m rows
 * of the handle's points; ace_apply_finish writes out = -xi C ([m][points], host or device, dtype
 * as given) from the summed C (device FP64).  On one GPU the two in sequence equal ace_apply.
 * Synchronous. */
ace_status ace_apply_coeffs(const ace_op *op, const void *psi, ace_dtype dtype, int m, double *C,
                            void *cuda_stream);
ace_status ace_apply_finish(const ace_op *op, const double *C, ace_dtype dtype, int m, void *out,
                            void *cuda_stream);

/* k independent builds (replicas or snapshots) issued back to back on one stream.  desc, phi and
 * out are arrays of length k; each build is as in ace_build.  On the first failing build the
 * handles already created are destroyed, every out[i] is NULL, and its status is returned.
 * By default the builds run one after another, each with the pair chain of ace_build (all screens
 * first, then one wait for every pair list); each build's M, Cholesky and xi run on a second stream
 * of its lane, beside the next build's pair chain (ACE_BATCH_TAIL=0 keeps them on the lane, after
 * the chain).  The environment variable ACE_BATCH_LANES (1-4) runs that many builds at a time on
 * concurrent stream lanes.  With the environment variable ACE_BATCH_QUEUE=1, and every build in the mixed form on
 * a grid with a persistent chain plan (see ace_graph_create), the chains run instead as one
 * persistent launch per grid over the builds' concatenated device pack lists, with no host wait
 * between the screens and the chains. */
ace_status ace_build_batched(int k, const ace_desc *desc, const void *const *phi, ace_dtype dtype,
                             void *cuda_stream, ace_op **out);

/* ---- Many builds as one CUDA graph ----
 * The reuse steps of a multiple-time-step run (section III) rebuild the operator on the pair lists
 * of the last outer step while only the orbitals change; with the pair counts known on the host no
 * build needs a host wait, so k of them (snapshots or replicas; each as in ace_build_pairs) can be
 * recorded once and replayed with one launch.  Screened builds (each as in ace_build) need no host
 * wait either when their pair chains run from device pack queues: the screen's compaction writes
 * the packs, and one persistent chain launch per grid walks the concatenated lists of all builds on
 * that grid, reading the counts on the device (pairs_host = NULL below).
 *
 * ace_graph_create records the k builds from a private stream and instantiates the graph; it runs
 * no build.  The builds follow one another (each spreads its pair chain over side streams, with
 * the same chain settings and L2 window as ace_build_pairs); the environment variable
 * ACE_GRAPH_LANES (1-4, default 1) runs that many builds at a time instead.  desc, phi, pairs_host
 * and npairs are arrays of length k.
 *   phi[i]:        device orbitals [norb][N1][N2][N3] in the working dtype of desc[i].prec (ACE_F32
 *                  for ACE_MIXED, ACE_F64 for ACE_FP64), 16-byte aligned (ACE_ERR_ARG otherwise).
 *                  The graph keeps the pointers and reads the arrays at every launch: the caller
 *                  overwrites their contents between launches, and frees them after the graph.
 *   pairs_host[i]: the pair list of build i, checked as in ace_build_pairs and copied; or
 *                  pairs_host = NULL (npairs ignored): every build screens with its desc->rho_cut at
 *                  every launch (mixed form only, ACE_ERR_ARG for ACE_FP64; grids with a persistent
 *                  chain plan: 32^3, 48^3, 64^3, 72^3, 96^3, 108^3, 128^3, 144^3, 160x144x128, else
 *                  ACE_ERR_UNSUPPORTED_GRID); ace_pair_count and ACE_GET_PAIRS give the last
 *                  synchronised launch's list.
 *   cuda_stream:   the kernel tables of every grid are made on it first (synchronously); it must
 *                  not be capturing.
 * The handles of the builds (ace_graph_op) exist from creation on and keep their buffers (xi, W, M,
 * L, pair list) at fixed addresses; each launch overwrites them.  They are owned by the graph:
 * ace_destroy ignores them and ace_graph_destroy releases them.
 * Errors: ACE_ERR_ARG, ACE_ERR_UNSUPPORTED_GRID, ACE_ERR_OOM, ACE_ERR_CUDA (nothing is created). */
typedef struct ace_graph ace_graph;
ace_status ace_graph_create(int k, const ace_desc *desc, const void *const *phi, ace_dtype dtype,
                            const int *const *pairs_host, const long *npairs, void *cuda_stream,
                            ace_graph **out);

/* Enqueue one replay of all k builds on `cuda_stream`; returns without waiting.  Work the caller
 * queues on the same stream afterwards (ace_apply, ace_get on a handle) sees its results.  One
 * replay runs at a time: a launch starts after the previous one has finished. */
ace_status ace_graph_launch(ace_graph *g, void *cuda_stream);

/* Wait for the last launch, then read every build's Cholesky status, give-up flag and E_x into its
 * handle (exchange_energy).  Returns the first failing build's status (ACE_ERR_NOT_POSDEF,
 * ACE_ERR_NONFINITE, ACE_ERR_TIMEOUT) or ACE_OK; ACE_ERR_ARG before the first launch. */
ace_status ace_graph_sync(ace_graph *g);

/* Number of builds in the graph (0 for NULL), and the handle of build i (borrowed). */
int ace_graph_size(const ace_graph *g);
ace_status ace_graph_op(const ace_graph *g, int i, ace_op **op);

/* Waits for the last launch, then frees the graph and its handles.  NULL is a no-op. */
void ace_graph_destroy(ace_graph *g);

/* Apply the ACE operator (section II): out = -xi (dV xi^T psi) = V_X^ACE psi, dense (no screen).
 *   psi, out: [m][N1][N2][N3] of `dtype`, host or device (both on the same side), m >= 1.
 * Runs on `cuda_stream` and returns after the result is complete (it reads back a device error
 * flag).  Errors: ACE_ERR_ARG, ACE_ERR_CUDA, ACE_ERR_OOM, ACE_ERR_TIMEOUT. */
ace_status ace_apply(const ace_op *op, const void *psi, ace_dtype dtype, int m, void *out,
                     void *cuda_stream);

/* SCDM localisation (section II, Eq. unit, with the selected columns of the density matrix that
 * section II names; the paper gives no formulas for it, this is the method of Damle, Lin and Ying,
 * J. Chem. Theory Comput. 11, 1463 (2015)): phi_k = sum_i psi_i U[i][k] with U orthogonal,
 *   1. c_0..c_{n-1}: greedy column-pivoted QR of Psi^T (n x npts): step k takes the grid point of
 *      largest residual norm |psi(r)|^2 - sum_{j<k} (u_j . psi(r))^2 (the smallest index on ties),
 *      u_j the orthonormalised columns chosen before;
 *   2. M[i][j] = psi_i(c_j) (columns of the density matrix Psi Psi^T at the chosen points);
 *   3. U = M (M^T M)^{-1/2} (symmetric orthonormalisation, so phi is orthonormal under dV whenever
 *      psi is).
 *   psi:  canonical orbitals [norb][npts] (npts = N1 N2 N3 in any grid order), host or device.
 *   phi:  output [norb][npts] of `dtype`, on the same side as psi (may not alias it).
 *   piv_host: optional host int32 [norb] receiving c_0..c_{n-1}; u_host: optional host double
 *         [norb][norb] receiving U; launches: optional, the number of this library's kernels run.
 *   prec: ACE_FP64 every step in FP64.  ACE_MIXED: psi in FP32, residual norms in FP64 with the
 *         projections u_k . psi(r) summed as FP32 products in 8-term FP32 partials; M, U and
 *         (M^T M)^{-1/2} (coupled Newton-Schulz) in FP64; Phi = U^T Psi by BF16x3 tensor-core
 *         products (FP32-level).  Near-equal residuals may then select another, equally valid,
 *         point than FP64 arithmetic would.
 * 1 <= norb <= 1024, norb <= npts < 2^31.  Synchronous.  Errors: ACE_ERR_ARG, ACE_ERR_CUDA,
 * ACE_ERR_OOM, ACE_ERR_TIMEOUT, ACE_ERR_NOT_POSDEF (the chosen columns are linearly dependent:
 * psi has rank < norb, and the Newton-Schulz iteration did not converge). */
ace_status ace_scdm(int norb, long long npts, ace_precision prec, const void *psi, ace_dtype dtype, void *phi,
                    int *piv_host, double *u_host, void *cuda_stream, long *launches);

/* E_x = (f/2) tr M in Hartree (host scalar), computed in FP64 during the build. */
ace_status exchange_energy(const ace_op *op, double *ex_hartree);

/* Copy an internal array to `dst` (host or device) of `bytes` bytes (must equal the size):
 *   ACE_GET_XI      xi  [norb][N]  working dtype (float for ACE_MIXED, double for ACE_FP64)
 *   ACE_GET_W       W   [norb][N]  working dtype
 *   ACE_GET_M       M   [norb][norb] double, symmetrised
 *   ACE_GET_M_RAW   M   [norb][norb] double, before symmetrisation
 *   ACE_GET_L       L   [norb][norb] double, lower triangular, -M = L L^T
 *   ACE_GET_PAIRS   kept pairs, int32 [npairs][2] with i <= j, sorted by (i, j)
 *   ACE_GET_OVERLAP screen values O_ij = dV sum_r |phi_i phi_j|, [norb][norb] double
 * Synchronous with respect to the host. */
enum {
  ACE_GET_XI = 0,
  ACE_GET_W = 1,
  ACE_GET_M = 2,
  ACE_GET_M_RAW = 3,
  ACE_GET_L = 4,
  ACE_GET_PAIRS = 5,
  ACE_GET_OVERLAP = 6
};
ace_status ace_get(const ace_op *op, int what, void *dst, size_t bytes, void *cuda_stream);

/* Number of kept (i <= j) pairs in the build, and the byte size of an ace_get item. */
ace_status ace_pair_count(const ace_op *op, long *npairs);
ace_status ace_get_size(const ace_op *op, int what, size_t *bytes);

/* Per-stage device times of the last build in milliseconds (CUDA events on the build stream):
 * [0] screen, [1] pair chain (W), [2] M, [3] Cholesky/L^-1/E_x, [4] xi, [5] total.  The handles of
 * a graph (ace_graph_op) record no timing events and report zeros. */
ace_status ace_stage_times(const ace_op *op, float ms[6]);

/* Number of this library's CUDA kernels that the build of `op` launched. */
ace_status ace_kernel_launches(const ace_op *op, long *launches);

/* Autotuner of the pair chain; the paper has no counterpart (it is a property of this GPU code).
 * Screens `phi` as ace_build does, then times the pair chain on a sample of up to 480 of its packs
 * for each candidate setting of the stream-batched chain: packs per batch {1,2,3,4,6}, side streams
 * {2,4,8}, L2 set-aside for the scratch {0, 60 MB}, rows per block of the pack order {1,2,4,8};
 * then, on the best of those, the pencil tile of the axis-1 pass (FP32: 32 columns with the default
 * or the other thread count, or 16 columns); and the persistent chain (one launch walking the pack
 * list through a device task queue) with queue lags {2,3,4} where its grid is compiled.  The
 * fastest setting is kept for this grid and precision and used by later builds in the process;
 * with the environment variable ACE_TUNE_FILE set, the table is also read from and written to that
 * file (one line per grid: n1 n2 n3 fp64 group batch streams l2_mb row_block persistent lag
 * pencil_tile; lines without the last field read as pencil tile 0).  params (optional, 7 ints)
 * receives {group, batch, streams, l2_mb, row_block, persistent lag or 0, pencil tile}.
 * Environment variables ACE_PLANE_BATCH, ACE_STREAMS, ACE_L2_PERSIST_MB, ACE_GROUP, ACE_ROW_BLOCK,
 * ACE_PERSISTENT, ACE_PERSIST_LAG, ACE_CONV_TILE override the table.  Grids without a plane-pass
 * plan keep the defaults.  Synchronous.  Errors as ace_build. */
ace_status ace_autotune(const ace_desc *desc, const void *phi, ace_dtype dtype, void *cuda_stream,
                        int *params);

/* 1 if an axis length has a compiled FFT plan for precision `prec`, else 0. */
int ace_grid_supported(int n_axis, ace_precision prec);

/* Frees a handle and everything it owns.  NULL, and handles that belong to a graph, are no-ops. */
void ace_destroy(ace_op *op);

/* W without device allocation.  The paper has no counterpart: this entry point exists for callers
 * that may not call cudaMalloc (or any allocator) while they run -- applications that hand the
 * library pre-allocated buffers under a fixed memory budget, allocation-free inner loops, or hosts
 * whose framework owns all device memory.
 *
 * Computes the pair-potential chain of Eq. (vx) for an explicit pair list:
 *   W_i = sum_{j : (i,j) or (j,i) listed} v_ij phi_j,  v_ij by FFT with the kernel desc->coulomb selects,
 * the same arithmetic as the W step of ace_build (desc->rho_cut and desc->spin_factor are ignored).
 *   phi_dev:    device orbitals [norb][N1][N2][N3]; W_dev: device output of the same shape (zeroed
 *               by the call); both 16-byte aligned (else ACE_ERR_ARG: this entry point makes no
 *               copies).  dtype must be the working type of desc->prec (ACE_F32 for ACE_MIXED,
 *               ACE_F64 for ACE_FP64).
 *   pairs_host: host int32 [npairs][2] with 0 <= i <= j < norb (checked before any work is queued).
 * All workspace (FFT scratch, pack list, kernel table, twiddles) lives in one array of
 * ACE_NOALLOC_SCRATCH_BYTES compiled into the library; every GPU that loads the library holds that
 * array until the process exits.  A grid needs (3 * sizeof(T) * N + about 80 KB) bytes of it; larger
 * grids return ACE_ERR_ARG.  Every call on a device shares the array and finds the previous call's
 * contents in it: the call rewrites what it reads and zeroes W.  Calls whose GPU work overlaps (other
 * streams or host threads) race on the array and must be serialised by the caller.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, with that device current)
 * and caches it.  Stream-ordered on `cuda_stream`; pair uploads go through a
 * small pageable host buffer.  Errors: ACE_ERR_ARG, ACE_ERR_UNSUPPORTED_GRID, ACE_ERR_CUDA. */
#define ACE_NOALLOC_SCRATCH_BYTES (32u << 20)
ace_status ace_exchange_w_noalloc(const ace_desc *desc, const void *phi_dev, ace_dtype dtype,
                                  const int *pairs_host, long npairs, void *W_dev, void *cuda_stream);

/* Message of the last failing call on this thread ("" if none). */
const char *ace_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* ACE_GB300_H */
