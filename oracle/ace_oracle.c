/*
 * ace_oracle.c -- plain FP64 CPU oracle for the (screened) ACE exchange build.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's CPU-baseline
 * leg load this library.  It shares no code, table or helper with the CUDA path.
 *
 * What it computes, step by step, in the paper's order (arXiv:2101.03155):
 *   - Eq. (vx):   V_X psi_i = - sum_j v_ij(r) psi_j            (W_i below is -V_X psi_i)
 *   - Eq. (e:vij): v_ij = <psi_j | 1/r12 | psi_i>, evaluated in reciprocal space by FFT
 *                  (section II, "Computation of v_ij ... in reciprocal space").
 *   - Screen (section II, display after Eq. (unit)): pair i-j kept iff
 *                  int |phi_i phi_j| dr >= rho_cut.
 *   - Appendix A:  W_i = V_X psi_i;  M_kl = <psi_k|V_X|psi_l>;  -M = L L^T (Cholesky);
 *                  P = W L^-T;  V_X^ACE = - sum_k |P_k><P_k|.
 *
 * Readings where the paper is silent (each one is the plain definition written out):
 *   - sign: W here is +sum_j v_ij phi_j (= -V_X phi_i), so M = -dV Phi^T W equals the paper's M;
 *     L = chol(-M); xi = W L^-T = -P, and K = -xi xi^T is the same operator V_X^ACE.
 *   - discrete metric: every inner product carries dV = Omega / N.
 *   - Fourier convention: rho~(m) = (1/N) sum_r rho(r) exp(-i G_m.x_r),
 *     v(r) = sum_m 4 pi/|G_m|^2 rho~(m) exp(+i G_m.x_r); G_m = sum_k m_k b_k, b = 2 pi A^-T,
 *     m_k wrapped to [-N_k/2, N_k/2); full FFT box; G = 0 dropped; at a Nyquist index the
 *     kernel is the mean of 4 pi/|G|^2 over the +-N_k/2 choices (keeps it even, v real).
 *   - isolated cell (the QM box of section III's enzyme application, for which the paper names no
 *     Poisson solver): the interaction 1/r cut off at r = rc, i.e. the kernel
 *     4 pi (1 - cos(|G| rc))/|G|^2 with the G = 0 term 2 pi rc^2 kept; rc defaults to the radius
 *     of the largest sphere inside the cell.  For a density of diameter D with D <= rc and
 *     D + rc <= the distance to its nearest periodic image this is the open-boundary Coulomb
 *     interaction exactly (pinned against closed-form Gaussian self-energies).
 *   - energy: E_x = (f/2) tr M.
 *   - diagonal pairs contribute once; the mask is symmetric; M is symmetrised before Cholesky.
 *
 * Parity: pinned by the closed-form Gaussian lattice sum, a naive DFT, and the ACE invariants
 * (see tests/test_oracle_pins.py).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_in_parallel(void) { return 1; }
#endif

typedef double complex cplx;

static const double ORACLE_PI = 3.14159265358979323846264338327950288;

void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------------------------
 * 1D DFT by recursive mixed-radix decimation in time (Cooley-Tukey), any length.
 * tw[e] = exp(-2 pi i e / ntab) for the full length ntab; a sub-transform of length n uses
 * every (ntab/n)-th entry.  sign = -1: forward exp(-i...), +1: inverse exp(+i...), unnormalised.
 * ---------------------------------------------------------------------------------------- */
static int smallest_factor(int n) {
  for (int p = 2; p * p <= n; ++p)
    if (n % p == 0) return p;
  return n;
}

static void dft_rec(const cplx *x, long xs, cplx *y, int n, int sign, const cplx *tw, int step,
                    cplx *tmp) {
  if (n == 1) {
    y[0] = x[0];
    return;
  }
  const int p = smallest_factor(n), m = n / p;
  /* Y_q[k] = sum_t x[(p t + q) xs] w_m^{t k}, stored at y[q m + k] */
  for (int q = 0; q < p; ++q) dft_rec(x + q * xs, xs * p, y + q * m, m, sign, tw, step * p, tmp);
  /* X[k + m s] = sum_q w_n^{q (k + m s)} Y_q[k] */
  for (int k = 0; k < m; ++k)
    for (int s = 0; s < p; ++s) {
      cplx acc = 0.0;
      for (int q = 0; q < p; ++q) {
        const long e = ((long)q * (long)(k + m * s)) % n;
        cplx w = tw[e * step];
        if (sign > 0) w = conj(w);
        acc += w * y[q * m + k];
      }
      tmp[k + m * s] = acc;
    }
  memcpy(y, tmp, (size_t)n * sizeof(cplx));
}

static cplx *twiddle_table(int n) {
  cplx *tw = (cplx *)malloc((size_t)n * sizeof(cplx));
  for (int e = 0; e < n; ++e) {
    const double a = 2.0 * ORACLE_PI * (double)e / (double)n;
    tw[e] = cos(a) - I * sin(a);
  }
  return tw;
}

typedef struct {
  int n[3];
  cplx *tw[3];
  int maxn;
} fft3_plan;

static void plan_init(fft3_plan *pl, int n1, int n2, int n3) {
  pl->n[0] = n1;
  pl->n[1] = n2;
  pl->n[2] = n3;
  pl->maxn = n1;
  if (n2 > pl->maxn) pl->maxn = n2;
  if (n3 > pl->maxn) pl->maxn = n3;
  for (int a = 0; a < 3; ++a) pl->tw[a] = twiddle_table(pl->n[a]);
}

static void plan_free(fft3_plan *pl) {
  for (int a = 0; a < 3; ++a) free(pl->tw[a]);
}

/* In-place unnormalised 3D DFT of z[i1][i2][i3] along each axis in turn.  Lines are independent;
 * when called outside a parallel region they are spread over threads (each line is computed the
 * same way whatever the thread count, so results do not depend on it). */
#define ORACLE_MAXN 1024
static void fft_line(const fft3_plan *pl, int axis, cplx *base, long stride, int sign) {
  cplx line[ORACLE_MAXN], out[ORACLE_MAXN], tmp[ORACLE_MAXN];
  const int n = pl->n[axis];
  for (int k = 0; k < n; ++k) line[k] = base[(long)k * stride];
  dft_rec(line, 1, out, n, sign, pl->tw[axis], 1, tmp);
  for (int k = 0; k < n; ++k) base[(long)k * stride] = out[k];
}

static void fft3(const fft3_plan *pl, cplx *z, int sign, cplx *work) {
  const int n1 = pl->n[0], n2 = pl->n[1], n3 = pl->n[2];
  (void)work;
  const int par = !omp_in_parallel();
  /* axis 3 (contiguous) */
#pragma omp parallel for schedule(static) if (par)
  for (long a = 0; a < (long)n1 * n2; ++a) fft_line(pl, 2, z + a * n3, 1, sign);
  /* axis 2 */
#pragma omp parallel for schedule(static) if (par)
  for (long a = 0; a < (long)n1 * n3; ++a) fft_line(pl, 1, z + (a / n3) * n2 * n3 + (a % n3), n3, sign);
  /* axis 1 */
#pragma omp parallel for schedule(static) if (par)
  for (long a = 0; a < (long)n2 * n3; ++a) fft_line(pl, 0, z + a, (long)n2 * n3, sign);
}

/* Exported for the naive-DFT check: z is interleaved (re, im) of shape [n1][n2][n3]. */
int oracle_fft3d(double *z, int n1, int n2, int n3, int sign) {
  if (n1 < 1 || n2 < 1 || n3 < 1 || n1 > ORACLE_MAXN || n2 > ORACLE_MAXN || n3 > ORACLE_MAXN) return 1;
  fft3_plan pl;
  plan_init(&pl, n1, n2, n3);
  cplx *work = (cplx *)malloc(3 * (size_t)pl.maxn * sizeof(cplx));
  fft3(&pl, (cplx *)z, sign, work);
  free(work);
  plan_free(&pl);
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Coulomb kernel on the FFT box: K[m] = 4 pi / |G_m|^2, K[0] = 0, Nyquist-averaged.
 * ---------------------------------------------------------------------------------------- */
static void reciprocal(const double A[9], double B[9]) {
  /* rows b_k with a_j . b_k = 2 pi delta_jk, i.e. B = 2 pi A^-T */
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  /* inverse of A via cofactors: inv[i][j] = cof[j][i] / det; b_k = 2 pi * (column k of A^-1) */
  double inv[9];
  inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
  inv[1] = -(A[1] * A[8] - A[2] * A[7]) / det;
  inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
  inv[3] = -(A[3] * A[8] - A[5] * A[6]) / det;
  inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
  inv[5] = -(A[0] * A[5] - A[2] * A[3]) / det;
  inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
  inv[7] = -(A[0] * A[7] - A[1] * A[6]) / det;
  inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) B[k * 3 + c] = 2.0 * ORACLE_PI * inv[c * 3 + k];
}

static double cell_volume(const double A[9]) {
  const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                     A[2] * (A[3] * A[7] - A[4] * A[6]);
  return fabs(det);
}

/* Radius of the largest sphere inside the cell: half the smallest distance between lattice
 * planes, pi / |b_k| minimised over k. */
double oracle_inscribed_radius(const double *lattice) {
  double B[9];
  reciprocal(lattice, B);
  double r = HUGE_VAL;
  for (int k = 0; k < 3; ++k) {
    const double b = sqrt(B[k * 3] * B[k * 3] + B[k * 3 + 1] * B[k * 3 + 1] + B[k * 3 + 2] * B[k * 3 + 2]);
    if (ORACLE_PI / b < r) r = ORACLE_PI / b;
  }
  return r;
}

/* Coulomb kernel at G of |G|^2 = g2:
 *   kind 0 (periodic cell): 4 pi / |G|^2, and the G = 0 term is dropped;
 *   kind 1 (isolated cell, the interaction 1/r cut off at r = rc): the Fourier transform of
 *          theta(rc - r) / r, 4 pi (1 - cos(|G| rc)) / |G|^2, whose G -> 0 limit is 2 pi rc^2. */
static double kernel_at(double g2, int kind, double rc) {
  if (kind == 1) return g2 == 0.0 ? 2.0 * ORACLE_PI * rc * rc : 4.0 * ORACLE_PI * (1.0 - cos(sqrt(g2) * rc)) / g2;
  return 4.0 * ORACLE_PI / g2;
}

int oracle_coulomb_kernel(const double *lattice, int n1, int n2, int n3, int kind, double rc, double *K) {
  const int n[3] = {n1, n2, n3};
  double B[9];
  reciprocal(lattice, B);
  if (kind == 1 && rc <= 0.0) rc = oracle_inscribed_radius(lattice);
  for (int i1 = 0; i1 < n1; ++i1)
    for (int i2 = 0; i2 < n2; ++i2)
      for (int i3 = 0; i3 < n3; ++i3) {
        const int idx[3] = {i1, i2, i3};
        int m[3], nyq[3];
        for (int k = 0; k < 3; ++k) {
          m[k] = (2 * idx[k] < n[k]) ? idx[k] : idx[k] - n[k];
          nyq[k] = (n[k] % 2 == 0) && (2 * idx[k] == n[k]);
        }
        const long lin = ((long)i1 * n2 + i2) * n3 + i3;
        if (m[0] == 0 && m[1] == 0 && m[2] == 0) {
          K[lin] = kind == 1 ? kernel_at(0.0, kind, rc) : 0.0;
          continue;
        }
        double acc = 0.0;
        int cnt = 0;
        for (int s = 0; s < 8; ++s) {
          int ok = 1, mm[3];
          for (int k = 0; k < 3; ++k) {
            const int flip = (s >> k) & 1;
            if (flip && !nyq[k]) ok = 0;
            mm[k] = flip ? -m[k] : m[k];
          }
          if (!ok) continue;
          double G[3];
          for (int c = 0; c < 3; ++c) G[c] = mm[0] * B[0 * 3 + c] + mm[1] * B[1 * 3 + c] + mm[2] * B[2 * 3 + c];
          acc += kernel_at(G[0] * G[0] + G[1] * G[1] + G[2] * G[2], kind, rc);
          ++cnt;
        }
        K[lin] = acc / cnt;
      }
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * v_ij(r) of Eq. (e:vij): forward DFT of rho_ij = phi_i phi_j, multiply by K/N, inverse DFT.
 * ---------------------------------------------------------------------------------------- */
static void pair_potential(const fft3_plan *pl, const double *K, const double *pi_, const double *pj,
                           long npts, cplx *z, cplx *work, double *v) {
  const int par = !omp_in_parallel();
#pragma omp parallel for schedule(static) if (par)
  for (long r = 0; r < npts; ++r) z[r] = pi_[r] * pj[r];
  fft3(pl, z, -1, work);
  const double invN = 1.0 / (double)npts;
#pragma omp parallel for schedule(static) if (par)
  for (long r = 0; r < npts; ++r) z[r] *= K[r] * invN;
  fft3(pl, z, +1, work);
#pragma omp parallel for schedule(static) if (par)
  for (long r = 0; r < npts; ++r) v[r] = creal(z[r]);
}

int oracle_pair_potential(const double *phi_i, const double *phi_j, int n1, int n2, int n3,
                          const double *lattice, int kind, double rc, double *v) {
  if (n1 > ORACLE_MAXN || n2 > ORACLE_MAXN || n3 > ORACLE_MAXN) return 1;
  const long npts = (long)n1 * n2 * n3;
  fft3_plan pl;
  plan_init(&pl, n1, n2, n3);
  double *K = (double *)malloc((size_t)npts * sizeof(double));
  cplx *z = (cplx *)malloc((size_t)npts * sizeof(cplx));
  cplx *work = (cplx *)malloc(3 * (size_t)pl.maxn * sizeof(cplx));
  oracle_coulomb_kernel(lattice, n1, n2, n3, kind, rc, K);
  pair_potential(&pl, K, phi_i, phi_j, npts, z, work, v);
  free(work);
  free(z);
  free(K);
  plan_free(&pl);
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Pair screen: O_ij = dV sum_r |phi_i(r) phi_j(r)|; keep iff O_ij >= rho_cut (rho_cut <= 0:
 * keep all); the diagonal is always kept.  O and mask are norb x norb, symmetric.
 * ---------------------------------------------------------------------------------------- */
int oracle_screen(const double *phi, int norb, long npts, double dV, double rho_cut, double *O,
                  unsigned char *mask) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < norb; ++i)
    for (int j = i; j < norb; ++j) {
      const double *a = phi + (long)i * npts, *b = phi + (long)j * npts;
      double s = 0.0;
      for (long r = 0; r < npts; ++r) s += fabs(a[r] * b[r]);
      s *= dV;
      O[(long)i * norb + j] = s;
      O[(long)j * norb + i] = s;
      const unsigned char keep = (i == j) || (rho_cut <= 0.0) || (s >= rho_cut);
      mask[(long)i * norb + j] = keep;
      mask[(long)j * norb + i] = keep;
    }
  return 0;
}

/* ------------------------------------------------------------------------------------------
 * Eq. (vx), row by row: W_i = sum_{j : mask_ij} v_ij phi_j (= -V_X phi_i).
 * rows (optional) selects which i to compute; W has nrows rows of npts.
 * mask (optional, norb x norb) restricts j; NULL means all pairs.
 * ---------------------------------------------------------------------------------------- */
int oracle_exchange_w(const double *phi, int norb, int n1, int n2, int n3, const double *lattice,
                      int kind, double rc, const unsigned char *mask, const int *rows, int nrows, double *W) {
  if (n1 > ORACLE_MAXN || n2 > ORACLE_MAXN || n3 > ORACLE_MAXN) return 2;
  const long npts = (long)n1 * n2 * n3;
  fft3_plan pl;
  plan_init(&pl, n1, n2, n3);
  double *K = (double *)malloc((size_t)npts * sizeof(double));
  oracle_coulomb_kernel(lattice, n1, n2, n3, kind, rc, K);
  int err = 0;
  /* many rows: one row per thread; few rows: rows in sequence, parallel inside each transform */
  const int outer = nrows >= oracle_max_threads();
#pragma omp parallel if (outer)
  {
    cplx *z = (cplx *)malloc((size_t)npts * sizeof(cplx));
    cplx *work = (cplx *)malloc(3 * (size_t)pl.maxn * sizeof(cplx));
    double *v = (double *)malloc((size_t)npts * sizeof(double));
    if (!z || !work || !v) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 1)
      for (int ri = 0; ri < nrows; ++ri) {
        const int i = rows ? rows[ri] : ri;
        double *Wi = W + (long)ri * npts;
        memset(Wi, 0, (size_t)npts * sizeof(double));
        for (int j = 0; j < norb; ++j) {
          if (mask && !mask[(long)i * norb + j]) continue;
          const double *pj = phi + (long)j * npts;
          pair_potential(&pl, K, phi + (long)i * npts, pj, npts, z, work, v);
#pragma omp parallel for schedule(static) if (!omp_in_parallel())
          for (long r = 0; r < npts; ++r) Wi[r] += v[r] * pj[r];
        }
      }
    }
    free(v);
    free(work);
    free(z);
  }
  free(K);
  plan_free(&pl);
  return err;
}

/* (ij|ij) = dV sum_r rho_ij(r) v_ij(r) */
double oracle_pair_energy(const double *phi_i, const double *phi_j, int n1, int n2, int n3,
                          const double *lattice, int kind, double rc) {
  const long npts = (long)n1 * n2 * n3;
  double *v = (double *)malloc((size_t)npts * sizeof(double));
  oracle_pair_potential(phi_i, phi_j, n1, n2, n3, lattice, kind, rc, v);
  double s = 0.0;
  for (long r = 0; r < npts; ++r) s += phi_i[r] * phi_j[r] * v[r];
  free(v);
  return s * cell_volume(lattice) / (double)npts;
}

/* ------------------------------------------------------------------------------------------
 * Appendix A: M = -dV Phi^T W (raw and symmetrised), -M = L L^T, xi = W L^-T.
 * Returns 0, or k+1 if the Cholesky pivot k of -M is not positive.
 * Layouts: phi, W, xi are [norb][npts]; M_raw, M, L are [norb][norb] row-major.
 * ---------------------------------------------------------------------------------------- */
int oracle_ace_from_w(const double *phi, const double *W, int norb, long npts, double dV,
                      double *M_raw, double *M, double *L, double *xi) {
  const int n = norb;
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) {
      const double *a = phi + (long)k * npts, *b = W + (long)l * npts;
      double s = 0.0;
      for (long r = 0; r < npts; ++r) s += a[r] * b[r];
      M_raw[(long)k * n + l] = -dV * s;
    }
  for (int k = 0; k < n; ++k)
    for (int l = 0; l < n; ++l) M[(long)k * n + l] = 0.5 * (M_raw[(long)k * n + l] + M_raw[(long)l * n + k]);
  /* Cholesky of A = -M */
  memset(L, 0, (size_t)n * n * sizeof(double));
  for (int j = 0; j < n; ++j) {
    double d = -M[(long)j * n + j];
    for (int k = 0; k < j; ++k) d -= L[(long)j * n + k] * L[(long)j * n + k];
    if (!(d > 0.0)) return j + 1;
    const double ljj = sqrt(d);
    L[(long)j * n + j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double s = -M[(long)i * n + j];
      for (int k = 0; k < j; ++k) s -= L[(long)i * n + k] * L[(long)j * n + k];
      L[(long)i * n + j] = s / ljj;
    }
  }
  /* xi = W L^-T: for each grid point r, L xi_r^T = W_r^T by forward substitution */
  if (xi) {
#pragma omp parallel for schedule(static)
    for (long r = 0; r < npts; ++r)
      for (int k = 0; k < n; ++k) {
        double s = W[(long)k * npts + r];
        for (int l = 0; l < k; ++l) s -= L[(long)k * n + l] * xi[(long)l * npts + r];
        xi[(long)k * npts + r] = s / L[(long)k * n + k];
      }
  }
  return 0;
}

/* C = dV xi^T psi (norb x m), the projection that the ACE application multiplies back by -xi */
static void ace_coefficients(const double *xi, int norb, const double *psi, int m, long npts, double dV, double *C) {
#pragma omp parallel for collapse(2) schedule(static)
  for (int k = 0; k < norb; ++k)
    for (int c = 0; c < m; ++c) {
      double s = 0.0;
      for (long r = 0; r < npts; ++r) s += xi[(long)k * npts + r] * psi[(long)c * npts + r];
      C[(long)k * m + c] = dV * s;
    }
}

/* K psi = -xi (dV xi^T psi) (section II, ACE application).  xi [norb][npts], psi/out [m][npts]. */
int oracle_ace_apply(const double *xi, int norb, const double *psi, int m, long npts, double dV,
                     double *out) {
  double *C = (double *)malloc((size_t)norb * m * sizeof(double));
  ace_coefficients(xi, norb, psi, m, npts, dV, C);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m; ++c)
    for (long r = 0; r < npts; ++r) {
      double s = 0.0;
      for (int k = 0; k < norb; ++k) s += xi[(long)k * npts + r] * C[(long)k * m + c];
      out[(long)c * npts + r] = -s;
    }
  free(C);
  return 0;
}

/* The same application evaluated at nidx chosen grid points only: C = dV xi^T psi over the whole
 * grid (norb x m, returned), then out[c][q] = -sum_k xi_k(idx[q]) C[k][c] (m x nidx). */
int oracle_ace_apply_at(const double *xi, int norb, const double *psi, int m, long npts, double dV,
                        const long *idx, int nidx, double *C, double *out) {
  ace_coefficients(xi, norb, psi, m, npts, dV, C);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m; ++c)
    for (int q = 0; q < nidx; ++q) {
      double s = 0.0;
      for (int k = 0; k < norb; ++k) s += xi[(long)k * npts + idx[q]] * C[(long)k * m + c];
      out[(long)c * nidx + q] = -s;
    }
  return 0;
}

/* E_x = (f/2) tr M */
double oracle_exchange_energy(const double *M, int norb, double spin_factor) {
  double t = 0.0;
  for (int k = 0; k < norb; ++k) t += M[(long)k * norb + k];
  return 0.5 * spin_factor * t;
}

/* ------------------------------------------------------------------------------------------
 * SCDM column selection (the localisation step before the path, section II: selected columns
 * of the density matrix): the greedy choice of column-pivoted QR of Psi^T (norb x npts, whose
 * column r is the vector psi(r) = (psi_1(r), ..., psi_n(r))).  Step k takes the column of largest
 * residual norm d(r) = |psi(r)|^2 - sum_{j<k} (u_j . psi(r))^2 (the first such index on ties),
 * then extends the orthonormal basis u_j of the chosen columns by Gram-Schmidt (applied twice).
 * piv receives the npiv chosen grid indices in order.  Returns 0.
 * ---------------------------------------------------------------------------------------- */
int oracle_scdm_select(const double *psi, int norb, long npts, int npiv, int *piv) {
  double *d = (double *)malloc((size_t)npts * sizeof(double));
  double *U = (double *)malloc((size_t)npiv * norb * sizeof(double));
#pragma omp parallel for schedule(static)
  for (long r = 0; r < npts; ++r) {
    double s = 0.0;
    for (int i = 0; i < norb; ++i) s += psi[(long)i * npts + r] * psi[(long)i * npts + r];
    d[r] = s;
  }
  for (int k = 0; k < npiv; ++k) {
    long best = 0;
    for (long r = 1; r < npts; ++r)
      if (d[r] > d[best]) best = r;
    piv[k] = (int)best;
    double *u = U + (long)k * norb;
    for (int i = 0; i < norb; ++i) u[i] = psi[(long)i * npts + best];
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < k; ++j) {
        const double *v = U + (long)j * norb;
        double c = 0.0;
        for (int i = 0; i < norb; ++i) c += v[i] * u[i];
        for (int i = 0; i < norb; ++i) u[i] -= c * v[i];
      }
    double nrm = 0.0;
    for (int i = 0; i < norb; ++i) nrm += u[i] * u[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < norb; ++i) u[i] /= nrm;
#pragma omp parallel for schedule(static)
    for (long r = 0; r < npts; ++r) {
      double p = 0.0;
      for (int i = 0; i < norb; ++i) p += u[i] * psi[(long)i * npts + r];
      d[r] -= p * p;
    }
    d[best] = -1.0; /* chosen columns leave the candidate set (their residual is zero) */
  }
  free(U);
  free(d);
  return 0;
}
