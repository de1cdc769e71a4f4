"""Pins of the FP64 oracle against facts the paper and the mathematics fix (no GPU).

* naive DFT sums pin the oracle's mixed-radix FFT (every radix 2/3/5, odd axes, Nyquist);
* closed-form Gaussian lattice sums (Poisson summation, tests/closed_form.py) pin the pair
  density spectrum, the Coulomb kernel, the 1/N normalisation and E_x on cubic and triclinic cells;
* the ACE identities of Appendix A (M symmetric negative definite, K_ACE phi_k = V_X phi_k,
  Phi^T K Phi = M) pin M, the Cholesky factor and xi = W L^-T;
* unitary invariance of the occupied span (Eq. unit) pins the pair sum;
* brute force pins the pair screen (section II, display after Eq. unit).
"""

import itertools

import numpy as np
import pytest

import closed_form as cf
from workloads.generators import gaussian_orbitals, periodic_gaussian, random_orthogonal, loewdin, config1

TRICLINIC = np.array([[7.5, 0.0, 0.0], [1.2, 7.0, 0.0], [0.6, -0.9, 6.8]])


def naive_dft_full(z, sign):
    """X[m] = sum_r z[r] exp(sign 2 pi i sum_k m_k r_k / N_k), as one dense N x N matrix."""
    shape = z.shape
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), -1).reshape(-1, 3)
    phase = np.zeros((len(idx), len(idx)))
    for k in range(3):
        phase += np.outer(idx[:, k], idx[:, k]) / shape[k]
    F = np.exp(sign * 2j * np.pi * phase)
    return (F @ z.reshape(-1)).reshape(shape)


def naive_dft_separable(z, sign):
    """Same sums taken one axis at a time with dense 1D DFT matrices."""
    out = z
    for axis, n in enumerate(z.shape):
        k = np.arange(n)
        F = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, axis, 0), axes=(1, 0)), 0, axis)
    return out


@pytest.mark.parametrize(
    "shape,full",
    [((8, 8, 8), True), ((6, 6, 6), True), ((10, 10, 10), True), ((12, 12, 12), False), ((15, 15, 15), False),
     ((6, 10, 15), True), ((2, 3, 5), True), ((1, 4, 9), True)],
)
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_matches_naive_dft(oracle_mod, shape, full, sign):
    rng = np.random.default_rng(hash(shape) % 1000)
    z = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = naive_dft_full(z, sign) if full else naive_dft_separable(z, sign)
    got = oracle_mod.fft3d(z, sign)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_fft_roundtrip(oracle_mod):
    rng = np.random.default_rng(3)
    z = rng.standard_normal((9, 20, 25)) + 1j * rng.standard_normal((9, 20, 25))
    back = oracle_mod.fft3d(oracle_mod.fft3d(z, -1), 1) / z.size
    assert np.abs(back - z).max() < 1e-13


def test_kernel_orthorhombic_textbook(oracle_mod):
    """Orthorhombic cell: 4 pi / sum_k (2 pi m_k / L_k)^2 with m wrapped to [-N/2, N/2)."""
    L = np.array([9.0, 7.0, 11.0])
    grid = (12, 9, 16)
    K = oracle_mod.coulomb_kernel(np.diag(L), grid)
    m = [np.where(2 * np.arange(n) < n, np.arange(n), np.arange(n) - n) for n in grid]
    g2 = sum(np.meshgrid(*[(2 * np.pi * m[k] / L[k]) ** 2 for k in range(3)], indexing="ij"))
    ref = np.where(g2 > 0, 4 * np.pi / np.where(g2 > 0, g2, 1), 0.0)
    assert K[0, 0, 0] == 0.0
    assert np.abs(K - ref).max() <= 1e-14 * ref.max()


def test_kernel_even_and_rotation_invariant(oracle_mod):
    grid = (12, 14, 15)
    K = oracle_mod.coulomb_kernel(TRICLINIC, grid)
    neg = K[(-np.arange(12)) % 12][:, (-np.arange(14)) % 14][:, :, (-np.arange(15)) % 15]
    assert np.abs(K - neg).max() <= 1e-15 * K.max()
    rng = np.random.default_rng(11)
    R = random_orthogonal(3, rng)
    if np.linalg.det(R) < 0:
        R[:, 0] *= -1
    K2 = oracle_mod.coulomb_kernel(TRICLINIC @ R.T, grid)
    assert np.abs(K - K2).max() <= 1e-13 * K.max()


@pytest.fixture(scope="module", params=["cubic", "triclinic"])
def gaussian_case(request):
    rng = np.random.default_rng(7)
    if request.param == "cubic":
        lat, grid = np.diag([8.0, 8.0, 8.0]), (16, 16, 16)
    else:
        lat, grid = TRICLINIC, (12, 14, 15)
    phi, prims, D = gaussian_orbitals(grid, lat, 3, 2, rng)
    coeffs = cf.prim_pair_coefficients(prims, lat, grid, nalias=2, nimg=2)
    return dict(lat=lat, grid=grid, phi=phi, prims=prims, D=D, coeffs=coeffs)


def test_orbitals_rebuild_from_primitives(gaussian_case):
    c = gaussian_case
    G = np.stack([periodic_gaussian(c["grid"], c["lat"], A, a) for a, A in c["prims"]])
    assert np.abs(np.tensordot(c["D"], G, 1) - c["phi"]).max() < 1e-13


def test_pair_spectrum_closed_form(oracle_mod, gaussian_case):
    """Forward transform of rho_ij = phi_i phi_j / N equals the Poisson-summed closed form."""
    c = gaussian_case
    N = int(np.prod(c["grid"]))
    for i, j in [(0, 1), (1, 2), (2, 2)]:
        z = oracle_mod.fft3d((c["phi"][i] * c["phi"][j]).astype(complex), -1) / N
        ref = cf.orbital_pair_coefficients(c["D"], c["coeffs"], i, j).reshape(c["grid"])
        assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()


def test_exchange_energy_closed_form(oracle_mod, gaussian_case):
    c = gaussian_case
    E = cf.pair_energies(c["D"], c["coeffs"], c["lat"], c["grid"])
    for f in (2.0, 1.0):
        res = oracle_mod.ace_build(c["phi"], c["lat"], rho_cut=0.0, spin_factor=f)
        ref = -(f / 2) * E.sum()
        assert abs(res["E_x"] - ref) <= 1e-12 * abs(ref)
    for i, j in [(0, 0), (0, 1), (1, 2)]:
        pe = oracle_mod.pair_energy(c["phi"][i], c["phi"][j], c["lat"])
        assert abs(pe - E[i, j]) <= 1e-12 * E.max()


def test_single_orbital(oracle_mod):
    """n = 1: E_x = -(f/2)(11|11), L = sqrt((11|11)), xi = W / L (closed form for one Gaussian)."""
    lat, grid = np.diag([7.0, 8.0, 9.0]), (14, 16, 18)
    A = np.array([2.0, 3.5, 1.0])
    g = periodic_gaussian(grid, lat, A, 1.3)
    dV = np.prod(np.diag(lat)) / np.prod(grid)
    phi = (g / np.sqrt(dV * np.sum(g * g)))[None]
    coeffs = cf.prim_pair_coefficients([(1.3, A)], lat, grid, nalias=2, nimg=2)
    D = np.array([[1.0 / np.sqrt(dV * np.sum(g * g))]])
    e11 = cf.pair_energies(D, coeffs, lat, grid)[0, 0]
    res = oracle_mod.ace_build(phi, lat, 0.0, 2.0)
    assert abs(res["E_x"] + e11) <= 1e-12 * e11
    assert abs(res["L"][0, 0] - np.sqrt(e11)) <= 1e-12 * np.sqrt(e11)
    assert np.abs(res["xi"] - res["W"] / res["L"][0, 0]).max() <= 1e-14 * np.abs(res["W"]).max()


@pytest.fixture(scope="module")
def cfg1_build(oracle_mod):
    w = config1()
    return w, oracle_mod.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)


def test_ace_invariants_all_pairs(oracle_mod, cfg1_build):
    """Appendix A identities, all pairs (config 1: 16 orbitals, 32^3)."""
    w, r = cfg1_build
    M_raw, M, L, xi, W = r["M_raw"], r["M"], r["L"], r["xi"], r["W"]
    assert r["status"] == 0
    assert np.linalg.norm(M_raw - M_raw.T) <= 1e-14 * np.linalg.norm(M_raw)
    assert np.linalg.eigvalsh(M).max() < 0
    assert np.allclose(np.tril(L), L) and np.all(np.diag(L) > 0)
    assert np.abs(L @ L.T + M).max() <= 1e-14 * np.abs(M).max()
    K = oracle_mod.ace_apply(xi, w.phi, w.dV)
    for k in range(w.norb):
        assert np.linalg.norm(K[k] + W[k]) <= 1e-12 * np.linalg.norm(W[k])
    PKP = w.dV * K.reshape(w.norb, -1) @ w.phi.reshape(w.norb, -1).T
    assert np.abs(PKP - M).max() <= 1e-12 * np.abs(M).max()
    tr = 0.5 * w.spin_factor * np.trace(M)
    assert abs(r["E_x"] - tr) <= 1e-14 * abs(tr)
    proj = w.dV * xi.reshape(w.norb, -1) @ w.phi.reshape(w.norb, -1).T
    assert abs(r["E_x"] + 0.5 * w.spin_factor * np.sum(proj**2)) <= 1e-12 * abs(r["E_x"])


def test_factorisation_matches_library(oracle_mod, cfg1_build):
    """Cholesky and the triangular solve reduce to LAPACK routines."""
    import scipy.linalg as sla

    w, r = cfg1_build
    Lref = np.linalg.cholesky(-r["M"])
    assert np.abs(r["L"] - Lref).max() <= 1e-13 * np.abs(Lref).max()
    Wm = r["W"].reshape(w.norb, -1)
    xi_ref = sla.solve_triangular(Lref, Wm, lower=True)  # xi^T = L^-1 W^T in the [norb][npts] layout
    assert np.abs(r["xi"].reshape(w.norb, -1) - xi_ref).max() <= 1e-12 * np.abs(xi_ref).max()


def test_apply_matches_library(oracle_mod, cfg1_build):
    w, r = cfg1_build
    rng = np.random.default_rng(5)
    psi = rng.standard_normal((5,) + w.grid)
    got = oracle_mod.ace_apply(r["xi"], psi, w.dV)
    X = r["xi"].reshape(w.norb, -1)
    ref = -(X.T @ (w.dV * X @ psi.reshape(5, -1).T)).T
    assert np.abs(got.reshape(5, -1) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_apply_at_points_matches_library(oracle_mod, cfg1_build):
    """The application evaluated at chosen points only (the form the stored full-size values use):
    C = dV xi^T psi and -xi C at those points, from library matrix products; on the orbitals
    themselves it gives -W_k at the points (App. A, K phi_k = V_X phi_k)."""
    from workloads.generators import probe_vectors, sample_points

    w, r = cfg1_build
    X = r["xi"].reshape(w.norb, -1)
    idx = sample_points(w.npts, 300, 11)
    assert len(np.unique(idx)) == 300 and idx.min() >= 0 and idx.max() < w.npts
    psi = probe_vectors(w.phi, w.dV, 3)
    assert np.allclose(w.dV * np.sum(psi.reshape(2, -1) ** 2, axis=1), 1.0, rtol=1e-14)
    C, out = oracle_mod.ace_apply_at(r["xi"], psi, w.dV, idx)
    C_ref = w.dV * X @ psi.reshape(2, -1).T
    assert np.abs(C - C_ref).max() <= 1e-13 * np.abs(C_ref).max()
    ref = -(X[:, idx].T @ C_ref).T
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()
    _, kphi = oracle_mod.ace_apply_at(r["xi"], w.phi, w.dV, idx)
    Wm = r["W"].reshape(w.norb, -1)[:, idx]
    assert np.abs(kphi + Wm).max() <= 1e-12 * np.abs(Wm).max()


def test_unitary_invariance(oracle_mod):
    """Eq. unit: a unitary mix of the occupied orbitals leaves E_x and the operator unchanged."""
    rng = np.random.default_rng(21)
    lat, grid = np.diag([8.0, 8.0, 8.0]), (12, 12, 12)
    phi, _, _ = gaussian_orbitals(grid, lat, 5, 2, rng)
    U = random_orthogonal(5, rng)
    phi2 = np.tensordot(U.T, phi, 1)
    r1 = oracle_mod.ace_build(phi, lat, 0.0, 2.0)
    r2 = oracle_mod.ace_build(phi2, lat, 0.0, 2.0)
    assert abs(r1["E_x"] - r2["E_x"]) <= 1e-12 * abs(r1["E_x"])
    dV = np.prod(np.diag(lat)) / np.prod(grid)
    psi = rng.standard_normal((3,) + grid)
    k1 = oracle_mod.ace_apply(r1["xi"], psi, dV)
    k2 = oracle_mod.ace_apply(r2["xi"], psi, dV)
    assert np.abs(k1 - k2).max() <= 1e-12 * np.abs(k1).max()


def test_screen_bruteforce(oracle_mod):
    rng = np.random.default_rng(4)
    lat, grid = np.diag([10.0, 10.0, 10.0]), (10, 12, 14)
    phi, _, _ = gaussian_orbitals(grid, lat, 6, 1, rng)
    dV = 1000.0 / np.prod(grid)
    flat = phi.reshape(6, -1)
    ref = np.array([[dV * np.sum(np.abs(flat[i] * flat[j])) for j in range(6)] for i in range(6)])
    O, mask = oracle_mod.screen(phi, lat, 0.0)
    assert np.abs(O - ref).max() <= 1e-13 * ref.max()
    assert mask.all()
    iu = np.triu_indices(6, 1)
    order = np.argsort(O[iu])
    ti, tj = iu[0][order[len(order) // 2]], iu[1][order[len(order) // 2]]
    cut = O[ti, tj]  # threshold exactly on one pair's value: ">=" keeps that pair
    _, mask = oracle_mod.screen(phi, lat, cut)
    for i, j in itertools.product(range(6), range(6)):
        assert mask[i, j] == (i == j or O[i, j] >= cut)
    assert mask[ti, tj] and mask[tj, ti]
    assert mask.sum() == 6 + 2 * (len(order) - len(order) // 2)


def test_screened_far_pair_is_sum_of_singles(oracle_mod):
    """Two orbitals far apart, cross pair screened out: E_x splits into single-orbital values."""
    lat, grid = np.diag([24.0, 12.0, 12.0]), (36, 18, 18)
    dV = np.prod(np.diag(lat)) / np.prod(grid)
    chi = np.stack([periodic_gaussian(grid, lat, [4.0, 6.0, 6.0], 1.0),
                    periodic_gaussian(grid, lat, [16.0, 6.0, 6.0], 0.8)])
    phi, _ = loewdin(chi, dV)
    O, mask = oracle_mod.screen(phi, lat, 1e-3)
    assert not mask[0, 1] and mask[0, 0] and mask[1, 1]
    r = oracle_mod.ace_build(phi, lat, rho_cut=1e-3, spin_factor=2.0)
    e0 = oracle_mod.ace_build(phi[:1], lat, 0.0, 2.0)["E_x"]
    e1 = oracle_mod.ace_build(phi[1:], lat, 0.0, 2.0)["E_x"]
    assert abs(r["E_x"] - (e0 + e1)) <= 1e-13 * abs(r["E_x"])
    assert abs(r["M"][0, 1]) <= 1e-15 * abs(r["M"][0, 0])


def test_exchange_w_row_subset(oracle_mod, cfg1_build):
    w, r = cfg1_build
    rows = [3, 0, 11]
    Wsub = oracle_mod.exchange_w(w.phi, w.lattice, rows=rows)
    assert np.array_equal(Wsub, r["W"][rows])


def test_not_posdef_reported(oracle_mod):
    """A zero orbital makes pivot 3 of -M exactly zero: the Cholesky reports it (status = pivot + 1)."""
    rng = np.random.default_rng(8)
    lat, grid = np.diag([8.0, 8.0, 8.0]), (10, 10, 10)
    phi, _, _ = gaussian_orbitals(grid, lat, 3, 1, rng)
    phi = np.concatenate([phi, np.zeros_like(phi[:1])])
    W = oracle_mod.exchange_w(phi, lat)
    res = oracle_mod.ace_from_w(phi, W, 512.0 / 1000, want_xi=False)
    assert res["status"] == 4


# ------------------------------------------------------------------------------------------
# Isolated-cell kernel (the interaction 1/r cut off at r_cut): for a Gaussian density of
# diameter D with D <= r_cut and D + r_cut <= the nearest periodic image, the truncated
# interaction is the open-boundary Coulomb interaction, whose Gaussian values are closed forms:
# a charge-Q density (gamma/pi)^{3/2} Q exp(-gamma r^2) has self-energy Q^2 sqrt(2 gamma / pi).
# ------------------------------------------------------------------------------------------
def _gaussian_orbital(grid, lattice, alpha, centre):
    """(2 alpha / pi)^{3/4} exp(-alpha |r - centre|^2) sampled at the grid points (no images)."""
    frac = np.stack(np.meshgrid(*[np.arange(n) / n for n in grid], indexing="ij"), -1)
    r = frac @ np.asarray(lattice)
    d2 = np.sum((r - np.asarray(centre)) ** 2, axis=-1)
    return (2 * alpha / np.pi) ** 0.75 * np.exp(-alpha * d2)


ISO_L = 16.0
ISO_GRID = (48, 48, 48)


def test_truncated_kernel_values(oracle_mod):
    lat = np.diag([ISO_L, 12.0, 14.0])
    grid = (8, 6, 10)
    rc = 5.5
    K = oracle_mod.coulomb_kernel(lat, grid, oracle_mod.TRUNCATED, rc)
    assert K[0, 0, 0] == pytest.approx(2 * np.pi * rc * rc, rel=1e-15)
    for m in [(1, 0, 0), (0, 2, 3), (3, 1, 4), (1, 2, 1)]:
        G = 2 * np.pi * np.array(m) / np.diag(lat)
        g = np.linalg.norm(G)
        assert K[m] == pytest.approx(4 * np.pi * (1 - np.cos(g * rc)) / g**2, rel=1e-13)
    assert oracle_mod.inscribed_radius(lat) == pytest.approx(6.0, rel=1e-15)
    assert oracle_mod.inscribed_radius(TRICLINIC) < 3.5


def test_truncated_self_energy_closed_form(oracle_mod):
    lat = np.eye(3) * ISO_L
    alpha = 1.0
    phi = _gaussian_orbital(ISO_GRID, lat, alpha, [ISO_L / 2] * 3)
    ref = 2 * np.sqrt(alpha / np.pi)  # gamma = 2 alpha, Q = 1
    for rc in (0.0, 7.0, 8.0):  # 0: inscribed radius 8
        e = oracle_mod.pair_energy(phi, phi, lat, oracle_mod.TRUNCATED, rc)
        assert e == pytest.approx(ref, rel=1e-9), rc
    # the periodic kernel (G = 0 dropped) is a different interaction
    assert abs(oracle_mod.pair_energy(phi, phi, lat) - ref) > 1e-2


def test_truncated_cross_pair_closed_form(oracle_mod):
    lat = np.array([[ISO_L, 0.0, 0.0], [0.8, ISO_L, 0.0], [-0.5, 0.6, ISO_L]])
    alpha = 1.2
    c = np.array([ISO_L / 2, ISO_L / 2, ISO_L / 2]) @ np.eye(3)
    d = np.array([0.9, -0.4, 0.7])
    a = _gaussian_orbital(ISO_GRID, lat, alpha, c)
    b = _gaussian_orbital(ISO_GRID, lat, alpha, c + d)
    S = np.exp(-alpha * d @ d / 2)  # charge of phi_a phi_b, a Gaussian of exponent 2 alpha
    ref = S * S * 2 * np.sqrt(alpha / np.pi)
    assert oracle_mod.pair_energy(a, b, lat, oracle_mod.TRUNCATED, 7.5) == pytest.approx(ref, rel=1e-9)


def test_truncated_exchange_energy_of_separated_orbitals(oracle_mod):
    """Two far-apart Gaussian orbitals: E_x = -(f/2) sum of the two self-energies (the cross
    pair density vanishes), through the whole oracle build."""
    lat = np.eye(3) * ISO_L
    alpha = 1.0  # resolved by the 1/3-bohr grid to ~1e-10; overlap exp(-alpha 49 / 2) ~ 2e-11
    a = _gaussian_orbital(ISO_GRID, lat, alpha, [4.5, 8.0, 8.0])
    b = _gaussian_orbital(ISO_GRID, lat, alpha, [11.5, 8.0, 8.0])
    phi = np.stack([a, b])
    r = oracle_mod.ace_build(phi, lat, 0.0, 2.0, kind=oracle_mod.TRUNCATED, r_cut=0.0)
    assert r["status"] == 0
    ref = -(2.0 / 2) * 2 * (2 * np.sqrt(alpha / np.pi))
    assert r["E_x"] == pytest.approx(ref, rel=1e-9)


# ------------------------------------------------------------------------------------------
# SCDM localisation (selected columns of the density matrix, the step before the path):
# column-pivoted QR selection, then symmetric orthonormalisation of the selected columns.
# ------------------------------------------------------------------------------------------
def test_scdm_pivots_match_lapack_qrcp(oracle_mod):
    import scipy.linalg

    rng = np.random.default_rng(7)
    for n, m in [(6, 40), (12, 300), (20, 500)]:
        A = rng.standard_normal((n, m)) * rng.uniform(0.5, 2.0, size=m)
        _, _, P = scipy.linalg.qr(A, pivoting=True, mode="economic")
        assert list(oracle_mod.scdm_select(A)) == list(P[:n]), (n, m)


def test_scdm_localises_rotated_gaussians(oracle_mod):
    lat = np.diag([12.0, 12.0, 12.0])
    grid = (24, 24, 24)
    rng = np.random.default_rng(31)
    phi_loc, _, _ = gaussian_orbitals(grid, lat, 8, 1, rng, alpha_range=(1.0, 2.0))
    dV = np.prod(np.diag(lat)) / np.prod(grid)
    Q = random_orthogonal(8, rng)
    psi = np.tensordot(Q, phi_loc, axes=(1, 0))  # delocalised combinations, same span
    phi, piv = oracle_mod.scdm(psi, dV)
    flat_p, flat_s = phi.reshape(8, -1), psi.reshape(8, -1)
    # orthonormal under dV, and the same occupied space (psi = (dV psi phi^T) phi)
    assert np.abs(dV * flat_p @ flat_p.T - np.eye(8)).max() <= 1e-12
    assert np.abs((dV * flat_s @ flat_p.T) @ flat_p - flat_s).max() <= 1e-11 * np.abs(flat_s).max()
    assert len(set(piv.tolist())) == 8
    # E_x is invariant under the orthogonal change of basis (Eq. unit)
    e_psi = oracle_mod.ace_build(psi, lat, 0.0, 2.0, want_xi=False)["E_x"]
    e_phi = oracle_mod.ace_build(phi, lat, 0.0, 2.0, want_xi=False)["E_x"]
    assert e_phi == pytest.approx(e_psi, rel=1e-10)
    # localisation: the pair overlaps of the SCDM orbitals are those of the localized set, far
    # below those of the rotated set
    O_phi, _ = oracle_mod.screen(phi, lat, 0.0)
    O_psi, _ = oracle_mod.screen(psi, lat, 0.0)
    O_loc, _ = oracle_mod.screen(phi_loc, lat, 0.0)
    off = ~np.eye(8, dtype=bool)
    assert O_phi[off].mean() < 0.5 * O_psi[off].mean()
    assert O_phi[off].mean() < 2.0 * O_loc[off].mean()


def test_scdm_disjoint_orbitals_are_returned_unchanged(oracle_mod):
    """Orbitals on disjoint sets of grid points: the residual norm at a point is |psi_i(r)|^2 of
    the one orbital living there until that orbital's column is chosen, so the pivots are each
    orbital's largest point (in decreasing order of those maxima); M is diagonal, U = diag(sign),
    and the localized set is the input up to sign."""
    rng = np.random.default_rng(17)
    n, npts = 5, 400
    owner = rng.permutation(np.arange(npts) % n)  # every point belongs to one orbital
    psi = np.zeros((n, npts))
    for i in range(n):
        pts = np.flatnonzero(owner == i)
        psi[i, pts] = rng.standard_normal(pts.size)
        psi[i] /= np.linalg.norm(psi[i])
    phi, piv = oracle_mod.scdm(psi, 1.0)
    peaks = [int(np.argmax(np.abs(psi[i]))) for i in range(n)]
    order = np.argsort([-np.abs(psi[i, peaks[i]]) for i in range(n)], kind="stable")
    assert list(piv) == [peaks[i] for i in order]
    _, U = oracle_mod.scdm_orthonormalise(psi, piv)
    for col, i in enumerate(order):
        s = np.sign(psi[i, peaks[i]])
        assert abs(U[i, col] - s) <= 1e-14
        assert np.abs(np.delete(U[:, col], i)).max() <= 1e-14
        assert np.abs(phi[col] - s * psi[i]).max() <= 1e-14
