"""Seeded synthetic orbital sets that stand in for the paper's water boxes and QM region.

The paper's own systems (CPMD water boxes of 32/64/128 molecules, section III; the
beta-lactamase QM region, section III) are not available, so these generators produce
real, Gamma-point, orthonormal orbitals with the same shapes: a cubic cell at liquid-water
density with four localized orbitals per molecule (Eq. unit: localized, unitary-equivalent
orbitals), or a compact cluster of orbitals in a mostly empty orthorhombic cell.

Conventions shared by everything that consumes these arrays:
  * grid index r = (i1, i2, i3), i3 fastest; point x_r = sum_k (i_k / N_k) a_k;
  * ``lattice`` rows are a1, a2, a3 in bohr;
  * orbitals are ``phi[n, N1, N2, N3]`` (float64), orthonormal under the discrete metric
    dV * sum_r phi_i(r) phi_j(r) = delta_ij with dV = Omega / N.

Nothing here computes pair densities, potentials or any part of the exchange operator.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

WATER_CELL_32 = 18.63  # bohr; 9.85 Angstrom cell of 32 molecules (section III)
WATER_CELL_64 = 23.47  # bohr; same density, 64 molecules


@dataclasses.dataclass
class Workload:
    """One synthetic ACE build input."""

    name: str
    phi: np.ndarray  # (n, N1, N2, N3) float64, orthonormal under dV
    lattice: np.ndarray  # (3, 3) rows a1, a2, a3 (bohr)
    rho_cut: float  # pair-screen threshold; <= 0 keeps all pairs
    spin_factor: float
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def grid(self) -> tuple[int, int, int]:
        return tuple(int(v) for v in self.phi.shape[1:])

    @property
    def norb(self) -> int:
        return int(self.phi.shape[0])

    @property
    def npts(self) -> int:
        g = self.grid
        return g[0] * g[1] * g[2]

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.lattice)))

    @property
    def dV(self) -> float:
        return self.volume / self.npts


# ----------------------------------------------------------------------------------------
# Sampling of periodised Gaussians
# ----------------------------------------------------------------------------------------


def _is_diagonal(lattice: np.ndarray) -> bool:
    off = lattice - np.diag(np.diag(lattice))
    return bool(np.all(off == 0.0))


def periodic_gaussian(grid, lattice, centre, alpha, images: int = 2) -> np.ndarray:
    """Sample sum_T exp(-alpha |x_r - centre - T|^2) over lattice vectors T with |t_k| <= images."""
    grid = tuple(int(v) for v in grid)
    lattice = np.asarray(lattice, dtype=np.float64)
    centre = np.asarray(centre, dtype=np.float64)
    ts = np.arange(-images, images + 1)
    if _is_diagonal(lattice):
        # exp(-alpha|d|^2) factorises over orthogonal axes, and so does the image sum.
        out = None
        for k in range(3):
            L = lattice[k, k]
            x = np.arange(grid[k]) * (L / grid[k])
            d = x[:, None] - centre[k] - ts[None, :] * L
            g = np.exp(-alpha * d * d).sum(axis=1)
            out = g if out is None else np.multiply.outer(out, g)
        return out
    frac = np.stack(
        np.meshgrid(*[np.arange(n) / n for n in grid], indexing="ij"), axis=-1
    )  # (N1,N2,N3,3)
    pts = frac @ lattice
    out = np.zeros(grid)
    for t1 in ts:
        for t2 in ts:
            for t3 in ts:
                T = t1 * lattice[0] + t2 * lattice[1] + t3 * lattice[2]
                d = pts - centre - T
                out += np.exp(-alpha * np.einsum("...k,...k->...", d, d))
    return out


def loewdin(chi: np.ndarray, dV: float):
    """Symmetric orthonormalisation: returns (phi, C) with phi = C chi and dV phi phi^T = I.

    C = S^{-1/2}, S = dV chi chi^T, from a symmetric eigendecomposition.
    """
    n = chi.shape[0]
    flat = chi.reshape(n, -1)
    S = dV * (flat @ flat.T)
    S = 0.5 * (S + S.T)
    w, V = np.linalg.eigh(S)
    if w.min() <= 0:
        raise ValueError("orbital set is linearly dependent")
    C = (V * (1.0 / np.sqrt(w))) @ V.T
    phi = (C @ flat).reshape(chi.shape)
    return phi, C


def random_orthogonal(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal matrix (QR of a Gaussian matrix with sign fix)."""
    A = rng.standard_normal((n, n))
    Q, R = np.linalg.qr(A)
    return Q * np.sign(np.diag(R))[None, :]


def delocalised(phi: np.ndarray, seed: int) -> np.ndarray:
    """Canonical-like (delocalised) orbitals with the span of phi: Q phi with Q a seeded Haar-random
    orthogonal matrix, the input of a localisation step."""
    n = phi.shape[0]
    Q = random_orthogonal(n, np.random.default_rng(seed))
    return np.tensordot(Q, phi, axes=(1, 0))


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    Q = random_orthogonal(3, rng)
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


# ----------------------------------------------------------------------------------------
# Config-1 style: orbitals that are sums of primitive s-Gaussians
# ----------------------------------------------------------------------------------------


def gaussian_orbitals(
    grid,
    lattice,
    norb: int,
    prims_per_orb: int,
    rng: np.random.Generator,
    alpha_range=(0.5, 2.0),
    coeff_range=(0.5, 1.5),
    images: int = 2,
    centres=None,
):
    """Orbitals chi_i = sum_a c_a exp(-alpha_a |r - A_a|^2) (periodised), Loewdin-orthonormalised.

    Returns (phi, prims, D): ``prims`` is a list of (alpha, centre) for every primitive and
    ``D`` (norb x nprim) gives phi_i = sum_a D[i, a] g_a on the grid, so that closed-form
    checks can rebuild each orbital from its primitives.
    """
    lattice = np.asarray(lattice, dtype=np.float64)
    grid = tuple(int(v) for v in grid)
    nprim = norb * prims_per_orb
    alphas = rng.uniform(*alpha_range, size=nprim)
    coeffs = rng.uniform(*coeff_range, size=nprim)
    if centres is None:
        frac = rng.uniform(0.0, 1.0, size=(nprim, 3))
        centres = frac @ lattice
    centres = np.asarray(centres, dtype=np.float64).reshape(nprim, 3)
    prims = [(float(alphas[a]), centres[a].copy()) for a in range(nprim)]
    G = np.stack([periodic_gaussian(grid, lattice, centres[a], alphas[a], images) for a in range(nprim)])
    Cblock = np.zeros((norb, nprim))
    for i in range(norb):
        sl = slice(i * prims_per_orb, (i + 1) * prims_per_orb)
        Cblock[i, sl] = coeffs[sl]
    chi = np.tensordot(Cblock, G, axes=(1, 0))
    dV = abs(np.linalg.det(lattice)) / (grid[0] * grid[1] * grid[2])
    phi, C = loewdin(chi, dV)
    D = C @ Cblock
    return phi, prims, D


# ----------------------------------------------------------------------------------------
# Water-like and cluster-like localized orbitals
# ----------------------------------------------------------------------------------------

_TETRA = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) / math.sqrt(3.0)


def _rsa_sites_periodic(nsites, lattice, dmin, rng, max_tries=200000):
    """Random sequential addition in a periodic orthorhombic cell with minimum-image distance >= dmin."""
    Ls = np.diag(lattice)
    sites = []
    tries = 0
    while len(sites) < nsites:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("site placement failed; lower the density or dmin")
        p = rng.uniform(0.0, 1.0, size=3) * Ls
        ok = True
        for q in sites:
            d = p - q
            d -= Ls * np.round(d / Ls)
            if d @ d < dmin * dmin:
                ok = False
                break
        if ok:
            sites.append(p)
    return np.array(sites)


def _rsa_sites_sphere(nsites, centre, radius, dmin, rng, max_tries=200000):
    sites = []
    tries = 0
    while len(sites) < nsites:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("site placement failed; lower dmin")
        v = rng.uniform(-1.0, 1.0, size=3)
        if v @ v > 1.0:
            continue
        p = centre + radius * v
        if all((p - q) @ (p - q) >= dmin * dmin for q in sites):
            sites.append(p)
    return np.array(sites)


def _orbital_centres(sites, rng, bond=0.9, lone=0.6):
    """Four centres per site along a randomly rotated tetrahedron: two 'bond' and two 'lone-pair'."""
    out = []
    for s in sites:
        R = _random_rotation(rng)
        dirs = _TETRA @ R.T
        out.append(s + bond * dirs[0])
        out.append(s + bond * dirs[1])
        out.append(s + lone * dirs[2])
        out.append(s + lone * dirs[3])
    return np.array(out)


def _spread_orbitals(grid, lattice, centres, spreads, images=1):
    """chi_k = exp(-|r - c_k|^2 / (2 s_k^2)), periodised."""
    return np.stack(
        [periodic_gaussian(grid, lattice, c, 1.0 / (2.0 * s * s), images) for c, s in zip(centres, spreads)]
    )


def water_like(nmol: int, cell: float, grid, rng, rho_cut=1e-3, dmin=4.6, spread=(0.8, 1.4), name="water"):
    lattice = np.diag([cell, cell, cell]).astype(np.float64)
    sites = _rsa_sites_periodic(nmol, lattice, dmin, rng)
    centres = _orbital_centres(sites, rng)
    spreads = rng.uniform(*spread, size=len(centres))
    chi = _spread_orbitals(grid, lattice, centres, spreads)
    dV = cell**3 / (grid[0] * grid[1] * grid[2])
    phi, _ = loewdin(chi, dV)
    return Workload(
        name=name,
        phi=phi,
        lattice=lattice,
        rho_cut=rho_cut,
        spin_factor=2.0,
        meta={"centres": centres, "spreads": spreads, "sites": sites},
    )


def enzyme_like(
    rng,
    ncentres=112,
    cell=(38.0, 34.0, 30.0),
    grid=(160, 144, 128),
    radius=9.0,
    dmin=3.6,
    nsnap=8,
    step=0.05,
    rho_cut=1e-3,
    spread=(0.8, 1.4),
):
    """A compact cluster of localized orbitals in a mostly empty cell, with ``nsnap`` snapshots.

    Sites fill a sphere of the given radius at the cell centre; each later snapshot moves every
    orbital centre by ``step`` bohr in a random direction and re-orthonormalises.
    """
    lattice = np.diag(cell).astype(np.float64)
    ctr = 0.5 * np.array(cell)
    nsites = ncentres // 4
    sites = _rsa_sites_sphere(nsites, ctr, radius - 0.9, dmin, rng)
    centres = _orbital_centres(sites, rng)
    spreads = rng.uniform(*spread, size=len(centres))
    dV = float(np.prod(cell)) / (grid[0] * grid[1] * grid[2])
    snaps = []
    for k in range(nsnap):
        if k > 0:
            d = rng.standard_normal(centres.shape)
            d /= np.linalg.norm(d, axis=1, keepdims=True)
            centres = centres + step * d
        chi = _spread_orbitals(grid, lattice, centres, spreads)
        phi, _ = loewdin(chi, dV)
        snaps.append(
            Workload(
                name=f"enzyme_snap{k}",
                phi=phi,
                lattice=lattice,
                rho_cut=rho_cut,
                spin_factor=2.0,
                meta={"centres": centres.copy(), "spreads": spreads},
            )
        )
    return snaps


def moved_snapshot(w: Workload, step: float, rng) -> Workload:
    """The next snapshot of a water_like workload: every orbital centre moved by ``step`` bohr in a
    random direction, same spreads, re-orthonormalised (the snapshot recipe of enzyme_like)."""
    centres = np.asarray(w.meta["centres"], dtype=np.float64)
    d = rng.standard_normal(centres.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centres = centres + step * d
    chi = _spread_orbitals(w.grid, w.lattice, centres, w.meta["spreads"])
    phi, _ = loewdin(chi, w.dV)
    meta = dict(w.meta, centres=centres)
    return Workload(name=w.name + "_moved", phi=phi, lattice=w.lattice, rho_cut=w.rho_cut,
                    spin_factor=w.spin_factor, meta=meta)


def batched_set(rng, nbuild=24, norbs=(64, 96, 128, 192, 256), grids=(72, 96, 108, 128), rho_cut=1e-3):
    """Descriptors (n, grid, cell) of uneven builds at water density; orbitals drawn lazily.

    Returns a list of (norb, N, cell, seed) so that callers can generate one build at a time.
    """
    out = []
    for b in range(nbuild):
        n = int(rng.choice(norbs))
        N = int(rng.choice(grids))
        cell = WATER_CELL_32 * (n / 128.0) ** (1.0 / 3.0)
        out.append((n, N, cell, int(rng.integers(1 << 31))))
    return out


# ----------------------------------------------------------------------------------------
# The named configurations (seed = 1000 + config number)
# ----------------------------------------------------------------------------------------


def config1(seed: int = 1001, grid=(32, 32, 32), cell=15.0, norb=16) -> Workload:
    """16 orbitals of 3 s-Gaussians each, cubic 15 bohr cell, 32^3 grid, all pairs, f = 2."""
    rng = np.random.default_rng(seed)
    lattice = np.diag([cell, cell, cell]).astype(np.float64)
    phi, prims, D = gaussian_orbitals(grid, lattice, norb, 3, rng)
    return Workload("config1_plain_16orb_32c", phi, lattice, 0.0, 2.0, {"prims": prims, "D": D})


def config2(seed: int = 1002, grid=(96, 96, 96), rho_cut=1e-3) -> Workload:
    """128 water-like localized orbitals in an 18.63 bohr cube on a 96^3 grid."""
    rng = np.random.default_rng(seed)
    return water_like(32, WATER_CELL_32, grid, rng, rho_cut=rho_cut, name="water32_128orb_96c")


def config3(seed: int = 1003, grid=(128, 128, 128), rho_cut=1e-3) -> Workload:
    """256 water-like localized orbitals in a 23.47 bohr cube on a 128^3 grid."""
    rng = np.random.default_rng(seed)
    return water_like(64, WATER_CELL_64, grid, rng, rho_cut=rho_cut, name="water64_256orb_128c")


def config4(seed: int = 1004, builds=None):
    """The 24 uneven builds of the batched configuration (or the ones listed in ``builds``): n from
    {64, ..., 256}, N^3 from {72^3, ..., 128^3}, cells scaled to water density, rho_cut 1e-3."""
    specs = batched_set(np.random.default_rng(seed))
    out = []
    for b in (range(len(specs)) if builds is None else builds):
        n, N, cell, s = specs[b]
        out.append(water_like(n // 4, cell, (N, N, N), np.random.default_rng(s), rho_cut=1e-3,
                              name=f"water{n // 4}_{n}orb_{N}c"))
    return out


def config5(seed: int = 1005, nsnap: int = 8):
    rng = np.random.default_rng(seed)
    return enzyme_like(rng, nsnap=nsnap)


# ----------------------------------------------------------------------------------------
# Seeded probes for comparing whole-grid outputs at full size
# ----------------------------------------------------------------------------------------


def sample_points(npts: int, k: int, seed: int) -> np.ndarray:
    """k distinct flat grid indices drawn uniformly (seeded), sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(npts, size=min(k, npts), replace=False)).astype(np.int64)


def probe_vectors(phi: np.ndarray, dV: float, seed: int) -> np.ndarray:
    """Two seeded test vectors for the ACE application, shape (2,) + grid, each with dV sum psi^2 = 1:
    psi_0 a random combination of the orbitals (inside their span), psi_1 white noise on the grid."""
    rng = np.random.default_rng(seed)
    n = phi.shape[0]
    c = rng.standard_normal(n)
    a = np.tensordot(c, phi, axes=(0, 0))
    b = rng.standard_normal(phi.shape[1:])
    out = np.stack([a, b])
    for v in out:
        v /= np.sqrt(dV * float((v * v).sum()))
    return out
