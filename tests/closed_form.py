"""Closed-form Fourier coefficients of sampled products of periodised Gaussians.

Used to pin the oracle without an FFT.  For g_a(r) = sum_S exp(-alpha_a |r - A_a - S|^2) the
product g_a g_b is lattice-periodic with Fourier coefficients (Gaussian product theorem)

    f_ab(G) = (1/Omega) sum_T (pi/p)^{3/2} exp(-mu |A_a - A_b - T|^2) exp(-|G|^2/(4p)) exp(-i G.P_T),
    p = alpha_a + alpha_b,  mu = alpha_a alpha_b / p,  P_T = (alpha_a A_a + alpha_b (A_b + T)) / p,

and by Poisson summation the grid coefficient (1/N) sum_r f(x_r) exp(-i G_m.x_r) is the sum of
f_ab over the aliases G_m + K, K = sum_k n_k N_k b_k.  With orbitals phi_i = sum_a D_ia g_a this
gives every pair-density coefficient, hence (ij|ij) = Omega sum_{m != 0} 4 pi/|G_m|^2 |rho~_ij(m)|^2,
without sampling or transforming anything on the grid.
"""

from __future__ import annotations

import itertools

import numpy as np


def reciprocal(lattice: np.ndarray) -> np.ndarray:
    """Rows b_k with a_j . b_k = 2 pi delta_jk."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(lattice, dtype=np.float64)).T


def wrapped_indices(grid) -> np.ndarray:
    """(N, 3) integer m_k in [-N_k/2, N_k/2), C order over (i1, i2, i3)."""
    axes = [np.where(2 * np.arange(n) < n, np.arange(n), np.arange(n) - n) for n in grid]
    return np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)


def box_kernel(lattice, grid) -> np.ndarray:
    """4 pi/|G_m|^2 on the FFT box, 0 at G = 0, averaged over the +-N_k/2 choices at Nyquist."""
    B = reciprocal(lattice)
    m = wrapped_indices(grid).astype(np.float64)
    nyq = np.stack([(np.asarray(grid)[k] % 2 == 0) & (m[:, k] == -grid[k] // 2) for k in range(3)], axis=1)
    total = np.zeros(len(m))
    count = np.zeros(len(m))
    for signs in itertools.product((1.0, -1.0), repeat=3):
        s = np.array(signs)
        allowed = np.all((s > 0) | nyq, axis=1)
        G = (m * s) @ B
        g2 = np.einsum("ij,ij->i", G, G)
        with np.errstate(divide="ignore"):
            val = np.where(g2 > 0, 4.0 * np.pi / np.where(g2 > 0, g2, 1.0), 0.0)
        total += np.where(allowed, val, 0.0)
        count += allowed
    return (total / count).reshape(tuple(grid))


def prim_pair_coefficients(prims, lattice, grid, nalias: int = 2, nimg: int = 3, tol: float = 1e-30):
    """rho~_ab(m) for every primitive pair: array (nprim, nprim, N) complex."""
    lattice = np.asarray(lattice, dtype=np.float64)
    B = reciprocal(lattice)
    omega = abs(np.linalg.det(lattice))
    G = wrapped_indices(grid).astype(np.float64) @ B
    shifts = np.array(list(itertools.product(range(-nalias, nalias + 1), repeat=3)), dtype=np.float64)
    K = (shifts * np.asarray(grid, dtype=np.float64)) @ B
    Gall = G[:, None, :] + K[None, :, :]
    G2 = np.einsum("mak,mak->ma", Gall, Gall)
    imgs = np.array(list(itertools.product(range(-nimg, nimg + 1), repeat=3)), dtype=np.float64) @ lattice
    n = len(prims)
    out = np.zeros((n, n, len(G)), dtype=np.complex128)
    for a in range(n):
        for b in range(a, n):
            aa, Aa = prims[a]
            bb, Ab = prims[b]
            p = aa + bb
            mu = aa * bb / p
            d = (Aa - Ab)[None, :] - imgs
            cT = (np.pi / p) ** 1.5 * np.exp(-mu * np.einsum("tk,tk->t", d, d))
            keep = cT > tol * cT.max()
            acc = np.zeros(Gall.shape[:2], dtype=np.complex128)
            for T, c in zip(imgs[keep], cT[keep]):
                P = (aa * Aa + bb * (Ab + T)) / p
                acc += c * np.exp(-1j * (Gall @ P))
            f = np.exp(-G2 / (4.0 * p)) * acc / omega
            out[a, b] = f.sum(axis=1)
            out[b, a] = out[a, b]
    return out


def orbital_pair_coefficients(D, prim_coeffs, i, j):
    """rho~_ij(m) = sum_ab D_ia D_jb rho~_ab(m)."""
    return np.einsum("a,b,abm->m", D[i], D[j], prim_coeffs)


def pair_energies(D, prim_coeffs, lattice, grid):
    """Matrix of (ij|ij) = Omega sum_m K(m) |rho~_ij(m)|^2 over orbital pairs."""
    omega = abs(np.linalg.det(np.asarray(lattice)))
    Kb = box_kernel(lattice, grid).reshape(-1)
    n = D.shape[0]
    E = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            r = orbital_pair_coefficients(D, prim_coeffs, i, j)
            E[i, j] = E[j, i] = omega * np.sum(Kb * np.abs(r) ** 2)
    return E
