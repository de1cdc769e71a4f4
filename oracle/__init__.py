"""FP64 CPU oracle for the screened ACE build (arXiv:2101.03155, Eq. vx, Eq. e:vij, App. A).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke()`` and by the
bench's CPU-baseline leg.  The product path (``paper_2101_03155_gb300``) never imports it.

The arithmetic lives in ``ace_oracle.c`` (plain C, double precision, its own mixed-radix FFT);
this module compiles it with gcc and marshals numpy arrays.  Readings of the paper that the
oracle fixes are listed at the top of ``ace_oracle.c``.
"""

from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ace_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libace_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_ubyte)


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp shared library from one C file (no -march flags: builds on x86 and Arm)."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library if missing or stale."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if stale:
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


def bind(path: str):
    """Load an oracle library from ``path`` and declare its C signatures."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = bind(build())
        return _lib


@contextlib.contextmanager
def using(lib):
    """Route the module-level functions through another loaded oracle library (tests only)."""
    global _lib
    prev = _load()
    _lib = lib
    try:
        yield lib
    finally:
        _lib = prev


def _declare(lib):
    """C signatures of the exported oracle entry points."""
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_fft3d.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    _i, _d = ctypes.c_int, ctypes.c_double
    lib.oracle_inscribed_radius.argtypes = [_dp]
    lib.oracle_inscribed_radius.restype = _d
    lib.oracle_coulomb_kernel.argtypes = [_dp, _i, _i, _i, _i, _d, _dp]
    lib.oracle_pair_potential.argtypes = [_dp, _dp, _i, _i, _i, _dp, _i, _d, _dp]
    lib.oracle_pair_energy.argtypes = [_dp, _dp, _i, _i, _i, _dp, _i, _d]
    lib.oracle_pair_energy.restype = ctypes.c_double
    lib.oracle_screen.argtypes = [_dp, ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_double, _dp, _up]
    lib.oracle_exchange_w.argtypes = [
        _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, _up, _ip,
        ctypes.c_int, _dp,
    ]
    lib.oracle_ace_from_w.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_long, ctypes.c_double, _dp, _dp, _dp, _dp]
    lib.oracle_ace_apply.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_long, ctypes.c_double, _dp]
    _lp = ctypes.POINTER(ctypes.c_long)
    lib.oracle_ace_apply_at.argtypes = [_dp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_long, ctypes.c_double, _lp,
                                        ctypes.c_int, _dp, _dp]
    lib.oracle_exchange_energy.argtypes = [_dp, ctypes.c_int, ctypes.c_double]
    lib.oracle_scdm_select.argtypes = [_dp, ctypes.c_int, ctypes.c_long, ctypes.c_int, _ip]
    lib.oracle_exchange_energy.restype = ctypes.c_double


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def fft3d(z: np.ndarray, sign: int = -1) -> np.ndarray:
    """Unnormalised 3D DFT, sum_r z(r) exp(sign * 2 pi i m.r/N), of a complex (n1, n2, n3) array."""
    z = np.ascontiguousarray(z, dtype=np.complex128).copy()
    n1, n2, n3 = z.shape
    buf = z.view(np.float64)
    _load().oracle_fft3d(_ptr(buf), n1, n2, n3, int(sign))
    return z


PERIODIC, TRUNCATED = 0, 1  # Coulomb kernel kinds: 4 pi/|G|^2 (G = 0 dropped); 1/r cut off at r_cut


def inscribed_radius(lattice) -> float:
    """Radius of the largest sphere inside the cell (the default cut-off of the truncated kernel)."""
    return float(_load().oracle_inscribed_radius(_ptr(_f64(lattice).reshape(3, 3))))


def coulomb_kernel(lattice, grid, kind: int = PERIODIC, r_cut: float = 0.0) -> np.ndarray:
    """Kernel on the FFT box, Nyquist-averaged, shape grid: PERIODIC 4 pi/|G_m|^2 with G = 0 -> 0;
    TRUNCATED 4 pi (1 - cos(|G| r_cut))/|G|^2 with G = 0 -> 2 pi r_cut^2 (r_cut <= 0: inscribed radius)."""
    lat = _f64(lattice).reshape(3, 3)
    K = np.empty(tuple(grid), dtype=np.float64)
    _load().oracle_coulomb_kernel(_ptr(lat), *[int(g) for g in grid], int(kind), float(r_cut), _ptr(K))
    return K


def pair_potential(phi_i, phi_j, lattice, kind: int = PERIODIC, r_cut: float = 0.0) -> np.ndarray:
    """v_ij(r) of Eq. (e:vij) on the grid."""
    a, b = _f64(phi_i), _f64(phi_j)
    lat = _f64(lattice).reshape(3, 3)
    v = np.empty_like(a)
    _load().oracle_pair_potential(_ptr(a), _ptr(b), *a.shape, _ptr(lat), int(kind), float(r_cut), _ptr(v))
    return v


def pair_energy(phi_i, phi_j, lattice, kind: int = PERIODIC, r_cut: float = 0.0) -> float:
    """(ij|ij) = dV sum_r phi_i phi_j v_ij."""
    a, b = _f64(phi_i), _f64(phi_j)
    lat = _f64(lattice).reshape(3, 3)
    return float(_load().oracle_pair_energy(_ptr(a), _ptr(b), *a.shape, _ptr(lat), int(kind), float(r_cut)))


def screen(phi, lattice, rho_cut: float):
    """O_ij = dV sum_r |phi_i phi_j| and the keep-mask (O_ij >= rho_cut, diagonal kept)."""
    phi = _f64(phi)
    n = phi.shape[0]
    npts = int(np.prod(phi.shape[1:]))
    dV = abs(np.linalg.det(_f64(lattice).reshape(3, 3))) / npts
    O = np.empty((n, n))
    mask = np.empty((n, n), dtype=np.uint8)
    _load().oracle_screen(_ptr(phi), n, npts, dV, float(rho_cut), _ptr(O), _ptr(mask, _up))
    return O, mask.astype(bool)


def exchange_w(phi, lattice, mask=None, rows=None, kind: int = PERIODIC, r_cut: float = 0.0) -> np.ndarray:
    """W_i = sum_j v_ij phi_j (Eq. vx with W = -V_X phi) for the requested rows."""
    phi = _f64(phi)
    n = phi.shape[0]
    grid = phi.shape[1:]
    lat = _f64(lattice).reshape(3, 3)
    rows_arr = None if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    nrows = n if rows_arr is None else len(rows_arr)
    W = np.empty((nrows,) + tuple(grid))
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    rc = _load().oracle_exchange_w(
        _ptr(phi), n, *grid, _ptr(lat), int(kind), float(r_cut),
        None if m is None else _ptr(m, _up),
        None if rows_arr is None else _ptr(rows_arr, _ip),
        nrows, _ptr(W),
    )
    if rc != 0:
        raise MemoryError("oracle_exchange_w: allocation failed")
    return W


def ace_from_w(phi, W, dV: float, want_xi: bool = True):
    """Appendix A from W: raw and symmetrised M, L = chol(-M), xi = W L^-T."""
    phi, W = _f64(phi), _f64(W)
    n = phi.shape[0]
    npts = int(np.prod(phi.shape[1:]))
    M_raw = np.empty((n, n))
    M = np.empty((n, n))
    L = np.empty((n, n))
    xi = np.empty_like(W) if want_xi else None
    st = _load().oracle_ace_from_w(
        _ptr(phi), _ptr(W), n, npts, float(dV), _ptr(M_raw), _ptr(M), _ptr(L),
        None if xi is None else _ptr(xi),
    )
    return {"M_raw": M_raw, "M": M, "L": L, "xi": xi, "status": int(st)}


def ace_apply(xi, psi, dV: float) -> np.ndarray:
    """K psi = -xi (dV xi^T psi)."""
    xi, psi = _f64(xi), _f64(psi)
    n = xi.shape[0]
    m = psi.shape[0]
    npts = int(np.prod(xi.shape[1:]))
    out = np.empty_like(psi)
    _load().oracle_ace_apply(_ptr(xi), n, _ptr(psi), m, npts, float(dV), _ptr(out))
    return out


def exchange_energy(M, spin_factor: float) -> float:
    M = _f64(M)
    return float(_load().oracle_exchange_energy(_ptr(M), M.shape[0], float(spin_factor)))


def ace_build(phi, lattice, rho_cut: float = 0.0, spin_factor: float = 2.0, mask=None, want_xi=True,
              kind: int = PERIODIC, r_cut: float = 0.0):
    """Whole build: optional screen (rho_cut > 0 and no explicit mask), W, M, L, xi, E_x."""
    phi = _f64(phi)
    lat = _f64(lattice).reshape(3, 3)
    npts = int(np.prod(phi.shape[1:]))
    dV = abs(np.linalg.det(lat)) / npts
    O = None
    if mask is None and rho_cut > 0:
        O, mask = screen(phi, lat, rho_cut)
    W = exchange_w(phi, lat, mask=mask, kind=kind, r_cut=r_cut)
    res = ace_from_w(phi, W, dV, want_xi=want_xi)
    res.update(W=W, mask=mask, O=O, dV=dV)
    res["E_x"] = exchange_energy(res["M"], spin_factor)
    return res


def scdm_select(psi, npiv=None) -> np.ndarray:
    """Greedy column-pivoted QR selection on Psi^T: the grid indices of the SCDM columns."""
    psi = _f64(psi)
    n = psi.shape[0]
    npts = int(np.prod(psi.shape[1:]))
    k = n if npiv is None else int(npiv)
    piv = np.empty(k, dtype=np.int32)
    _load().oracle_scdm_select(_ptr(psi), n, npts, k, _ptr(piv, _ip))
    return piv


def scdm(psi, dV: float):
    """SCDM localisation: columns C of the density matrix P = Psi Psi^T (rows of Psi at the selected
    grid points, M = Psi(C)^T), orthonormalised symmetrically under dV:
    Phi = Psi^T M (M^T M)^{-1/2} (as rows [n][grid]).  Returns (Phi, pivots)."""
    piv = scdm_select(psi)
    phi, _ = scdm_orthonormalise(psi, piv)
    return phi, piv


def scdm_orthonormalise(psi, piv):
    """Second half of SCDM for given grid columns piv: U = M (M^T M)^{-1/2} with M[i][j] = psi_i(c_j),
    and Phi = U^T Psi.  Returns (Phi, U)."""
    psi = _f64(psi)
    n = psi.shape[0]
    flat = psi.reshape(n, -1)
    M = flat[:, np.asarray(piv)]          # M[i][j] = psi_i(c_j)
    S = M.T @ M                           # = dV Phi~^T Phi~ for orthonormal Psi
    w, V = np.linalg.eigh(S)
    U = M @ (V * (1.0 / np.sqrt(w))) @ V.T
    phi = (U.T @ flat).reshape(psi.shape)
    return phi, U


def ace_apply_at(xi, psi, dV: float, idx):
    """K psi = -xi (dV xi^T psi) at the flat grid indices idx only.  Returns (C, out) with
    C = dV xi^T psi (norb x m) and out (m x len(idx))."""
    xi, psi = _f64(xi), _f64(psi)
    n, m = xi.shape[0], psi.shape[0]
    npts = int(np.prod(xi.shape[1:]))
    ix = np.ascontiguousarray(idx, dtype=np.int64)
    if ix.size and (ix.min() < 0 or ix.max() >= npts):
        raise IndexError("grid index out of range")
    C = np.empty((n, m))
    out = np.empty((m, len(ix)))
    _load().oracle_ace_apply_at(_ptr(xi), n, _ptr(psi), m, npts, float(dV), ix.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                len(ix), _ptr(C), _ptr(out))
    return C, out
