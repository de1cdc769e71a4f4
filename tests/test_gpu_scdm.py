"""SCDM localisation on the GPU (ace_scdm) against the oracle: the selected grid columns, the
orthogonal factor U and the localized orbitals Phi = U^T Psi, through the C ABI.

Where FP32 projections (mixed form) or rounding order (FP64 form) may break a near-tie between
grid points differently from the oracle, the GPU's own pivot sequence is checked for validity:
at every step its pivot has the largest residual norm, to within the stated tolerance, given the
pivots chosen before it.  U and Phi are then compared with the oracle's orthonormalisation on
the GPU's pivots."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from gpu_helpers import MIXED_W_RTOL, gpu_build, rel_max
from workloads.generators import config2, delocalised, gaussian_orbitals, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()
    oracle.build()


def _gpu_scdm(psi, prec, host=False, io_dtype=None):
    import torch

    dt = io_dtype or (np.float64 if prec == ace.ACE_FP64 else np.float32)
    arr = np.ascontiguousarray(psi, dtype=dt)
    odt = dt
    if host:
        src = arr
        out = np.zeros(arr.shape, dtype=odt)
    else:
        src = torch.from_numpy(arr).cuda()
        out = torch.zeros(arr.shape, dtype=torch.float64 if odt == np.float64 else torch.float32, device="cuda")
    st, piv, U, nl = ace.ace_scdm(src, out, prec, stream=torch.cuda.current_stream(), check=False)
    torch.cuda.synchronize()
    phi = out if host else out.cpu().numpy()
    return {"status": st, "piv": piv, "U": U, "phi": np.asarray(phi, dtype=np.float64), "launches": nl, "input": arr}


def _check_pivots(psi, piv, tol, piv_ref=None):
    """Every pivot has the largest residual norm given the earlier pivots, to within
    tol * max |psi(r)|^2 (FP64 restatement of the greedy step, test side).  Up to the first step
    where piv and piv_ref differ they must agree exactly; at that step both picks must be tied to
    within the tolerance.  Returns the number of leading pivots equal to piv_ref."""
    n = psi.shape[0]
    X = np.asarray(psi, dtype=np.float64).reshape(n, -1)
    d = np.einsum("ir,ir->r", X, X)
    scale = tol * d.max()
    basis = []
    same = 0
    following = piv_ref is not None
    assert len(set(int(c) for c in piv)) == n
    for k, c in enumerate(piv):
        best = d.max()
        assert d[c] >= best - scale, f"step {k}: residual {d[c]} vs max {best}"
        if following:
            if piv_ref[k] == c:
                same += 1
            else:
                assert abs(d[c] - d[piv_ref[k]]) <= scale, f"step {k}: no tie between {c} and {piv_ref[k]}"
                following = False
        u = X[:, c].copy()
        for _ in range(2):
            for v in basis:
                u -= (v @ u) * v
        u /= np.linalg.norm(u)
        basis.append(u)
        d -= (u @ X) ** 2
        d[np.asarray(piv[: k + 1])] = -1.0
    return same


@pytest.fixture(scope="module")
def gauss16():
    lat = np.diag([12.0, 12.0, 12.0])
    grid = (24, 24, 24)
    phi_loc, _, _ = gaussian_orbitals(grid, lat, 16, 1, np.random.default_rng(41), alpha_range=(1.0, 2.0))
    return lat, phi_loc, delocalised(phi_loc, 43)


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_scdm_small(gauss16, prec):
    lat, phi_loc, psi = gauss16
    g = _gpu_scdm(psi, prec)
    assert g["status"] == 0, ace.ace_last_error()
    assert g["launches"] > 2 * 16
    x = g["input"].astype(np.float64)  # what the GPU saw
    piv_ref = oracle.scdm_select(x)
    if prec == ace.ACE_FP64:
        assert _check_pivots(x, g["piv"], 1e-12, piv_ref) == 16
        phi_ref, U_ref = oracle.scdm_orthonormalise(x, g["piv"])
        assert rel_max(g["U"], U_ref) <= 1e-10
        assert rel_max(g["phi"], phi_ref) <= 1e-10
    else:
        _check_pivots(x, g["piv"], 2e-5, piv_ref)
        phi_ref, U_ref = oracle.scdm_orthonormalise(x, g["piv"])
        assert rel_max(g["U"], U_ref) <= 1e-9
        assert rel_max(g["phi"], phi_ref) <= MIXED_W_RTOL
    # U is orthogonal and Phi orthonormal under dV; the localized set is recovered (each SCDM
    # orbital overlaps one Gaussian orbital almost entirely)
    dV = np.prod(np.diag(lat)) / psi[0].size
    assert np.abs(g["U"].T @ g["U"] - np.eye(16)).max() <= 1e-9
    P = g["phi"].reshape(16, -1)
    assert np.abs(dV * P @ P.T - np.eye(16)).max() <= (1e-10 if prec == ace.ACE_FP64 else 1e-5)
    ov = np.abs(dV * P @ phi_loc.reshape(16, -1).T)
    assert ov.max(axis=1).min() > 0.9


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_scdm_ragged(prec):
    """13 orbitals (a partial 16-orbital chunk) on 20 x 20 x 21 points (not a multiple of the
    tensor-core tile, so the left multiply takes its general kernel)."""
    lat = np.diag([10.0, 10.0, 10.5])
    grid = (20, 20, 21)
    phi_loc, _, _ = gaussian_orbitals(grid, lat, 13, 2, np.random.default_rng(51), alpha_range=(0.8, 2.0))
    psi = delocalised(phi_loc, 53)
    g = _gpu_scdm(psi, prec)
    assert g["status"] == 0, ace.ace_last_error()
    x = g["input"].astype(np.float64)
    piv_ref = oracle.scdm_select(x)
    tol = 1e-12 if prec == ace.ACE_FP64 else 2e-5
    same = _check_pivots(x, g["piv"], tol, piv_ref)
    if prec == ace.ACE_FP64:
        assert same == 13
    phi_ref, U_ref = oracle.scdm_orthonormalise(x, g["piv"])
    assert rel_max(g["U"], U_ref) <= 1e-9
    assert rel_max(g["phi"], phi_ref) <= (1e-10 if prec == ace.ACE_FP64 else MIXED_W_RTOL)


def test_scdm_host_buffers_and_conversion(gauss16):
    """Host input and output, FP64 arrays in the mixed form: the same result as device FP32 arrays."""
    _, _, psi = gauss16
    dev = _gpu_scdm(psi, ace.ACE_MIXED)
    host = _gpu_scdm(np.ascontiguousarray(psi, dtype=np.float32).astype(np.float64), ace.ACE_MIXED, host=True,
                     io_dtype=np.float64)
    assert host["status"] == 0
    assert np.array_equal(host["piv"], dev["piv"])
    assert rel_max(host["phi"], dev["phi"]) <= 1e-6


def test_scdm_single_orbital():
    """n = 1: the pivot is the point of largest |psi|, U = sign psi(c) (the orthogonal 1 x 1 factor
    that M (M^T M)^{-1/2} gives)."""
    rng = np.random.default_rng(61)
    psi = rng.standard_normal((1, 8, 8, 8))
    g = _gpu_scdm(psi, ace.ACE_FP64)
    assert g["status"] == 0
    c = int(np.argmax(np.abs(psi.reshape(-1))))
    assert g["piv"][0] == c
    sign = np.sign(psi.reshape(-1)[c])
    assert g["U"][0, 0] == pytest.approx(sign, rel=1e-12)
    assert rel_max(g["phi"], sign * psi) <= 1e-14


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_scdm_rank_deficient_is_refused(gauss16, prec):
    """Two equal orbitals: the chosen columns are dependent and the call reports it."""
    _, _, psi = gauss16
    bad = psi.copy()
    bad[5] = bad[2]
    g = _gpu_scdm(bad, prec)
    assert g["status"] == ace.ace.ACE_ERR_NOT_POSDEF
    assert "rank" in ace.ace_last_error()


def test_scdm_localises_for_the_screen():
    """The purpose of the step in section II: SCDM orbitals of a delocalised 16-water-like set
    (64 orbitals, 64^3 points) give the same E_x (Eq. unit leaves it invariant), and the screen keeps
    about as few pairs as for the localized set the delocalised one was made from, far fewer than
    for the delocalised orbitals themselves."""
    w = water_like(16, 14.79, (64, 64, 64), np.random.default_rng(1011), rho_cut=1e-3, dmin=4.6)
    psi = delocalised(w.phi, 71)
    g = _gpu_scdm(psi, ace.ACE_FP64)
    assert g["status"] == 0
    x = psi.reshape(w.norb, -1)
    assert _check_pivots(x, g["piv"], 1e-12, oracle.scdm_select(x)) == w.norb
    phi = g["phi"].reshape(psi.shape)
    b_psi = gpu_build(psi, w.lattice, ace.ACE_FP64, rho_cut=0.0)
    b_phi = gpu_build(phi, w.lattice, ace.ACE_FP64, rho_cut=0.0)
    assert b_phi["E_x"] == pytest.approx(b_psi["E_x"], rel=1e-10)
    npairs = {name: len(gpu_build(v, w.lattice, ace.ACE_FP64, rho_cut=w.rho_cut)["pairs"])
              for name, v in (("psi", psi), ("scdm", phi), ("localized", w.phi))}
    assert npairs["scdm"] <= 1.1 * npairs["localized"], npairs
    assert npairs["scdm"] < 0.6 * npairs["psi"], npairs


@pytest.mark.slow
@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_scdm_water32_full_size(prec):
    """128 delocalised orbitals on 96^3 points (the 32-water-like set, rotated): pivots checked
    against the oracle's greedy selection, U and sampled rows of Phi against its orthonormalisation."""
    w = config2()
    psi = delocalised(w.phi, 81)
    g = _gpu_scdm(psi, prec)
    assert g["status"] == 0, ace.ace_last_error()
    x = g["input"].astype(np.float64).reshape(w.norb, -1)
    del psi
    piv_ref = oracle.scdm_select(x)
    if prec == ace.ACE_FP64:
        assert _check_pivots(x, g["piv"], 1e-12, piv_ref) == w.norb
    else:
        _check_pivots(x, g["piv"], 2e-5, piv_ref)
    phi_ref, U_ref = oracle.scdm_orthonormalise(x, g["piv"])
    assert rel_max(g["U"], U_ref) <= 1e-9
    tol = 1e-10 if prec == ace.ACE_FP64 else MIXED_W_RTOL
    for i in (0, 63, 127):
        assert rel_max(g["phi"].reshape(w.norb, -1)[i], phi_ref[i]) <= tol, f"row {i}"
