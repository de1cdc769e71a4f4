"""Precision of the GPU forms against the FP64 oracle at the full configuration sizes.

The stored oracle values (tests/golden/, written by make_golden.py from oracle/ and the input
generators only) hold, per build: E_x, the oracle's pair list, and for the two water-like
configurations xi at seeded grid points (every row), K phi_k at those points for every orbital,
and K psi for two seeded probe vectors (App. A: xi = W L^-T; section II: K psi = -xi (dV xi^T psi)).

The GPU builds here run on the oracle's own pair list (ace_build_pairs), so that the comparison
measures arithmetic and not the screen; the screen's own decisions are checked against the
oracle's list outside the band of 1e-6 rho_cut.  Errors checked (and printed):
  |dE_x| per orbital, ||K phi - K_oracle phi|| / ||K_oracle phi|| over every orbital,
  ||K psi - K_oracle psi|| / ||K_oracle psi|| for the probes, ||xi - xi_oracle|| / ||xi_oracle||.
"""

import json
import os

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from paper_2101_03155_gb300 import ace as abi
from gpu_helpers import (FP64_ARRAY_RTOL, FP64_EX_TOL, MIXED_EX_TOL_PER_ORB, MIXED_KPHI_RTOL, MIXED_KPSI_RTOL,
                         MIXED_XI_RTOL, gpu_build, mask_from_pairs, rel_max, screen_band)
from workloads.generators import config2, config3, config4, config5, probe_vectors

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()
    oracle.build()


def golden(key):
    """(JSON entry, arrays) of one stored oracle build."""
    values = json.load(open(os.path.join(GOLD, "oracle_values.json")))
    if key not in values:
        pytest.skip(f"no stored oracle values for {key} (tests/golden/make_golden.py writes them)")
    entry = values[key]
    arrays = dict(np.load(os.path.join(GOLD, entry["arrays"])))
    return entry, arrays


def _dtype(prec):
    import torch

    return torch.float64 if prec == ace.ACE_FP64 else torch.float32


def sampled_errors(op, w, arrays, prec):
    """Errors of the GPU operator at the stored sample points: xi (every row), K phi_k (every
    orbital, through ace_apply on the whole grid) and K psi of the two probe vectors."""
    import torch

    n, N = w.norb, w.npts
    dt = _dtype(prec)
    idx = torch.from_numpy(arrays["idx"]).cuda()
    xi = torch.empty((n, N), dtype=dt, device="cuda")
    ace.ace_get(op, abi.ACE_GET_XI, xi, torch.cuda.current_stream())
    xi_s = xi[:, idx].double().cpu().numpy()
    del xi
    phi = torch.from_numpy(w.phi).to(device="cuda", dtype=dt)
    out = torch.empty_like(phi)
    ace.ace_apply(op, phi, out, torch.cuda.current_stream())
    kphi_s = out.reshape(n, N)[:, idx].double().cpu().numpy()
    del phi, out
    psi = torch.from_numpy(probe_vectors(w.phi, w.dV, int(arrays["probe_seed"]))).to(device="cuda", dtype=dt)
    kout = torch.empty_like(psi)
    ace.ace_apply(op, psi, kout, torch.cuda.current_stream())
    kpsi_s = kout.reshape(2, N)[:, idx].double().cpu().numpy()
    fro = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))  # noqa: E731
    return {"xi_rel": fro(xi_s, arrays["xi"]), "xi_max": rel_max(xi_s, arrays["xi"]),
            "kphi_rel": fro(kphi_s, arrays["kphi"]), "kphi_max": rel_max(kphi_s, arrays["kphi"]),
            "kpsi_rel": max(fro(kpsi_s[c], arrays["kpsi"][c]) for c in range(2)),
            "kpsi_max": max(rel_max(kpsi_s[c], arrays["kpsi"][c]) for c in range(2))}


def _pairs_build(w, pairs, prec):
    import torch

    x = torch.from_numpy(w.phi).to(device="cuda", dtype=_dtype(prec))
    d = ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=w.spin_factor, prec=prec)
    return ace.ace_build_pairs(d, x, pairs, torch.cuda.current_stream())


def _check_report(key, w, prec):
    entry, arrays = golden(key)
    op = _pairs_build(w, arrays["pairs"], prec)
    e = ace.exchange_energy(op)
    err = sampled_errors(op, w, arrays, prec)
    err["ex_per_orb"] = abs(e - entry["E_x"]) / w.norb
    print(f"\n{key} {'fp64' if prec == ace.ACE_FP64 else 'mixed'}: {json.dumps(err)}")
    if prec == ace.ACE_FP64:
        assert abs(e - entry["E_x"]) <= FP64_EX_TOL
        assert err["xi_max"] <= FP64_ARRAY_RTOL
        assert err["kphi_max"] <= FP64_ARRAY_RTOL
        assert err["kpsi_max"] <= FP64_ARRAY_RTOL
    else:
        assert err["ex_per_orb"] <= MIXED_EX_TOL_PER_ORB
        assert err["kphi_rel"] <= MIXED_KPHI_RTOL
        assert err["kpsi_rel"] <= MIXED_KPSI_RTOL
        assert err["xi_rel"] <= MIXED_XI_RTOL
    op.close()


@pytest.mark.parametrize("prec", [ace.ACE_MIXED, ace.ACE_FP64])
def test_water32_precision_report(prec):
    """Config 2 (128 orbitals, 96^3): E_x, xi, K phi and K psi against the oracle."""
    _check_report("water32_128orb_96c_rhocut1e-3", config2(), prec)


@pytest.mark.parametrize("prec", [ace.ACE_MIXED, ace.ACE_FP64])
def test_water64_precision_report(prec):
    """Config 3 (256 orbitals, 128^3): E_x, xi, K phi and K psi against the oracle."""
    _check_report("water64_256orb_128c_rhocut1e-3", config3(), prec)


@pytest.mark.parametrize("prec", [ace.ACE_MIXED, ace.ACE_FP64])
def test_water64_screened_build(prec):
    """Config 3 through the screen: the pair list is the oracle's outside the band, E_x within the
    target of its form."""
    w = config3()
    entry, arrays = golden("water64_256orb_128c_rhocut1e-3")
    g = gpu_build(w.phi, w.lattice, prec, rho_cut=w.rho_cut)
    assert g["status"] == 0
    mask_ref = mask_from_pairs(arrays["pairs"], w.norb)
    O_ref, _ = oracle.screen(w.phi, w.lattice, w.rho_cut)
    band = screen_band(O_ref, w.rho_cut)
    assert np.array_equal(g["mask"] | band, mask_ref | band)
    if np.array_equal(g["mask"], mask_ref):
        tol = FP64_EX_TOL if prec == ace.ACE_FP64 else MIXED_EX_TOL_PER_ORB * w.norb
        assert abs(g["E_x"] - entry["E_x"]) <= tol


@pytest.mark.parametrize("prec", [ace.ACE_MIXED, ace.ACE_FP64])
def test_enzyme_periodic_full_size(prec):
    """Config 5 snapshot 0 with the periodic kernel (112 orbitals, 160 x 144 x 128): the screen's
    pair list and E_x against the oracle."""
    w = config5(nsnap=1)[0]
    entry, arrays = golden("enzyme_snap0_periodic")
    g = gpu_build(w.phi, w.lattice, prec, rho_cut=w.rho_cut)
    assert g["status"] == 0
    mask_ref = mask_from_pairs(arrays["pairs"], w.norb)
    O_ref, _ = oracle.screen(w.phi, w.lattice, w.rho_cut)
    band = screen_band(O_ref, w.rho_cut)
    assert np.array_equal(g["mask"] | band, mask_ref | band)
    p = _pairs_build(w, arrays["pairs"], prec)
    e = ace.exchange_energy(p)
    tol = FP64_EX_TOL if prec == ace.ACE_FP64 else MIXED_EX_TOL_PER_ORB * w.norb
    assert abs(e - entry["E_x"]) <= tol
    print(f"\nenzyme_snap0_periodic {'fp64' if prec == ace.ACE_FP64 else 'mixed'}: "
          f"ex_per_orb {abs(e - entry['E_x']) / w.norb:.3e}")


BATCHED = [1, 15, 12]  # 64 orbitals on 72^3, 96 on 108^3, 64 on 128^3


@pytest.mark.parametrize("prec", [ace.ACE_MIXED, ace.ACE_FP64])
def test_batched_uneven_builds_against_oracle(prec):
    """Three builds of the uneven batched set in one ace_build_batched call (72^3, 108^3 and 128^3
    planes): each screen's pair list and each E_x against the oracle."""
    import torch

    ws = config4(builds=BATCHED)
    keys = [f"batched24_b{b}_{w.norb}orb_{w.grid[0]}c" for b, w in zip(BATCHED, ws)]
    descs = [ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=w.spin_factor, prec=prec)
             for w in ws]
    phis = [torch.from_numpy(w.phi).to(device="cuda", dtype=_dtype(prec)) for w in ws]
    ops = ace.ace_build_batched(descs, phis, torch.cuda.current_stream())
    for w, key, op in zip(ws, keys, ops):
        entry, arrays = golden(key)
        pairs = abi.get_numpy(op, abi.ACE_GET_PAIRS)
        mask = mask_from_pairs(pairs, w.norb)
        mask_ref = mask_from_pairs(arrays["pairs"], w.norb)
        O_ref, _ = oracle.screen(w.phi, w.lattice, w.rho_cut)
        band = screen_band(O_ref, w.rho_cut)
        assert np.array_equal(mask | band, mask_ref | band), key
        e = ace.exchange_energy(op)
        if np.array_equal(mask, mask_ref):
            tol = FP64_EX_TOL if prec == ace.ACE_FP64 else MIXED_EX_TOL_PER_ORB * w.norb
            assert abs(e - entry["E_x"]) <= tol, key
        print(f"\n{key} {'fp64' if prec == ace.ACE_FP64 else 'mixed'}: ex_per_orb {abs(e - entry['E_x']) / w.norb:.3e}")
        op.close()
