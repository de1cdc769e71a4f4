"""ace_build_pairs: the build on a given pair list (the reuse step of a multiple-time-step run),
against the oracle with the same pair mask, through the C ABI."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from paper_2101_03155_gb300 import ace as abi
from gpu_helpers import FP64_ARRAY_RTOL, FP64_EX_TOL, MIXED_EX_TOL_PER_ORB, MIXED_W_RTOL, gpu_build, mask_from_pairs, rel_max
from workloads.generators import enzyme_like, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()
    oracle.build()


def _pairs_build(w, prec, pairs, host=False):
    import torch

    dt = np.float64 if prec == ace.ACE_FP64 else np.float32
    arr = np.ascontiguousarray(w.phi, dtype=dt)
    src = arr if host else torch.from_numpy(arr).cuda()
    d = ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=w.spin_factor, prec=prec)
    st, op = ace.ace_build_pairs(d, src, pairs, torch.cuda.current_stream(), check=False)
    out = {"status": st, "op": op}
    if op is not None:
        out["E_x"] = ace.exchange_energy(op)
        for key, what in (("W", abi.ACE_GET_W), ("M_raw", abi.ACE_GET_M_RAW), ("pairs", abi.ACE_GET_PAIRS),
                          ("O", abi.ACE_GET_OVERLAP)):
            out[key] = abi.get_numpy(op, what)
    return out


@pytest.fixture(scope="module")
def water_small():
    return water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_screened_list_replayed(water_small, prec):
    """The screen's own pair list given back: the same operator as the screened build."""
    w = water_small
    g = gpu_build(w.phi, w.lattice, prec, rho_cut=w.rho_cut)
    p = _pairs_build(w, prec, g["pairs"][::-1])  # order does not matter
    assert p["status"] == 0
    assert np.array_equal(p["pairs"], g["pairs"])
    assert not p["O"].any()
    tol = FP64_EX_TOL if prec == ace.ACE_FP64 else 0.1 * MIXED_EX_TOL_PER_ORB * w.norb  # FP32 atomics: order varies run to run
    assert abs(p["E_x"] - g["E_x"]) <= tol


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_arbitrary_list_against_oracle(water_small, prec):
    """A list without its diagonal pairs and with some distant pairs: W and M_raw of the oracle on
    the same mask (the operator need not be definite, so the Cholesky status is not checked)."""
    w = water_small
    rng = np.random.default_rng(5)
    n = w.norb
    cand = [(i, j) for i in range(n) for j in range(i + 1, n)]
    pick = rng.choice(len(cand), size=len(cand) // 3, replace=False)
    pairs = np.array([cand[k] for k in sorted(pick)], dtype=np.int32)
    p = _pairs_build(w, prec, pairs)
    assert p["op"] is not None
    mask = mask_from_pairs(pairs, n)
    W_ref = oracle.exchange_w(w.phi, w.lattice, mask=mask)
    r = oracle.ace_from_w(w.phi, W_ref, w.dV, want_xi=False)
    rtol = FP64_ARRAY_RTOL if prec == ace.ACE_FP64 else MIXED_W_RTOL
    assert rel_max(p["W"].reshape(W_ref.shape), W_ref) <= rtol
    assert np.abs(p["M_raw"] - r["M_raw"]).max() <= (1e-10 if prec == ace.ACE_FP64 else 2e-5) * np.abs(r["M_raw"]).max()


@pytest.mark.parametrize("host", [False, True])
def test_reuse_across_snapshots(host):
    """Snapshot 1 (every centre moved 0.05 bohr) built on snapshot 0's screened pair list."""
    snaps = enzyme_like(np.random.default_rng(1051), ncentres=16, cell=(16.0, 16.0, 16.0), grid=(48, 48, 48),
                        radius=3.5, dmin=2.0, nsnap=2)
    g0 = gpu_build(snaps[0].phi, snaps[0].lattice, ace.ACE_FP64, rho_cut=snaps[0].rho_cut)
    w1 = snaps[1]
    p = _pairs_build(w1, ace.ACE_FP64, g0["pairs"], host=host)
    assert p["status"] == 0
    ref = oracle.ace_build(w1.phi, w1.lattice, mask=mask_from_pairs(g0["pairs"], w1.norb), spin_factor=w1.spin_factor)
    assert abs(p["E_x"] - ref["E_x"]) <= FP64_EX_TOL
    assert rel_max(p["W"].reshape(ref["W"].shape), ref["W"]) <= FP64_ARRAY_RTOL


def test_pair_list_errors(water_small):
    import torch

    w = water_small
    x = torch.from_numpy(w.phi.astype(np.float32)).cuda()
    d = ace.make_desc(w.grid, w.lattice, w.norb)
    for bad in ([[0, w.norb]], [[-1, 0]], [[0, 1], [1, 0]]):
        with pytest.raises(ace.AceError) as e:
            ace.ace_build_pairs(d, x, np.array(bad))
        assert e.value.status == ace.ace.ACE_ERR_ARG
