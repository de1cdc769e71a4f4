"""Failure and repeatability behaviour of the GPU path, through the C ABI.

Give-up paths: every wait inside a kernel is bounded.  Host-side test knobs make one wait run out
on purpose -- the first wait of the tensor-core Gram for its TMA box (given zero polls), or the
persistent chain's pencil tasks waiting for a word that nothing sets (with a 1 ms limit) -- and the
call must report ACE_ERR_TIMEOUT, leave the context usable, and the next build must succeed.
No GPU fault, trap or hang is involved: the kernels drain their own copies and return.

Repeatability: the FP64 form adds every W element's terms in one fixed order (rounds of packs on
disjoint orbitals) and sums the Gram chunks in a fixed order, so two FP64 builds agree bit for bit.
"""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from paper_2101_03155_gb300 import ace as abi
from gpu_helpers import FP64_EX_TOL, MIXED_EX_TOL_PER_ORB, gpu_build
from workloads.generators import config1, gaussian_orbitals, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()
    oracle.build()


@pytest.fixture(scope="module")
def cfg1():
    w = config1()
    return w, oracle.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)


def test_tensor_core_wait_gives_up_then_next_build_succeeds(cfg1, monkeypatch):
    w, ref = cfg1
    monkeypatch.setenv("ACE_TC_FIRST_WAIT_POLLS", "0")
    g = gpu_build(w.phi, w.lattice, ace.ACE_MIXED)
    monkeypatch.delenv("ACE_TC_FIRST_WAIT_POLLS")
    assert g["status"] == abi.ACE_ERR_TIMEOUT
    assert "gave up waiting" in ace.ace_last_error()
    if g["op"] is not None:
        g["op"].close()
    ok = gpu_build(w.phi, w.lattice, ace.ACE_MIXED)
    assert ok["status"] == 0
    assert abs(ok["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * w.norb


def test_persistent_chain_wait_gives_up_then_next_build_succeeds(cfg1, monkeypatch):
    w, ref = cfg1
    monkeypatch.setenv("ACE_PERSISTENT", "1")
    monkeypatch.setenv("ACE_PERSIST_TEST_STALL", "1")
    monkeypatch.setenv("ACE_PERSIST_WAIT_NS", "1000000")
    g = gpu_build(w.phi, w.lattice, ace.ACE_MIXED)
    monkeypatch.delenv("ACE_PERSIST_TEST_STALL")
    monkeypatch.delenv("ACE_PERSIST_WAIT_NS")
    assert g["status"] == abi.ACE_ERR_TIMEOUT
    if g["op"] is not None:
        g["op"].close()
    ok = gpu_build(w.phi, w.lattice, ace.ACE_MIXED)
    monkeypatch.delenv("ACE_PERSISTENT")
    assert ok["status"] == 0
    assert abs(ok["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * w.norb


def _same(a, b):
    for key in ("W", "xi", "M_raw", "M", "L", "O", "pairs"):
        assert np.array_equal(a[key], b[key]), key
    assert a["E_x"] == b["E_x"]


# (20, 12, 24): the plane passes (24-point rows); (12, 20, 8): the five pencil passes
@pytest.mark.parametrize("grid", [(20, 12, 24), (12, 20, 8)])
def test_fp64_build_repeats_bit_for_bit(grid):
    lat = np.diag([8.0, 8.5, 9.0])
    phi, _, _ = gaussian_orbitals(grid, lat, 7, 2, np.random.default_rng(sum(grid)))
    a = gpu_build(phi, lat, ace.ACE_FP64)
    b = gpu_build(phi, lat, ace.ACE_FP64)
    assert a["status"] == 0 and b["status"] == 0
    _same(a, b)
    ref = oracle.ace_build(phi, lat, 0.0, 2.0)
    assert abs(a["E_x"] - ref["E_x"]) <= FP64_EX_TOL


def test_fp64_screened_build_and_apply_repeat_bit_for_bit():
    import torch

    w = water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)
    a = gpu_build(w.phi, w.lattice, ace.ACE_FP64, rho_cut=w.rho_cut)
    b = gpu_build(w.phi, w.lattice, ace.ACE_FP64, rho_cut=w.rho_cut)
    assert a["status"] == 0 and b["status"] == 0
    _same(a, b)
    psi = torch.from_numpy(np.random.default_rng(3).standard_normal((5,) + w.grid)).cuda()
    outs = []
    for g in (a, b):
        out = torch.empty_like(psi)
        ace.ace_apply(g["op"], psi, out)
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
