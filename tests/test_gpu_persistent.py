"""The persistent pair chain (ACE_PERSISTENT=1): one launch walks the whole screened pack list
through a device-side task queue (forward planes, pencils, inverse planes with the W
accumulation of Eq. vx).  Parity with the FP64 oracle and with the default stream-batched chain,
through the C ABI."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from gpu_helpers import MIXED_EX_TOL_PER_ORB, MIXED_W_RTOL, gpu_build, rel_max
from workloads.generators import config1, config4, gaussian_orbitals, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()
    oracle.build()


@pytest.fixture
def persistent(monkeypatch):
    monkeypatch.setenv("ACE_PERSISTENT", "1")
    yield
    monkeypatch.delenv("ACE_PERSISTENT")


def test_persistent_config1(persistent):
    """16 orbitals on 32^3, all pairs (68 packs, fewer than the queue's slots x rounds)."""
    w = config1()
    ref = oracle.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)
    g = gpu_build(w.phi, w.lattice, ace.ACE_MIXED)
    assert g["status"] == 0
    assert rel_max(g["W"].reshape(ref["W"].shape), ref["W"]) <= MIXED_W_RTOL
    assert abs(g["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * w.norb


@pytest.mark.parametrize("n1", [72, 108])
def test_persistent_plane_shapes(persistent, n1):
    lat = np.diag([11.0, 11.5, 12.0])
    phi, _, _ = gaussian_orbitals((n1,) * 3, lat, 4, 2, np.random.default_rng(n1))
    ref = oracle.ace_build(phi, lat, 0.0, 2.0)
    g = gpu_build(phi, lat, ace.ACE_MIXED)
    assert g["status"] == 0
    assert rel_max(g["W"].reshape(ref["W"].shape), ref["W"]) <= MIXED_W_RTOL
    assert abs(g["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * 4


def test_persistent_screened_matches_batched_chain(monkeypatch):
    """A screened 32-orbital build on 48^3: the persistent chain and the stream-batched chain give
    the same W (up to FP32 atomic order) and the oracle's W on the same pair list."""
    w = water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)
    d = gpu_build(w.phi, w.lattice, ace.ACE_MIXED, rho_cut=w.rho_cut)
    monkeypatch.setenv("ACE_PERSISTENT", "1")
    p = gpu_build(w.phi, w.lattice, ace.ACE_MIXED, rho_cut=w.rho_cut)
    monkeypatch.delenv("ACE_PERSISTENT")
    assert p["status"] == 0 and np.array_equal(p["pairs"], d["pairs"])
    assert rel_max(p["W"], d["W"]) <= MIXED_W_RTOL
    ref = oracle.ace_build(w.phi, w.lattice, mask=p["mask"], spin_factor=w.spin_factor)
    assert rel_max(p["W"].reshape(ref["W"].shape), ref["W"]) <= MIXED_W_RTOL
    assert abs(p["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * w.norb


def test_persistent_batched_uneven(persistent):
    """Two uneven builds of the batched set (64 orbitals on 72^3 and 128^3) in one batched call."""
    import torch

    ws = config4(builds=[1, 12])
    descs = [ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=2.0, prec=ace.ACE_MIXED)
             for w in ws]
    phis = [torch.from_numpy(w.phi.astype(np.float32)).cuda() for w in ws]
    ops = ace.ace_build_batched(descs, phis, torch.cuda.current_stream())
    for w, op in zip(ws, ops):
        pairs = ace.ace.get_numpy(op, ace.ace.ACE_GET_PAIRS)
        mask = np.zeros((w.norb, w.norb), bool)
        mask[pairs[:, 0], pairs[:, 1]] = mask[pairs[:, 1], pairs[:, 0]] = True
        rows = [0, w.norb - 1]
        W = ace.ace.get_numpy(op, ace.ace.ACE_GET_W).reshape((w.norb,) + w.grid)
        Wref = oracle.exchange_w(w.phi, w.lattice, mask=mask, rows=rows)
        for k, i in enumerate(rows):
            assert rel_max(W[i], Wref[k]) <= MIXED_W_RTOL
        op.close()
