"""ace_exchange_w_noalloc: W for an explicit pair list with no device allocation inside the call.

Callers that may not allocate device memory while they run (fixed memory budgets, allocation-free
inner loops, frameworks that own all device memory) use this entry point; it takes its workspace
from a fixed array compiled into the library.  These tests check, through the C ABI, that its W
equals the W of ace_build (the allocating path) on the same pair list, within the tolerances the
other parity tests use, for two calls in a row (the shared array keeps the previous call's
contents, and the output is filled with garbage before each call), and that grids too large for
the array are refused.  This file is collected last so that a failure here does not hide others.
"""

import numpy as np
import pytest

import paper_2101_03155_gb300 as ace
from gpu_helpers import FP64_ARRAY_RTOL, MIXED_W_RTOL, gpu_build, rel_max
from workloads.generators import config1, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()


def _cases():
    w1 = config1()
    w2 = water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)
    return [(w1, 0.0), (w2, w2.rho_cut)]


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_noalloc_matches_build_on_consecutive_calls(prec):
    import torch

    dtype = torch.float64 if prec == ace.ACE_FP64 else torch.float32
    tol = FP64_ARRAY_RTOL if prec == ace.ACE_FP64 else MIXED_W_RTOL
    stream = torch.cuda.current_stream()
    refs = []
    for w, rho_cut in _cases():
        g = gpu_build(w.phi, w.lattice, prec, rho_cut=rho_cut)
        assert g["status"] == 0
        refs.append((w, rho_cut, g["W"].reshape(w.phi.shape), g["pairs"]))
        g["op"].close()
    # two calls in a row on the same input, then a call on a different grid and pair list
    for w, rho_cut, W_ref, pairs in (refs[0], refs[0], refs[1], refs[1]):
        desc = ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=rho_cut, spin_factor=w.spin_factor, prec=prec)
        phi = torch.from_numpy(w.phi).to(device="cuda", dtype=dtype)
        W = torch.full_like(phi, float("nan"))
        ace.ace.ace_exchange_w_noalloc(desc, phi, pairs, W, stream)
        torch.cuda.synchronize()
        assert rel_max(W.cpu().numpy(), W_ref) <= tol


def test_noalloc_refuses_grids_beyond_its_array():
    import torch

    lat = np.eye(3) * 20.0
    desc = ace.make_desc((128, 128, 128), lat, 2, prec=ace.ACE_FP64)  # 3 * 8 B * 128^3 > 32 MiB
    tiny = torch.zeros(16, dtype=torch.float64, device="cuda")  # refused before any access
    with pytest.raises(ace.AceError) as e:
        ace.ace.ace_exchange_w_noalloc(desc, tiny, np.array([[0, 0]], np.int32), tiny)
    assert e.value.status == ace.ace.ACE_ERR_ARG
    assert "fixed array" in str(e.value)


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_noalloc_truncated_kernel(prec):
    """The isolated-cell kernel table built on the device matches ace_build's host-built table."""
    import torch

    from workloads.generators import enzyme_like

    w = enzyme_like(np.random.default_rng(1050), ncentres=16, cell=(16.0, 16.0, 16.0), grid=(48, 48, 48),
                    radius=3.5, dmin=2.0, nsnap=1)[0]
    dtype = torch.float64 if prec == ace.ACE_FP64 else torch.float32
    tol = FP64_ARRAY_RTOL if prec == ace.ACE_FP64 else MIXED_W_RTOL
    for rc in (0.0, 6.5):
        g = gpu_build(w.phi, w.lattice, prec, rho_cut=w.rho_cut, coulomb=ace.ACE_COULOMB_TRUNCATED, r_cut=rc)
        assert g["status"] == 0
        desc = ace.make_desc(w.grid, w.lattice, w.norb, prec=prec, coulomb=ace.ACE_COULOMB_TRUNCATED, r_cut=rc)
        phi = torch.from_numpy(w.phi).to(device="cuda", dtype=dtype)
        W = torch.full_like(phi, float("nan"))
        ace.ace.ace_exchange_w_noalloc(desc, phi, g["pairs"], W, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert rel_max(W.cpu().numpy(), g["W"].reshape(w.phi.shape)) <= tol
        g["op"].close()


def test_noalloc_refuses_unaligned_buffers():
    import torch

    lat = np.eye(3) * 8.0
    desc = ace.make_desc((16, 16, 16), lat, 1, prec=ace.ACE_MIXED)
    big = torch.zeros(2 * 4096 + 1, dtype=torch.float32, device="cuda")
    phi, W = big[1:4097], big[4097:]  # 4 bytes past a 16-byte boundary: refused before any access
    with pytest.raises(ace.AceError) as e:
        ace.ace.ace_exchange_w_noalloc(desc, phi, np.array([[0, 0]], np.int32), W)
    assert e.value.status == ace.ace.ACE_ERR_ARG
    assert "aligned" in str(e.value)


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_noalloc_pair_list_beyond_one_pack_chunk(prec):
    """130 orbitals, every pair (8,515 pairs, an odd count: 4,258 packs, more than one upload chunk
    of the fixed array's pack list, the last pack holding a single pair): the same W as the
    allocating per-rank entry point ace_exchange_w on the same list, on two calls in a row."""
    import torch

    from workloads.generators import gaussian_orbitals

    grid, lat = (16, 16, 16), np.diag([9.0, 9.5, 10.0])
    phi_h, _, _ = gaussian_orbitals(grid, lat, 130, 1, np.random.default_rng(77))
    iu = np.triu_indices(130)
    pairs = np.stack(iu, axis=1).astype(np.int32)
    assert len(pairs) == 8515
    dtype = torch.float64 if prec == ace.ACE_FP64 else torch.float32
    tol = FP64_ARRAY_RTOL if prec == ace.ACE_FP64 else MIXED_W_RTOL
    desc = ace.make_desc(grid, lat, 130, prec=prec)
    phi = torch.from_numpy(phi_h).to(device="cuda", dtype=dtype)
    stream = torch.cuda.current_stream()
    W_ref = torch.empty_like(phi)
    ace.ace.ace_exchange_w(desc, phi, pairs, W_ref, stream)
    for _ in range(2):
        W = torch.full_like(phi, float("nan"))
        ace.ace.ace_exchange_w_noalloc(desc, phi, pairs, W, stream)
        torch.cuda.synchronize()
        assert rel_max(W.cpu().numpy(), W_ref.cpu().numpy()) <= tol


@pytest.mark.parametrize("coulomb", [ace.ACE_COULOMB_PERIODIC, ace.ACE_COULOMB_TRUNCATED])
def test_noalloc_triclinic_cell(coulomb):
    """A triclinic cell: the device-built reciprocal basis and kernel table of the no-alloc path
    against ace_build's host-built ones (FP64, both kernels)."""
    import torch

    from workloads.generators import gaussian_orbitals

    lat = np.array([[7.5, 0.0, 0.0], [1.2, 7.0, 0.0], [0.6, -0.9, 6.8]])
    grid = (12, 16, 20)
    phi_h, _, _ = gaussian_orbitals(grid, lat, 4, 2, np.random.default_rng(5))
    g = gpu_build(phi_h, lat, ace.ACE_FP64, coulomb=coulomb)
    assert g["status"] == 0
    desc = ace.make_desc(grid, lat, 4, prec=ace.ACE_FP64, coulomb=coulomb)
    phi = torch.from_numpy(phi_h).cuda()
    W = torch.full_like(phi, float("nan"))
    ace.ace.ace_exchange_w_noalloc(desc, phi, g["pairs"], W, torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert rel_max(W.cpu().numpy(), g["W"].reshape(phi_h.shape)) <= FP64_ARRAY_RTOL
    g["op"].close()
