"""The per-rank entry points of one build over several GPUs (ace_exchange_w, ace_m_partial,
ace_build_from_m, ace_apply_coeffs, ace_apply_finish), through the C ABI on one GPU.

Two ranks are emulated one after the other in this process: each rank's calls run to completion
before the next, and the collectives (sums of the ranks' W, M and C) are done here between the
steps; no kernel waits for another.  The result must equal the one-GPU build on the same pair list
(FP64: to 1e-10; mixed: within the mixed form's tolerances against the FP64 oracle)."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from paper_2101_03155_gb300 import ace as abi
from paper_2101_03155_gb300.sharding import GpuSlabKernels, point_slabs, shard_pairs, sharded_apply, sharded_build
from gpu_helpers import (FP64_ARRAY_RTOL, FP64_EX_TOL, MIXED_EX_TOL_PER_ORB, MIXED_KPSI_RTOL, MIXED_XI_RTOL,
                         mask_from_pairs, rel_max)
from workloads.generators import probe_vectors, water_like

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
def case():
    w = water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)
    _, mask = oracle.screen(w.phi, w.lattice, w.rho_cut)
    iu = np.triu_indices(w.norb)
    pairs = np.stack([iu[0][mask[iu]], iu[1][mask[iu]]], axis=1).astype(np.int32)
    ref = oracle.ace_build(w.phi, w.lattice, mask=mask, spin_factor=w.spin_factor)
    return w, pairs, ref


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_two_emulated_ranks_equal_the_one_gpu_build(case, prec):
    import torch

    w, pairs, ref = case
    dt = torch.float64 if prec == ace.ACE_FP64 else torch.float32
    desc = ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=w.spin_factor, prec=prec)
    k = GpuSlabKernels(desc, torch.cuda.current_stream())
    phi = torch.from_numpy(w.phi).to(device="cuda", dtype=dt).reshape(w.norb, -1)
    R = 2
    slabs = point_slabs(w.npts, R)
    # step 1 per rank, then the reduce-scatter (here: a sum and slicing)
    W = sum(k.exchange_w(phi, part) for part in shard_pairs(pairs, R))
    W_ref = ref["W"].reshape(w.norb, -1)
    tol_w = FP64_ARRAY_RTOL if prec == ace.ACE_FP64 else 2e-5
    assert rel_max(W.cpu().numpy(), W_ref) <= tol_w
    W_slabs = [W[:, p0:p1].contiguous() for p0, p1 in slabs]
    # step 3 per rank, the all-reduce of M, step 5 per rank
    M = sum(k.m_partial(phi[:, p0:p1], Ws) for (p0, p1), Ws in zip(slabs, W_slabs))
    assert np.abs(M.cpu().numpy() - ref["M_raw"]).max() <= (1e-10 if prec == ace.ACE_FP64 else 2e-5) * np.abs(
        ref["M"]).max()
    ops = [k.build_from_m(M, Ws) for Ws in W_slabs]
    xi_ref = ref["xi"].reshape(w.norb, -1)
    for (p0, p1), op in zip(slabs, ops):
        xi = abi.get_numpy(op, abi.ACE_GET_XI).astype(np.float64)
        if prec == ace.ACE_FP64:
            assert rel_max(xi, xi_ref[:, p0:p1]) <= FP64_ARRAY_RTOL
            assert abs(ace.exchange_energy(op) - ref["E_x"]) <= FP64_EX_TOL
        else:
            assert _rel(xi, xi_ref[:, p0:p1]) <= MIXED_XI_RTOL
            assert abs(ace.exchange_energy(op) - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * w.norb
    # the application: coefficients per rank, all-reduce, finish per rank
    psi = probe_vectors(w.phi, w.dV, 8).reshape(2, -1)
    psi_t = torch.from_numpy(psi).to(device="cuda", dtype=dt)
    C = sum(k.apply_coeffs(op, psi_t[:, p0:p1]) for (p0, p1), op in zip(slabs, ops))
    kref = oracle.ace_apply(ref["xi"], psi.reshape((2,) + w.grid), w.dV).reshape(2, -1)
    for (p0, p1), op in zip(slabs, ops):
        out = k.apply_finish(op, C, 2).double().cpu().numpy()
        if prec == ace.ACE_FP64:
            assert rel_max(out, kref[:, p0:p1]) <= FP64_ARRAY_RTOL
        else:
            assert _rel(out, kref[:, p0:p1]) <= MIXED_KPSI_RTOL
        op.close()


class _OneRank:
    rank, world = 0, 1

    def reduce_scatter_slabs(self, W, slabs):
        return W[:, slabs[0][0]:slabs[0][1]].contiguous()

    def all_reduce(self, t):
        return t


def test_sharded_driver_on_one_rank_equals_ace_build_pairs(case):
    """The per-rank driver with a world of one rank: the same operator as ace_build_pairs."""
    import torch

    w, pairs, ref = case
    desc = ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=w.spin_factor, prec=ace.ACE_FP64)
    stream = torch.cuda.current_stream()
    kern = GpuSlabKernels(desc, stream)
    phi = torch.from_numpy(w.phi).cuda()
    op, (p0, p1) = sharded_build(kern, _OneRank(), phi, pairs)
    assert (p0, p1) == (0, w.npts)
    full = ace.ace_build_pairs(desc, phi, pairs, stream)
    assert abs(ace.exchange_energy(op) - ace.exchange_energy(full)) <= 1e-12
    xi = abi.get_numpy(op, abi.ACE_GET_XI)
    assert rel_max(xi, abi.get_numpy(full, abi.ACE_GET_XI)) <= 1e-12
    psi = torch.from_numpy(probe_vectors(w.phi, w.dV, 9).reshape(2, -1)).cuda()
    out = sharded_apply(kern, _OneRank(), op, psi).cpu().numpy()
    out_full = torch.empty_like(psi)
    ace.ace_apply(full, psi, out_full, stream)
    assert rel_max(out, out_full.cpu().numpy()) <= 1e-12
    op.close()
    full.close()


def test_slab_entry_points_refuse_bad_arguments(case):
    import torch

    w, pairs, _ = case
    desc = ace.make_desc(w.grid, w.lattice, w.norb, prec=ace.ACE_MIXED)
    phi64 = torch.from_numpy(w.phi).cuda().reshape(w.norb, -1)
    M = torch.empty((w.norb, w.norb), dtype=torch.float64, device="cuda")
    with pytest.raises(ace.AceError) as e:  # FP64 slabs for the mixed form
        ace.ace.ace_m_partial(desc, phi64[:, :128].contiguous(), phi64[:, :128].contiguous(), M)
    assert e.value.status == abi.ACE_ERR_ARG
    with pytest.raises(ace.AceError) as e:
        ace.ace.ace_exchange_w(desc, phi64, np.array([[0, w.norb]], np.int32),
                               torch.empty_like(phi64, dtype=torch.float32))
    assert e.value.status == abi.ACE_ERR_ARG
