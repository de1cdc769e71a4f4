"""ace_build_batched: uneven builds (orbital counts, grids, screening, precision) on one stream lane
(the default) and on four concurrent lanes, with the steps after the pair chain on a tail stream (the
default) or on the lane, each checked against the FP64 oracle and against its single-build result."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from gpu_helpers import FP64_ARRAY_RTOL, FP64_EX_TOL, MIXED_EX_TOL_PER_ORB, MIXED_W_RTOL, mask_from_pairs, rel_max
from paper_2101_03155_gb300 import ace as abi
from workloads.generators import gaussian_orbitals, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    abi.load()
    oracle.build()


def _inputs():
    rng = np.random.default_rng(4004)
    cases = []
    for grid, cell, n in (((16, 16, 16), 8.0, 6), ((24, 24, 24), 10.0, 10), ((32, 32, 32), 12.0, 16),
                          ((20, 12, 24), 9.0, 8)):
        lat = np.diag([cell, cell * grid[1] / grid[0], cell * grid[2] / grid[0]])
        phi, _, _ = gaussian_orbitals(grid, lat, n, 2, rng)
        cases.append((phi, lat, 0.0))
    w = water_like(8, 11.74, (48, 48, 48), rng, rho_cut=1e-3, dmin=4.0)
    cases.append((w.phi, w.lattice, w.rho_cut))
    return cases


@pytest.mark.parametrize("lanes,tail", [("1", "1"), ("1", "0"), ("4", "1")])
@pytest.mark.parametrize("prec", [ace.ACE_FP64, ace.ACE_MIXED])
def test_batched_uneven_builds(prec, lanes, tail, monkeypatch):
    """tail = 1 (the default): each build's M, Cholesky and xi on the lane's tail stream beside the next
    build's chain; tail = 0: all of a build on its lane."""
    import torch

    monkeypatch.setenv("ACE_BATCH_LANES", lanes)
    monkeypatch.setenv("ACE_BATCH_TAIL", tail)

    cases = _inputs()
    dt = torch.float64 if prec == ace.ACE_FP64 else torch.float32
    descs = [ace.make_desc(p.shape[1:], lat, p.shape[0], rho_cut=rc, prec=prec) for p, lat, rc in cases]
    phis = [torch.from_numpy(p).to(device="cuda", dtype=dt) for p, _, _ in cases]
    ops = ace.ace_build_batched(descs, phis, torch.cuda.current_stream())
    assert len(ops) == len(cases)
    for (phi, lat, rc), op in zip(cases, ops):
        n = phi.shape[0]
        pairs = abi.get_numpy(op, abi.ACE_GET_PAIRS)
        mask = mask_from_pairs(pairs, n)
        ref = oracle.ace_build(phi, lat, spin_factor=2.0, mask=mask)
        W = abi.get_numpy(op, abi.ACE_GET_W).reshape(phi.shape)
        e = ace.exchange_energy(op)
        if prec == ace.ACE_FP64:
            assert abs(e - ref["E_x"]) <= FP64_EX_TOL
            assert rel_max(W, ref["W"]) <= FP64_ARRAY_RTOL
        else:
            assert abs(e - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * n
            assert rel_max(W, ref["W"]) <= MIXED_W_RTOL
        # the same input through the single-build entry point gives the same operator
        single = ace.ace_build(ace.make_desc(phi.shape[1:], lat, n, rho_cut=rc, prec=prec),
                               phis[ops.index(op)], torch.cuda.current_stream())
        assert abi.ace_pair_count(single) == abi.ace_pair_count(op)
        tol = 1e-12 if prec == ace.ACE_FP64 else 1e-6
        assert abs(ace.exchange_energy(single) - e) <= tol * abs(e)
        xi_b = abi.get_numpy(op, abi.ACE_GET_XI)
        xi_s = abi.get_numpy(single, abi.ACE_GET_XI)
        if prec == ace.ACE_FP64:
            assert np.array_equal(xi_b, xi_s)  # the FP64 form repeats bit for bit
        else:
            assert rel_max(xi_b, xi_s) <= MIXED_W_RTOL
        single.close()
    for op in ops:
        op.close()


def test_batched_reports_the_failing_build():
    import torch

    rng = np.random.default_rng(3)
    lat = np.diag([8.0, 8.0, 8.0])
    good, _, _ = gaussian_orbitals((16, 16, 16), lat, 3, 1, rng)
    bad = np.concatenate([good, np.zeros_like(good[:1])])
    descs = [ace.make_desc((16, 16, 16), lat, 3, prec=ace.ACE_FP64),
             ace.make_desc((16, 16, 16), lat, 4, prec=ace.ACE_FP64)]
    phis = [torch.from_numpy(good).cuda(), torch.from_numpy(bad).cuda()]
    with pytest.raises(ace.AceError) as e:
        ace.ace_build_batched(descs, phis, torch.cuda.current_stream())
    assert e.value.status == abi.ACE_ERR_NOT_POSDEF
    assert "build 1 of 2" in str(e.value)
