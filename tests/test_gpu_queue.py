"""Device pack queues: screened builds whose pair chains run as one persistent launch per grid over
the concatenated, build-tagged pack lists that the screen's compaction wrote, with no host wait
between screen and chain (ace_build_batched with ACE_BATCH_QUEUE=1; ace_graph_create without pair
lists).  Uneven builds, several on one grid with different cells (so different Coulomb tables in
one launch), each against the FP64 oracle on its own pair mask and against ace_build."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from gpu_helpers import MIXED_EX_TOL_PER_ORB, MIXED_W_RTOL, mask_from_pairs, rel_max
from paper_2101_03155_gb300 import ace as abi
from workloads.generators import config1, gaussian_orbitals, moved_snapshot, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    abi.load()
    oracle.build()


def _cases():
    """(workload-like tuple phi, lattice, rho_cut), grids interleaved: three builds on 32^3 with
    different cells and orbital counts, one screened 32-orbital build on 48^3, one on 72^3."""
    rng = np.random.default_rng(6006)
    out = []
    c1 = config1()
    out.append((c1.phi, c1.lattice, 0.0))
    w = water_like(8, 11.74, (48, 48, 48), rng, rho_cut=1e-3, dmin=4.0)
    out.append((w.phi, w.lattice, w.rho_cut))
    lat = np.diag([12.0, 12.5, 13.0])
    phi, _, _ = gaussian_orbitals((32, 32, 32), lat, 10, 2, rng)
    out.append((phi, lat, 1e-3))
    lat = np.diag([11.0, 11.0, 11.0])
    phi, _, _ = gaussian_orbitals((72, 72, 72), lat, 6, 2, rng)
    out.append((phi, lat, 0.0))
    lat = np.diag([9.0, 9.0, 9.0])
    phi, _, _ = gaussian_orbitals((32, 32, 32), lat, 7, 2, rng)
    out.append((phi, lat, 1e-2))
    return out, w


@pytest.fixture(scope="module")
def cases():
    return _cases()


def _descs(cases):
    return [ace.make_desc(p.shape[1:], lat, p.shape[0], rho_cut=rc, prec=ace.ACE_MIXED) for p, lat, rc in cases]


def _check_against_oracle(cases, ops):
    import torch

    for (phi, lat, rc), op in zip(cases, ops):
        n = phi.shape[0]
        pairs = abi.get_numpy(op, abi.ACE_GET_PAIRS)
        single = ace.ace_build(ace.make_desc(phi.shape[1:], lat, n, rho_cut=rc, prec=ace.ACE_MIXED),
                               torch.from_numpy(phi.astype(np.float32)).cuda(), torch.cuda.current_stream())
        assert np.array_equal(pairs, abi.get_numpy(single, abi.ACE_GET_PAIRS))
        assert abs(ace.exchange_energy(single) - ace.exchange_energy(op)) <= 0.1 * MIXED_EX_TOL_PER_ORB * n
        single.close()
        ref = oracle.ace_build(phi, lat, spin_factor=2.0, mask=mask_from_pairs(pairs, n), want_xi=False)
        W = abi.get_numpy(op, abi.ACE_GET_W).reshape(phi.shape)
        assert rel_max(W, ref["W"]) <= MIXED_W_RTOL
        assert abs(ace.exchange_energy(op) - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * n


def test_batched_queue_uneven_builds(cases, monkeypatch):
    import torch

    monkeypatch.setenv("ACE_BATCH_QUEUE", "1")
    cs, _ = cases
    phis = [torch.from_numpy(p.astype(np.float32)).cuda() for p, _, _ in cs]
    ops = ace.ace_build_batched(_descs(cs), phis, torch.cuda.current_stream())
    try:
        _check_against_oracle(cs, ops)
    finally:
        for op in ops:
            op.close()


def test_batched_queue_host_inputs(cases, monkeypatch):
    """Host FP64 inputs: staged and converted on the device before the screens, same operators."""
    import torch

    monkeypatch.setenv("ACE_BATCH_QUEUE", "1")
    cs, _ = cases
    ops = ace.ace_build_batched(_descs(cs[:3]), [np.ascontiguousarray(p) for p, _, _ in cs[:3]],
                                torch.cuda.current_stream())
    try:
        _check_against_oracle(cs[:3], ops)
    finally:
        for op in ops:
            op.close()


def test_screened_graph_replays(cases):
    """Five screened builds in one graph: a launch matches the oracle on each build's own list;
    after a build's input moves to the next snapshot the replay screens it again (its list and E_x
    are ace_build's on the new contents) while the others repeat."""
    import torch

    cs, w = cases
    stream = torch.cuda.current_stream()
    phis = [torch.from_numpy(p.astype(np.float32)).cuda() for p, _, _ in cs]
    with ace.ace_graph_create(_descs(cs), phis, None, stream) as g:
        g.launch(stream)
        g.sync()
        _check_against_oracle(cs, g.ops)
        e_before = [ace.exchange_energy(op) for op in g.ops]
        w1 = moved_snapshot(w, 0.3, np.random.default_rng(7))
        phis[1].copy_(torch.from_numpy(w1.phi.astype(np.float32)))
        g.launch(stream)
        g.sync()
        moved = list(cs)
        moved[1] = (w1.phi, w1.lattice, w1.rho_cut)
        _check_against_oracle(moved, g.ops)
        for i in (0, 2, 3, 4):
            assert abs(ace.exchange_energy(g.ops[i]) - e_before[i]) <= 0.1 * MIXED_EX_TOL_PER_ORB * cs[i][0].shape[0]
        assert ace.exchange_energy(g.ops[1]) != e_before[1]


def test_screened_graph_argument_checks(cases):
    import torch

    cs, _ = cases
    stream = torch.cuda.current_stream()
    phi, lat, rc = cs[0]
    d64 = ace.make_desc(phi.shape[1:], lat, phi.shape[0], rho_cut=rc, prec=ace.ACE_FP64)
    with pytest.raises(ace.AceError) as e:
        ace.ace_graph_create([d64], [torch.from_numpy(phi).cuda()], None, stream)
    assert e.value.status == abi.ACE_ERR_ARG
    lat = np.diag([8.0, 8.0, 8.0])
    p16, _, _ = gaussian_orbitals((16, 16, 16), lat, 3, 1, np.random.default_rng(1))
    d16 = ace.make_desc((16, 16, 16), lat, 3, prec=ace.ACE_MIXED)
    with pytest.raises(ace.AceError) as e:
        ace.ace_graph_create([d16], [torch.from_numpy(p16.astype(np.float32)).cuda()], None, stream)
    assert e.value.status == abi.ACE_ERR_UNSUPPORTED_GRID


def test_queue_give_up_marks_every_build(cases, monkeypatch):
    """A queue wait that gives up (pencil tasks waiting on a word nothing sets, 1 ms limit) reports
    ACE_ERR_TIMEOUT for the batch; the next batch in the process matches the oracle."""
    import torch

    cs, _ = cases
    monkeypatch.setenv("ACE_BATCH_QUEUE", "1")
    phis = [torch.from_numpy(p.astype(np.float32)).cuda() for p, _, _ in cs[:3]]
    monkeypatch.setenv("ACE_PERSIST_TEST_STALL", "1")
    monkeypatch.setenv("ACE_PERSIST_WAIT_NS", "1000000")
    with pytest.raises(ace.AceError) as e:
        ace.ace_build_batched(_descs(cs[:3]), phis, torch.cuda.current_stream())
    assert e.value.status == abi.ACE_ERR_TIMEOUT
    monkeypatch.delenv("ACE_PERSIST_TEST_STALL")
    monkeypatch.delenv("ACE_PERSIST_WAIT_NS")
    ops = ace.ace_build_batched(_descs(cs[:3]), phis, torch.cuda.current_stream())
    try:
        _check_against_oracle(cs[:3], ops)
    finally:
        for op in ops:
            op.close()
