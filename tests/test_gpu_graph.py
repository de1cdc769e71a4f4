"""ace_graph_*: k builds on given pair lists recorded once as a CUDA graph and replayed (the reuse
steps of a multiple-time-step run, section III).  Each replay must give what ace_build_pairs gives
on the orbitals the inputs hold at launch time: bit for bit in FP64 (the FP64 chain is
deterministic), within the mixed-form tolerances otherwise, and the oracle's W and E_x on the same
pair mask.  Through the C ABI."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from paper_2101_03155_gb300 import ace as abi
from gpu_helpers import MIXED_EX_TOL_PER_ORB, MIXED_W_RTOL, mask_from_pairs, rel_max
from workloads.generators import config1, moved_snapshot, water_like

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    abi.load()
    oracle.build()


def _snapshots(seed):
    """Two snapshots of a screened 32-orbital system on 48^3 (centres moved by ~0.05 bohr) and the
    pair list of the first, plus the 16-orbital 32^3 case with all pairs."""
    rng = np.random.default_rng(seed)
    w0 = water_like(8, 11.74, (48, 48, 48), rng, rho_cut=1e-3, dmin=4.0)
    w1 = moved_snapshot(w0, 0.05, rng)
    _, mask = oracle.screen(w0.phi, w0.lattice, w0.rho_cut)
    pairs0 = np.argwhere(np.triu(mask)).astype(np.int32)
    c1 = config1()
    n = c1.norb
    all_pairs = np.array([(i, j) for i in range(n) for j in range(i, n)], dtype=np.int32)
    return w0, w1, pairs0, c1, all_pairs


@pytest.fixture(scope="module")
def systems():
    return _snapshots(1010)


def _desc(w, prec):
    return ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, spin_factor=w.spin_factor, prec=prec)


def _direct(w, prec, pairs, phi_np):
    import torch

    dt = np.float64 if prec == ace.ACE_FP64 else np.float32
    phi = torch.from_numpy(np.ascontiguousarray(phi_np, dtype=dt)).cuda()
    op = ace.ace_build_pairs(_desc(w, prec), phi, pairs, torch.cuda.current_stream())
    out = {"E_x": ace.exchange_energy(op), "xi": abi.get_numpy(op, abi.ACE_GET_XI),
           "W": abi.get_numpy(op, abi.ACE_GET_W), "pairs": abi.get_numpy(op, abi.ACE_GET_PAIRS)}
    op.close()
    return out


def _read(op):
    return {"E_x": ace.exchange_energy(op), "xi": abi.get_numpy(op, abi.ACE_GET_XI),
            "W": abi.get_numpy(op, abi.ACE_GET_W), "pairs": abi.get_numpy(op, abi.ACE_GET_PAIRS)}


@pytest.mark.parametrize("lanes", ["1", "3"])
def test_graph_fp64_replays_bit_for_bit(systems, monkeypatch, lanes):
    """Three builds (two grids) in one graph, one after another or on three concurrent lanes;
    replays after the inputs are overwritten in place give exactly the results of ace_build_pairs
    on the new contents, and a second launch without new inputs repeats them."""
    import torch

    monkeypatch.setenv("ACE_GRAPH_LANES", lanes)
    w0, w1, pairs0, c1, all_pairs = systems
    prec = ace.ACE_FP64
    phis = [torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda() for x in (w0.phi, w0.phi, c1.phi)]
    descs = [_desc(w0, prec), _desc(w0, prec), _desc(c1, prec)]
    lists = [pairs0, pairs0[::-1].copy(), all_pairs]
    stream = torch.cuda.current_stream()
    g = ace.ace_graph_create(descs, phis, lists, stream)
    assert abi.ace_graph_size(g) == 3
    try:
        for step, inputs in enumerate(((w0.phi, w1.phi, c1.phi), (w1.phi, w0.phi, c1.phi))):
            for t, x in zip(phis, inputs):
                t.copy_(torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)))
            g.launch(stream)
            if step == 1:
                g.launch(stream)  # back to back: the second replay repeats the first
            g.sync()
            for i, (w, x, pr) in enumerate(zip((w0, w0, c1), inputs, lists)):
                want = _direct(w, prec, pr, x)
                got = _read(g.ops[i])
                assert got["E_x"] == want["E_x"], (step, i)
                assert np.array_equal(got["xi"], want["xi"]), (step, i)
                assert np.array_equal(got["W"], want["W"]), (step, i)
                assert np.array_equal(got["pairs"], want["pairs"])
    finally:
        g.close()
    assert all(op.handle is None for op in g.ops)


@pytest.mark.parametrize("persistent", [False, True])
def test_graph_mixed_against_oracle(systems, monkeypatch, persistent):
    """Mixed form, stream-batched or persistent pair chain recorded into the graph: W and E_x of
    each replay against the oracle on the same pair mask, for two successive snapshots."""
    import torch

    if persistent:
        monkeypatch.setenv("ACE_PERSISTENT", "1")
    w0, w1, pairs0, c1, _ = systems
    prec = ace.ACE_MIXED
    phis = [torch.from_numpy(np.ascontiguousarray(w0.phi, dtype=np.float32)).cuda() for _ in range(2)]
    stream = torch.cuda.current_stream()
    with ace.ace_graph_create([_desc(w0, prec)] * 2, phis, [pairs0, pairs0], stream) as g:
        phis[1].copy_(torch.from_numpy(np.ascontiguousarray(w1.phi, dtype=np.float32)))
        g.launch(stream)
        g.sync()
        mask = mask_from_pairs(pairs0, w0.norb)
        for i, w in enumerate((w0, w1)):
            W_ref = oracle.exchange_w(w.phi, w.lattice, mask=mask)
            r = oracle.ace_from_w(w.phi, W_ref, w.dV, want_xi=False)
            E_ref = oracle.exchange_energy(r["M"], w.spin_factor)
            got = _read(g.ops[i])
            assert rel_max(got["W"].reshape(W_ref.shape), W_ref) <= MIXED_W_RTOL
            assert abs(got["E_x"] - E_ref) <= MIXED_EX_TOL_PER_ORB * w.norb


def test_graph_apply_is_stream_ordered(systems):
    """ace_apply queued on the launch stream after ace_graph_launch sees the replay's xi: K phi of
    the replayed handle equals K phi of a direct build (FP64, exact inputs)."""
    import torch

    w0, w1, pairs0, _, _ = systems
    prec = ace.ACE_FP64
    phi = torch.from_numpy(np.ascontiguousarray(w0.phi, dtype=np.float64)).cuda()
    stream = torch.cuda.current_stream()
    with ace.ace_graph_create([_desc(w0, prec)], [phi], [pairs0], stream) as g:
        phi.copy_(torch.from_numpy(np.ascontiguousarray(w1.phi, dtype=np.float64)))
        g.launch(stream)
        psi = torch.from_numpy(np.ascontiguousarray(w1.phi, dtype=np.float64)).cuda()
        out = torch.empty_like(psi)
        ace.ace_apply(g.ops[0], psi, out, stream)
        g.sync()
        op = ace.ace_build_pairs(_desc(w0, prec), psi, pairs0, stream)
        ref = torch.empty_like(psi)
        ace.ace_apply(op, psi, ref, stream)
        op.close()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_graph_reports_failing_build(systems):
    """A build with an empty pair list has M = 0: the replay completes, ace_graph_sync reports
    ACE_ERR_NOT_POSDEF for that build, and the other build's results stand."""
    import torch

    w0, _, pairs0, _, _ = systems
    prec = ace.ACE_FP64
    phis = [torch.from_numpy(np.ascontiguousarray(w0.phi, dtype=np.float64)).cuda() for _ in range(2)]
    stream = torch.cuda.current_stream()
    with ace.ace_graph_create([_desc(w0, prec)] * 2, phis, [pairs0, np.zeros((0, 2), np.int32)], stream) as g:
        g.launch(stream)
        with pytest.raises(ace.AceError) as e:
            g.sync()
        assert e.value.status == ace.ace.ACE_ERR_NOT_POSDEF
        assert "build 1 of 2" in str(e.value)
        want = _direct(w0, prec, pairs0, w0.phi)
        assert ace.exchange_energy(g.ops[0]) == want["E_x"]


def test_graph_argument_checks(systems):
    import torch

    w0, _, pairs0, _, _ = systems
    stream = torch.cuda.current_stream()
    d = _desc(w0, ace.ACE_MIXED)
    f32 = np.ascontiguousarray(w0.phi, dtype=np.float32)
    cases = [
        (f32, pairs0),  # host input
        (torch.from_numpy(np.ascontiguousarray(w0.phi, dtype=np.float64)).cuda(), pairs0),  # not the working dtype
        (torch.from_numpy(f32).cuda(), np.array([[0, w0.norb]], np.int32)),  # orbital out of range
        (torch.from_numpy(f32).cuda(), np.array([[0, 1], [1, 0]], np.int32)),  # a pair twice
    ]
    for phi, pr in cases:
        with pytest.raises(ace.AceError) as e:
            ace.ace_graph_create([d], [phi], [pr], stream)
        assert e.value.status == ace.ace.ACE_ERR_ARG
    with ace.ace_graph_create([d], [torch.from_numpy(f32).cuda()], [pairs0], stream) as g:
        with pytest.raises(ace.AceError) as e:
            g.sync()  # not launched yet
        assert e.value.status == ace.ace.ACE_ERR_ARG
        g.ops[0].close()  # borrowed: nothing is freed
        assert g.handle
