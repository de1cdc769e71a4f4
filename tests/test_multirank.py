"""World-size-2 tests on CPU (gloo): the bench's whole-job aggregation and the pair-sharded
decomposition of one build (partial W per rank, summed over ranks, equals the full W)."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _init(rank, world, port):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _aggregate_worker(rank, world, port, out):
    dist = _init(rank, world, port)
    import bench

    ms, value = bench.combine_ranks(100.0 + 50.0 * rank, steps=10, units_per_step=1.0)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_combine_ranks_takes_the_slowest_rank():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_aggregate_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        ms, value = out[r]
        assert ms == 150.0
        assert abs(value - 2 * 10 / 0.150) < 1e-9


def _shard_worker(rank, world, port, out):
    dist = _init(rank, world, port)
    import torch

    import oracle
    from paper_2101_03155_gb300.sharding import pair_mask, shard_pairs
    from workloads.generators import water_like

    oracle.set_threads(2)
    w = water_like(4, 9.3, (24, 24, 24), np.random.default_rng(606), rho_cut=1e-3, dmin=3.5)
    _, mask = oracle.screen(w.phi, w.lattice, w.rho_cut)
    iu = np.triu_indices(w.norb)
    pairs = np.stack([iu[0][mask[iu]], iu[1][mask[iu]]], axis=1)
    mine = shard_pairs(pairs, world)[rank]
    W_part = oracle.exchange_w(w.phi, w.lattice, mask=pair_mask(mine, w.norb))
    # a diagonal pair contributes once; off-diagonal pairs once to each of their two rows
    t = torch.from_numpy(W_part.copy())
    dist.all_reduce(t)
    if rank == 0:
        full = oracle.exchange_w(w.phi, w.lattice, mask=mask)
        out["err"] = float(np.abs(t.numpy() - full).max() / np.abs(full).max())
        out["sizes"] = [len(x) for x in shard_pairs(pairs, world)]
    dist.destroy_process_group()


def test_pair_sharded_w_sums_to_the_full_w():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_shard_worker, args=(2, port, out), nprocs=2, join=True)
    assert out["err"] <= 1e-14
    assert abs(out["sizes"][0] - out["sizes"][1]) <= 1


def test_shard_pairs_partition():
    from paper_2101_03155_gb300.sharding import shard_pairs

    pairs = np.array([(i, j) for i in range(7) for j in range(i, 7) if (i + j) % 3], dtype=np.int32)
    for r in (1, 2, 3, 5):
        parts = shard_pairs(pairs, r)
        assert len(parts) == r
        assert np.array_equal(np.concatenate(parts), pairs)
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_pairs(pairs, 0)


class _OracleSlabKernels:
    """The per-rank steps restated with the FP64 oracle (and LAPACK for the factorisation of the
    summed M), on numpy-backed CPU tensors."""

    def __init__(self, w):
        self.w = w

    def exchange_w(self, phi, pairs):
        import torch

        import oracle
        from paper_2101_03155_gb300.sharding import pair_mask

        W = oracle.exchange_w(phi.numpy(), self.w.lattice, mask=pair_mask(pairs, self.w.norb))
        return torch.from_numpy(W.reshape(self.w.norb, -1).copy())

    def m_partial(self, phi_slab, W_slab):
        import torch

        import oracle

        r = oracle.ace_from_w(phi_slab.numpy(), W_slab.numpy(), self.w.dV, want_xi=False)
        return torch.from_numpy(r["M_raw"].copy())

    def build_from_m(self, M, W_slab):
        import scipy.linalg as sla

        Ms = 0.5 * (M.numpy() + M.numpy().T)
        L = np.linalg.cholesky(-Ms)
        xi = sla.solve_triangular(L, W_slab.numpy(), lower=True)
        return {"M": Ms, "L": L, "xi": xi, "E_x": 0.5 * self.w.spin_factor * np.trace(Ms)}

    def apply_coeffs(self, op, psi_slab):
        import torch

        return torch.from_numpy(self.w.dV * op["xi"] @ psi_slab.numpy().T)

    def apply_finish(self, op, C, m):
        import torch

        return torch.from_numpy(-(C.numpy().T @ op["xi"]))


def _slab_worker(rank, world, port, out):
    dist = _init(rank, world, port)
    import torch

    import oracle
    from paper_2101_03155_gb300.sharding import Collectives, point_slabs, sharded_apply, sharded_build
    from workloads.generators import probe_vectors, water_like

    oracle.set_threads(2)
    w = water_like(4, 9.3, (24, 24, 24), np.random.default_rng(606), rho_cut=1e-3, dmin=3.5)
    _, mask = oracle.screen(w.phi, w.lattice, w.rho_cut)
    iu = np.triu_indices(w.norb)
    pairs = np.stack([iu[0][mask[iu]], iu[1][mask[iu]]], axis=1)
    comm = Collectives(dist)
    kern = _OracleSlabKernels(w)
    slabs = point_slabs(w.npts, world)
    op, (p0, p1) = sharded_build(kern, comm, torch.from_numpy(w.phi.copy()), pairs, slabs)
    psi = probe_vectors(w.phi, w.dV, 5).reshape(2, -1)
    kpsi_slab = sharded_apply(kern, comm, op, torch.from_numpy(psi[:, p0:p1].copy())).numpy()
    ref = oracle.ace_build(w.phi, w.lattice, mask=mask, spin_factor=w.spin_factor)
    xi_ref = ref["xi"].reshape(w.norb, -1)[:, p0:p1]
    kref = oracle.ace_apply(ref["xi"], psi.reshape((2,) + w.grid), w.dV).reshape(2, -1)[:, p0:p1]
    out[rank] = {
        "slab": (p0, p1),
        "M": float(np.abs(op["M"] - ref["M"]).max() / np.abs(ref["M"]).max()),
        "L": float(np.abs(op["L"] - ref["L"]).max() / np.abs(ref["L"]).max()),
        "xi": float(np.abs(op["xi"] - xi_ref).max() / np.abs(xi_ref).max()),
        "E_x": abs(op["E_x"] - ref["E_x"]),
        "kpsi": float(np.abs(kpsi_slab - kref).max() / np.abs(kref).max()),
    }
    dist.destroy_process_group()


def test_slab_decomposition_matches_one_rank_build():
    """World size 2 (gloo): pair shards -> partial W -> reduce-scatter over point slabs -> M
    partials -> all-reduce -> replicated Cholesky and xi on each slab -> sharded application,
    each step restated with the oracle; equals the one-rank oracle build to 1e-12."""
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_slab_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0]["slab"][1] == out[1]["slab"][0]
    for r in range(2):
        for key in ("M", "L", "xi", "kpsi"):
            assert out[r][key] <= 1e-12, (r, key, out[r][key])
        assert out[r]["E_x"] <= 1e-12


def test_point_slabs_partition():
    from paper_2101_03155_gb300.sharding import point_slabs

    for npts, r in ((884736, 2), (884736, 8), (13824, 3), (1000, 4), (100, 1)):
        s = point_slabs(npts, r)
        assert s[0][0] == 0 and s[-1][1] == npts and len(s) == r
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        assert all(p1 % 128 == 0 for _, p1 in s[:-1])
        sizes = [p1 - p0 for p0, p1 in s]
        assert max(sizes) - min(sizes) <= 128
