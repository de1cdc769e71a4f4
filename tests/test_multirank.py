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
