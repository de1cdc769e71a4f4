"""One ACE build over several GPUs: the host-side decomposition that each rank runs.

The pairs of Eq. (vx) are independent terms of W (W_i = sum_j v_ij phi_j), and everything after
W in App. A splits over grid points: M_kl = -dV sum_r phi_k(r) W_l(r) is a sum over points, and
xi = W L^-T acts on each point separately.  On R ranks (one GPU and one process each):

  1. rank r computes the partial W^(r) of its contiguous share of the sorted pair list
     (ace_exchange_w);
  2. one reduce-scatter sums the W^(r) and leaves rank r the point slab W[:, slab_r];
  3. rank r forms M^(r) = -dV Phi[:, slab_r]^T W[:, slab_r] (ace_m_partial);
  4. one all-reduce (FP64, norb^2 values) gives every rank M; every rank factors it (replicated)
     and keeps xi on its slab (ace_build_from_m);
  5. the application needs one more all-reduce: C = dV xi^T psi summed over the slabs
     (ace_apply_coeffs, all-reduce, ace_apply_finish).

Only step 2 moves orbital-sized data (n N values once); the pair chain, which holds nearly all of
the work, needs no exchange at all.  ``kernels`` is the per-rank compute (the C ABI on the rank's
GPU, ``GpuSlabKernels``); ``comm`` is a ``Collectives`` over torch.distributed (NCCL on GPUs).
"""

from __future__ import annotations

import numpy as np


def shard_pairs(pairs: np.ndarray, nranks: int) -> list[np.ndarray]:
    """Split sorted (i, j) pairs into nranks contiguous, nearly equal blocks.

    Contiguous blocks keep each rank's pairs grouped by their first orbital (the packing of the
    pair chain relies on that); every pair costs the same transform work.
    """
    pairs = np.asarray(pairs, dtype=np.int32).reshape(-1, 2)
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    bounds = np.linspace(0, len(pairs), nranks + 1).round().astype(int)
    return [pairs[bounds[r]:bounds[r + 1]] for r in range(nranks)]


def pair_mask(pairs: np.ndarray, n: int) -> np.ndarray:
    """Symmetric boolean mask of the given (i <= j) pairs."""
    m = np.zeros((n, n), dtype=bool)
    p = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    m[p[:, 0], p[:, 1]] = True
    m[p[:, 1], p[:, 0]] = True
    return m


def point_slabs(npts: int, nranks: int, align: int = 128) -> list[tuple[int, int]]:
    """Contiguous slabs [p0, p1) of the grid points, one per rank, with every inner boundary on a
    multiple of `align` points (the tensor-core contractions step through 128 points) and sizes
    within `align` of each other."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    units = (npts + align - 1) // align
    cuts = [min(npts, int(round(units * r / nranks)) * align) for r in range(nranks + 1)]
    cuts[-1] = npts
    return [(cuts[r], cuts[r + 1]) for r in range(nranks)]


class Collectives:
    """The three collectives of the decomposition over a torch.distributed process group."""

    def __init__(self, dist, group=None):
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def reduce_scatter_slabs(self, W, slabs):
        """Sum of every rank's W (rows x points) restricted to this rank's slab, contiguous."""
        import torch

        rows = W.shape[0]
        chunks = [W[:, p0:p1].contiguous() for p0, p1 in slabs]
        equal = len({c.numel() for c in chunks}) == 1
        if equal and self.dist.get_backend(self.group) == "nccl":
            out = torch.empty_like(chunks[self.rank])
            self.dist.reduce_scatter(out, chunks, group=self.group)
            return out
        # backends without reduce-scatter, or uneven slabs: one reduce per destination slab
        for d, c in enumerate(chunks):
            self.dist.reduce(c, dst=d, group=self.group)
        return chunks[self.rank].reshape(rows, -1)

    def all_reduce(self, t):
        self.dist.all_reduce(t, group=self.group)
        return t


class GpuSlabKernels:
    """The per-rank steps through the C ABI on the current GPU (device tensors, working dtype)."""

    def __init__(self, desc, stream=None):
        self.desc = desc
        self.stream = stream

    def _dtype(self):
        import torch

        from .ace import ACE_FP64

        return torch.float64 if self.desc.prec == ACE_FP64 else torch.float32

    def exchange_w(self, phi, pairs):
        import torch

        from . import ace

        W = torch.empty((self.desc.norb, phi.numel() // self.desc.norb), dtype=self._dtype(), device=phi.device)
        return ace.ace_exchange_w(self.desc, phi, pairs, W, self.stream)

    def m_partial(self, phi_slab, W_slab):
        import torch

        from . import ace

        M = torch.empty((self.desc.norb, self.desc.norb), dtype=torch.float64, device=W_slab.device)
        return ace.ace_m_partial(self.desc, phi_slab.contiguous(), W_slab.contiguous(), M, self.stream)

    def build_from_m(self, M, W_slab):
        from . import ace

        return ace.ace_build_from_m(self.desc, M, W_slab.contiguous(), self.stream)

    def apply_coeffs(self, op, psi_slab):
        import torch

        from . import ace

        C = torch.empty((self.desc.norb, psi_slab.shape[0]), dtype=torch.float64, device=psi_slab.device)
        return ace.ace_apply_coeffs(op, psi_slab.contiguous(), C, self.stream)

    def apply_finish(self, op, C, m):
        import torch

        from . import ace

        out = torch.empty((m, op.npts), dtype=self._dtype(), device=C.device)
        return ace.ace_apply_finish(op, C, out, self.stream)


def sharded_build(kernels, comm, phi, pairs, slabs=None):
    """Steps 1-4 on this rank: returns (operator on this rank's slab, the slab (p0, p1)).
    phi: this rank's copy of all orbitals [norb][N]; pairs: the whole (sorted) pair list."""
    n = phi.shape[0]
    npts = phi.reshape(n, -1).shape[1]
    slabs = slabs or point_slabs(npts, comm.world)
    p0, p1 = slabs[comm.rank]
    W = kernels.exchange_w(phi, shard_pairs(pairs, comm.world)[comm.rank])
    W_slab = comm.reduce_scatter_slabs(W.reshape(n, npts), slabs)
    M = kernels.m_partial(phi.reshape(n, npts)[:, p0:p1], W_slab)
    comm.all_reduce(M)
    return kernels.build_from_m(M, W_slab), (p0, p1)


def sharded_apply(kernels, comm, op, psi_slab):
    """Step 5: K psi on this rank's slab, psi_slab [m][slab points]."""
    C = kernels.apply_coeffs(op, psi_slab)
    comm.all_reduce(C)
    return kernels.apply_finish(op, C, psi_slab.shape[0])
