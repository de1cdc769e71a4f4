"""Host-side partition of one build's screened pair list over several GPUs.

Pairs are independent units of the pair chain (Eq. vx: W_i = sum_j v_ij phi_j), so a build can be
split by giving each rank a subset of the kept pairs; rank r then produces a partial W^(r) over
its pairs and the full W is the sum over ranks (one reduce of n x N values), after which M,
the Cholesky factor and xi follow as on one GPU.  This module holds the partition only; the
one-GPU library is what each rank would run on its subset.
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
