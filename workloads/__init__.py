"""Seeded synthetic inputs (orbitals on periodic grids) shared by the tests and the bench.

This package holds input preparation only: Gaussian orbital sampling, site placement and
Loewdin orthonormalisation. None of the exchange method's arithmetic lives here; the CUDA path
and the FP64 oracle each implement that on their own.
"""

from .generators import (  # noqa: F401
    Workload,
    gaussian_orbitals,
    water_like,
    enzyme_like,
    batched_set,
    config1,
    config2,
    config3,
    config5,
    loewdin,
    random_orthogonal,
)
