"""Plane skip of the mixed form's pair chain: planes on which a pack's pair densities are negligible
(below ACE_PLANE_SKIP, default 1e-7, times the orbitals' maxima) get a zero spectrum instead of a
forward transform, and planes on which every orbital of the pack is negligible get no inverse
transform or W accumulation.  Sharp Gaussians in one corner of a large cell make most planes
negligible; W and E_x must still match the FP64 oracle (all pairs, mixed-form tolerances) on the
plane chain and the persistent chain, and match the build with the skip turned off."""

import numpy as np
import pytest

import oracle
import paper_2101_03155_gb300 as ace
from gpu_helpers import MIXED_EX_TOL_PER_ORB, MIXED_W_RTOL, gpu_build, rel_max
from workloads.generators import loewdin, periodic_gaussian

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    assert torch.cuda.is_available()
    from paper_2101_03155_gb300 import build

    build.build()
    ace.ace.load()
    oracle.build()


def _cluster(grid=(48, 48, 48), cell=20.0, n=6, seed=77):
    """n orthonormal orbitals from sharp Gaussians (exponents 1.5-3 bohr^-2) centred within 3 bohr of
    one point of a 20-bohr cubic cell: far from the cluster every orbital is below 1e-7 of its peak."""
    rng = np.random.default_rng(seed)
    lat = np.diag([cell, cell, cell])
    ctr = np.array([5.0, 6.0, 5.5])
    chi = np.stack([periodic_gaussian(grid, lat, ctr + rng.uniform(-3, 3, 3), rng.uniform(1.5, 3.0))
                    for _ in range(n)])
    dV = cell ** 3 / np.prod(grid)
    phi, _ = loewdin(chi, dV)
    return phi, lat


@pytest.mark.parametrize("persistent", ["0", "1"])
def test_plane_skip_matches_the_oracle(monkeypatch, persistent):
    phi, lat = _cluster()
    ref = oracle.ace_build(phi, lat, 0.0, 2.0, want_xi=False)
    monkeypatch.setenv("ACE_PERSISTENT", persistent)
    g = gpu_build(phi, lat, ace.ACE_MIXED)
    assert g["status"] == 0
    assert rel_max(g["W"].reshape(ref["W"].shape), ref["W"]) <= MIXED_W_RTOL
    assert abs(g["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * phi.shape[0]
    monkeypatch.setenv("ACE_PLANE_SKIP", "0")
    h = gpu_build(phi, lat, ace.ACE_MIXED)
    assert rel_max(g["W"], h["W"]) <= MIXED_W_RTOL
    assert abs(g["E_x"] - h["E_x"]) <= 0.1 * MIXED_EX_TOL_PER_ORB * phi.shape[0]


def test_fp64_form_never_skips(monkeypatch):
    """The FP64 form ignores ACE_PLANE_SKIP: the same W bit for bit with any setting."""
    phi, lat = _cluster()
    monkeypatch.setenv("ACE_PLANE_SKIP", "1e-3")
    a = gpu_build(phi, lat, ace.ACE_FP64)
    monkeypatch.setenv("ACE_PLANE_SKIP", "0")
    b = gpu_build(phi, lat, ace.ACE_FP64)
    assert np.array_equal(a["W"], b["W"]) and a["E_x"] == b["E_x"]
