"""ace_autotune: the pair-chain settings it picks (stream-batched settings with the pencil tile of
the axis-1 pass, or the persistent chain with its queue lag) are valid, are used by later builds
(same operator within the mixed-form tolerance), and persist through ACE_TUNE_FILE; every pencil
tile gives the oracle's W."""

import os

import numpy as np
import pytest

import paper_2101_03155_gb300 as ace
from gpu_helpers import MIXED_EX_TOL_PER_ORB
from paper_2101_03155_gb300 import ace as abi
from workloads.generators import water_like

pytestmark = pytest.mark.gpu


def test_autotune_picks_valid_settings_and_builds_agree(tmp_path):
    import torch

    from paper_2101_03155_gb300 import build

    build.build()
    abi.load()
    w = water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)
    phi = torch.from_numpy(w.phi.astype(np.float32)).cuda()
    d = ace.make_desc(w.grid, w.lattice, w.norb, rho_cut=w.rho_cut, prec=ace.ACE_MIXED)
    stream = torch.cuda.current_stream()
    before = ace.ace_build(d, phi, stream)
    e0 = ace.exchange_energy(before)
    before.close()
    tune_file = tmp_path / "ace_tune.txt"
    os.environ["ACE_TUNE_FILE"] = str(tune_file)
    try:
        p = abi.ace_autotune(d, phi, stream)
    finally:
        del os.environ["ACE_TUNE_FILE"]
    assert p["group"] >= 1 and p["batch"] in (1, 2, 3, 4, 6) and p["streams"] in (2, 4, 8) and p["l2_mb"] in (0, 60)
    assert p["row_block"] in (1, 2, 4, 8) and p["persistent_lag"] in (0, 2, 3, 4) and p["pencil_tile"] in (0, 1, 2)
    fields = tune_file.read_text().split()
    assert len(fields) == 12
    assert fields[:4] == ["48", "48", "48", "0"] and [int(x) for x in fields[4:9]] == [
        p["group"], p["batch"], p["streams"], p["l2_mb"], p["row_block"]]
    assert int(fields[9]) == (p["persistent_lag"] > 0) and int(fields[11]) == p["pencil_tile"]
    after = ace.ace_build(d, phi, stream)
    assert abs(ace.exchange_energy(after) - e0) <= MIXED_EX_TOL_PER_ORB * w.norb
    after.close()


@pytest.mark.parametrize("tile", ["1", "2"])
def test_pencil_tiles_match_the_oracle(tile, monkeypatch):
    """The two non-default pencil tiles of the axis-1 pass (FP32) on the 72^2 and 108^2 plane shapes
    and an axis-1 length of 40 with 32 x 32 planes: W of the oracle (all pairs)."""
    import oracle
    from gpu_helpers import MIXED_W_RTOL, gpu_build, rel_max
    from workloads.generators import gaussian_orbitals

    oracle.build()
    monkeypatch.setenv("ACE_CONV_TILE", tile)
    for grid, cell in (((72, 72, 72), 11.0), ((108, 108, 108), 12.0), ((40, 32, 32), 9.0)):
        lat = np.diag([cell, cell * grid[1] / grid[0], cell * grid[2] / grid[0]])
        phi, _, _ = gaussian_orbitals(grid, lat, 4, 2, np.random.default_rng(sum(grid)))
        ref = oracle.ace_build(phi, lat, 0.0, 2.0, want_xi=False)
        g = gpu_build(phi, lat, ace.ACE_MIXED)
        assert rel_max(g["W"].reshape(ref["W"].shape), ref["W"]) <= MIXED_W_RTOL, grid
