"""ace_autotune: the pair-chain settings it picks (stream-batched settings, or the persistent chain
with its queue lag) are valid, are used by later builds (same operator within the mixed-form
tolerance), and persist through ACE_TUNE_FILE."""

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
    assert p["row_block"] in (1, 2, 4, 8) and p["persistent_lag"] in (0, 2, 3, 4)
    fields = tune_file.read_text().split()
    assert fields[:4] == ["48", "48", "48", "0"] and [int(x) for x in fields[4:9]] == [
        p["group"], p["batch"], p["streams"], p["l2_mb"], p["row_block"]]
    assert int(fields[9]) == (p["persistent_lag"] > 0)
    after = ace.ace_build(d, phi, stream)
    assert abs(ace.exchange_energy(after) - e0) <= MIXED_EX_TOL_PER_ORB * w.norb
    after.close()
