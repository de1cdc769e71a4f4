"""The register-staged tensor-core kernels (used when TMA cannot map an operand, or with
ACE_NO_TMA=1) give the same mixed build and application as the TMA kernels, against the oracle.
The switch is read once per process, so the fallback runs in a child process."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from gpu_helpers import MIXED_EX_TOL_PER_ORB, MIXED_KPHI_RTOL

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
import paper_2101_03155_gb300 as ace
from workloads.generators import config1
w = config1()
d = ace.make_desc(w.grid, w.lattice, w.norb, prec=ace.ACE_MIXED)
op = ace.ace_build(d, torch.from_numpy(w.phi.astype(np.float32)).cuda())
psi = np.random.default_rng(21).standard_normal((3,) + w.grid).astype(np.float32)
out = torch.empty((3,) + w.grid, dtype=torch.float32, device="cuda")
ace.ace_apply(op, torch.from_numpy(psi).cuda(), out)
np.save(sys.argv[1], out.cpu().numpy())
print(json.dumps({{"E_x": ace.exchange_energy(op)}}))
"""


def test_fallback_kernels_match_oracle(tmp_path):
    from workloads.generators import config1

    w = config1()
    ref = oracle.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)
    out_file = tmp_path / "kphi.npy"
    env = dict(os.environ, ACE_NO_TMA="1")
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT), str(out_file)], env=env, capture_output=True,
                       text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert abs(res["E_x"] - ref["E_x"]) <= MIXED_EX_TOL_PER_ORB * w.norb
    psi = np.random.default_rng(21).standard_normal((3,) + w.grid).astype(np.float32)
    kref = oracle.ace_apply(ref["xi"], psi.astype(np.float64), w.dV)
    got = np.load(out_file)
    assert np.linalg.norm(got - kref) <= MIXED_KPHI_RTOL * np.linalg.norm(kref)


CHILD_CHOL = r"""
import sys
import numpy as np, torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_2101_03155_gb300 as ace
from gpu_helpers import gpu_build
from workloads.generators import water_like
w = water_like(8, 11.74, (48, 48, 48), np.random.default_rng(1010), rho_cut=1e-3, dmin=4.0)
g = gpu_build(w.phi, w.lattice, ace.ACE_FP64, rho_cut=w.rho_cut)
np.savez(sys.argv[1], L=g["L"], M=g["M"], E=np.array(g["E_x"]))
"""


CHILD_CHOL_WIDE = r"""
import sys
import numpy as np, torch
sys.path.insert(0, {root!r})
sys.path.insert(0, {tests!r})
import paper_2101_03155_gb300 as ace
from gpu_helpers import gpu_build
from workloads.generators import water_like
w = water_like({nmol}, {cell!r}, (48, 48, 48), np.random.default_rng(1011), rho_cut=1e-3)
g = gpu_build(w.phi, w.lattice, ace.ACE_FP64, rho_cut=w.rho_cut)
np.savez(sys.argv[1], L=g["L"], M=g["M"], E=np.array(g["E_x"]), xi=g["xi"], W=g["W"])
"""


@pytest.mark.parametrize("nmol", [48, 64])
def test_wide_cluster_cholesky_matches_one_cta(tmp_path, nmol):
    """Above 128 orbitals (192 and 256 here) the cluster kernel with columns spread over its CTAs and
    the one-CTA kernel (ACE_CHOLESKY_ONE_CTA=1) both factor -M = L L^T to FP64 rounding, and
    xi = L^-1 W holds with the GPU's own W and L (the FP64 left multiply adds no error of note)."""
    cell = 23.47 * (nmol / 64.0) ** (1.0 / 3.0)  # water density
    outs = {}
    for name, flag in (("cluster", "0"), ("one_cta", "1")):
        f = tmp_path / f"{name}.npz"
        env = dict(os.environ, ACE_CHOLESKY_ONE_CTA=flag)
        code = CHILD_CHOL_WIDE.format(root=ROOT, tests=os.path.join(ROOT, "tests"), nmol=nmol, cell=cell)
        r = subprocess.run([sys.executable, "-c", code, str(f)], env=env, capture_output=True, text=True,
                           timeout=900, cwd=ROOT)
        assert r.returncode == 0, r.stderr[-2000:]
        outs[name] = np.load(f)
    a, b = outs["cluster"], outs["one_cta"]
    assert a["L"].shape == (4 * nmol, 4 * nmol)
    assert np.abs(a["M"] - b["M"]).max() <= 1e-13 * np.abs(b["M"]).max()
    assert abs(float(a["E"]) - float(b["E"])) <= 1e-12 * abs(float(b["E"]))
    eps = np.finfo(np.float64).eps
    for o in (a, b):
        L, M = o["L"], o["M"]
        assert np.all(np.triu(L, 1) == 0.0)
        # backward error of the factorisation: L L^T = -M to rounding (n eps |M|, with margin)
        assert np.abs(L @ L.T + M).max() <= 1e-12 * np.abs(M).max()
        # forward error against LAPACK's factor of the same M: a multiple of cond(-M) eps (the
        # orbitals of a coarse 48^3 grid leave -M with cond ~ 1e6 at 256 orbitals)
        cond = np.linalg.cond(-M)
        L_ref = np.linalg.cholesky(-M)
        assert np.abs(L - L_ref).max() <= max(1e-12, 10 * cond * eps) * np.abs(L_ref).max()
        # xi = L^-1 W through L^-1 (forward substitution): a multiple of cond(L) eps
        W = o["W"].reshape(L.shape[0], -1)
        xi_ref = np.linalg.solve(L, W)
        tol = max(1e-10, 10 * np.sqrt(cond) * eps)
        assert np.abs(o["xi"].reshape(xi_ref.shape) - xi_ref).max() <= tol * np.abs(xi_ref).max()
    # the two kernels' factors agree to the same forward bound
    cond = np.linalg.cond(-b["M"])
    assert np.abs(a["L"] - b["L"]).max() <= max(1e-12, 20 * cond * eps) * np.abs(b["L"]).max()


def test_one_cta_cholesky_matches_cluster_cholesky(tmp_path):
    """The cluster Cholesky (default for n <= 128) and the one-CTA kernel (ACE_CHOLESKY_ONE_CTA=1)
    factor the same M to FP64 rounding, and both L L^T = -M."""
    outs = {}
    for name, flag in (("cluster", "0"), ("one_cta", "1")):
        f = tmp_path / f"{name}.npz"
        env = dict(os.environ, ACE_CHOLESKY_ONE_CTA=flag)
        r = subprocess.run([sys.executable, "-c", CHILD_CHOL.format(root=ROOT, tests=os.path.join(ROOT, "tests")),
                            str(f)], env=env, capture_output=True, text=True, timeout=600, cwd=ROOT)
        assert r.returncode == 0, r.stderr[-2000:]
        outs[name] = np.load(f)
    # the FP64 pair chain accumulates W with atomics, so M itself differs at the rounding level
    # between the two runs: each factor is checked against LAPACK's factor of its own M
    a, b = outs["cluster"], outs["one_cta"]
    assert np.abs(a["M"] - b["M"]).max() <= 1e-13 * np.abs(b["M"]).max()
    assert abs(float(a["E"]) - float(b["E"])) <= 1e-12 * abs(float(b["E"]))
    for o in (a, b):
        L = o["L"]
        L_ref = np.linalg.cholesky(-o["M"])
        assert np.abs(L - L_ref).max() <= 1e-12 * np.abs(L_ref).max()
        assert np.all(np.triu(L, 1) == 0.0)
