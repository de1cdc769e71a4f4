"""Write tests/golden/oracle_values.json (and one .npz of arrays per build) from the FP64 oracle.
It calls only oracle/ and the seeded input generators.  The paper prints no worked example for
this path, so these stored values are oracle outputs on the synthetic workloads.  The full-size
GPU tests and the bench compare against them without rerunning a full-size oracle build.

Per build the JSON entry holds E_x, the pair count and diag(M).  The .npz holds the oracle's pair
list (i <= j, the screen of section II) and, for the sampled builds, at seeded grid points:
xi (every row), K phi_k for every orbital, and for two seeded probe vectors psi their
C = dV xi^T psi and K psi = -xi C (section II, ACE application).

    python tests/golden/make_golden.py                 # every value
    python tests/golden/make_golden.py water64         # selected makers, merged into the file
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from workloads.generators import (config1, config2, config3, config4, config5, probe_vectors,  # noqa: E402
                                  sample_points)

HERE = os.path.dirname(os.path.abspath(__file__))
SAMPLE_SEED = 4242


def _entry(w, r, nsamples=0, kind=oracle.PERIODIC):
    """JSON entry and arrays of one oracle build."""
    n = w.norb
    mask = r["mask"] if r["mask"] is not None else np.ones((n, n), bool)
    pairs = np.argwhere(np.triu(mask)).astype(np.int32)
    entry = {"E_x": r["E_x"], "npairs": int(len(pairs)), "M_diag": np.diag(r["M"]).tolist(), "norb": n,
             "grid": list(w.grid)}
    arrays = {"pairs": pairs}
    if nsamples:
        idx = sample_points(w.npts, nsamples, SAMPLE_SEED)
        psi = probe_vectors(w.phi, w.dV, SAMPLE_SEED)
        C, kpsi = oracle.ace_apply_at(r["xi"], psi, w.dV, idx)
        _, kphi = oracle.ace_apply_at(r["xi"], w.phi, w.dV, idx)
        arrays.update(idx=idx, xi=r["xi"].reshape(n, -1)[:, idx], C=C, kpsi=kpsi, kphi=kphi,
                      probe_seed=np.int64(SAMPLE_SEED))
        entry["nsamples"] = int(len(idx))
    return entry, arrays


def _config1():
    w = config1()
    r = oracle.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)
    return w.name, _entry(w, r)


def _water32():
    w = config2()
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=True)
    return "water32_128orb_96c_rhocut1e-3", _entry(w, r, nsamples=4096)


def _water64():
    w = config3()
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=True)
    return "water64_256orb_128c_rhocut1e-3", _entry(w, r, nsamples=2048)


def _enzyme_snap0_isolated():
    """First snapshot of the enzyme-like cluster with the isolated-cell kernel (1/r cut off at the
    inscribed radius, 15 bohr)."""
    w = config5(nsnap=1)[0]
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=False,
                         kind=oracle.TRUNCATED, r_cut=0.0)
    return "enzyme_snap0_isolated", _entry(w, r)


def _enzyme_snap0_periodic():
    w = config5(nsnap=1)[0]
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=False)
    return "enzyme_snap0_periodic", _entry(w, r)


def _batched(b):
    def make():
        w = config4(builds=[b])[0]
        r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=False)
        return f"batched24_b{b}_{w.norb}orb_{w.grid[0]}c", _entry(w, r)
    return make


MAKERS = {"config1": _config1, "water32": _water32, "water64": _water64,
          "enzyme_snap0_isolated": _enzyme_snap0_isolated, "enzyme_snap0_periodic": _enzyme_snap0_periodic,
          "batched_b1": _batched(1), "batched_b15": _batched(15), "batched_b12": _batched(12)}


def main(keys):
    path = os.path.join(HERE, "oracle_values.json")
    out = json.load(open(path)) if keys and os.path.exists(path) else {}
    for key in keys or list(MAKERS):
        t0 = time.time()
        name, (val, arrays) = MAKERS[key]()
        val.update(seconds=time.time() - t0, threads=oracle.max_threads(), arrays=f"{name}.npz")
        np.savez_compressed(os.path.join(HERE, f"{name}.npz"), **arrays)
        out[name] = val
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(json.dumps({name: {kk: val[kk] for kk in ("E_x", "npairs", "seconds")}}), flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
