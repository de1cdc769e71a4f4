"""Write tests/golden/oracle_values.json from the FP64 oracle (calls only oracle/ and the seeded
input generators).  The paper prints no worked example for this path, so these stored values are
oracle outputs on the synthetic workloads, used by the bench to report the E_x error of the GPU
forms without rerunning a full-size oracle build.

    python tests/golden/make_golden.py                      # every value
    python tests/golden/make_golden.py enzyme_snap0_isolated   # selected keys, merged into the file
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from workloads.generators import config1, config2, config5  # noqa: E402


def _config1():
    w = config1()
    r = oracle.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)
    npairs = int(np.triu(r["mask"] if r["mask"] is not None else np.ones((w.norb, w.norb), bool)).sum())
    return w.name, {"E_x": r["E_x"], "npairs": npairs, "M_diag": np.diag(r["M"]).tolist()}


def _water32():
    w = config2()
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=False)
    return "water32_128orb_96c_rhocut1e-3", {"E_x": r["E_x"], "npairs": int(np.triu(r["mask"]).sum()),
                                             "M_diag": np.diag(r["M"]).tolist()}


def _enzyme_snap0_isolated():
    """First snapshot of the enzyme-like cluster with the isolated-cell kernel (1/r cut off at the
    inscribed radius, 15 bohr)."""
    w = config5(nsnap=1)[0]
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=False,
                         kind=oracle.TRUNCATED, r_cut=0.0)
    return "enzyme_snap0_isolated", {"E_x": r["E_x"], "npairs": int(np.triu(r["mask"]).sum()),
                                     "M_diag": np.diag(r["M"]).tolist()}


MAKERS = {"config1_plain_16orb_32c": _config1, "water32_128orb_96c_rhocut1e-3": _water32,
          "enzyme_snap0_isolated": _enzyme_snap0_isolated}


def main(keys):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")
    out = json.load(open(path)) if keys and os.path.exists(path) else {}
    for key in keys or list(MAKERS):
        t0 = time.time()
        name, val = MAKERS[key]()
        val.update(seconds=time.time() - t0, threads=oracle.max_threads())
        out[name] = val
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: {kk: v[kk] for kk in ("E_x", "npairs", "seconds")} for k, v in out.items()}))


if __name__ == "__main__":
    main(sys.argv[1:])
