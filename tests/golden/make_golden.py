"""Write tests/golden/oracle_values.json from the FP64 oracle (calls only oracle/ and the seeded
input generators).  The paper prints no worked example for this path, so these stored values are
oracle outputs on the synthetic workloads, used by the bench to report the E_x error of the GPU
forms without rerunning a full-size oracle build.

    python tests/golden/make_golden.py
"""

import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from workloads.generators import config1, config2  # noqa: E402


def main():
    out = {}
    w = config1()
    t0 = time.time()
    r = oracle.ace_build(w.phi, w.lattice, 0.0, w.spin_factor)
    out[w.name] = {"E_x": r["E_x"], "npairs": int(np.triu(r["mask"] if r["mask"] is not None else
                                                          np.ones((w.norb, w.norb), bool)).sum()),
                   "M_diag": np.diag(r["M"]).tolist(), "seconds": time.time() - t0}
    w = config2()
    t0 = time.time()
    r = oracle.ace_build(w.phi, w.lattice, rho_cut=w.rho_cut, spin_factor=w.spin_factor, want_xi=False)
    out["water32_128orb_96c_rhocut1e-3"] = {
        "E_x": r["E_x"], "npairs": int(np.triu(r["mask"]).sum()), "M_diag": np.diag(r["M"]).tolist(),
        "seconds": time.time() - t0, "threads": oracle.max_threads(),
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: {kk: v[kk] for kk in ("E_x", "npairs", "seconds")} for k, v in out.items()}))


if __name__ == "__main__":
    main()
