"""bench.py --impl reference: the FP64 oracle timed on a bounded sample of the config-2 build.  One
short step must print one JSON line whose timed region (steps x ms_per_step) fits inside the run's
own wall clock, with value = the fraction of a build the steps computed per second of step time."""

import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_fits_its_run():
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-step-s", "2"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["unit"] == "builds/s" and d["value"] > 0
    frac = d["build_fraction_per_step"]
    assert 0.0 < frac <= 1.0
    # the timed region is the measured step time, inside the run's own clock
    assert d["steps"] * d["ms_per_step"] / 1e3 <= wall
    # value: build fractions per second of step time
    assert abs(d["value"] - frac / (d["ms_per_step"] / 1e3)) <= 1e-9 * d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
