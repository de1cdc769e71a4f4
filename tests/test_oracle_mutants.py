"""Plant plausible mistakes in a copy of the oracle and check that the pins catch each one.

Every mutant is a one-line textual change to ``oracle/ace_oracle.c`` compiled into a temporary
library on the CPU.  The battery below is a fast subset of tests/test_oracle_pins.py; a mutant
that passes the whole battery would mean the pins cannot see that class of mistake.
"""

import os
import shutil

import numpy as np
import pytest

import closed_form as cf
from workloads.generators import gaussian_orbitals

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "ace_oracle.c")
TRICLINIC = np.array([[7.5, 0.0, 0.0], [1.2, 7.0, 0.0], [0.6, -0.9, 6.8]])

MUTANTS = {
    "twiddle_sign": ("if (sign > 0) w = conj(w);", "if (sign < 0) w = conj(w);"),
    "combine_index": ("acc += w * y[q * m + k];", "acc += w * y[q * m + (k + 1) % m];"),
    "missing_1_over_N": ("z[r] *= K[r] * invN;", "z[r] *= K[r];"),
    "nyquist_sum_not_mean": ("K[lin] = acc / cnt;", "K[lin] = acc;"),
    "reciprocal_transposed": ("2.0 * ORACLE_PI * inv[c * 3 + k]", "2.0 * ORACLE_PI * inv[k * 3 + c]"),
    "kernel_not_squared": ("return 4.0 * ORACLE_PI / g2;", "return 4.0 * ORACLE_PI / sqrt(g2);"),
    "trunc_g0_dropped": ("g2 == 0.0 ? 2.0 * ORACLE_PI * rc * rc :", "g2 == 0.0 ? 0.0 :"),
    "trunc_radius_doubled": ("(1.0 - cos(sqrt(g2) * rc))", "(1.0 - cos(sqrt(g2) * 2.0 * rc))"),
    "trunc_cos_sign": ("(1.0 - cos(sqrt(g2) * rc))", "(1.0 + cos(sqrt(g2) * rc))"),
    "inscribed_radius_2pi": ("if (ORACLE_PI / b < r) r = ORACLE_PI / b;", "if (ORACLE_PI / b < r) r = 2.0 * ORACLE_PI / b;"),
    "diagonal_pair_dropped": (
        "if (mask && !mask[(long)i * norb + j]) continue;",
        "if (j == i || (mask && !mask[(long)i * norb + j])) continue;",
    ),
    "w_uses_phi_i": ("Wi[r] += v[r] * pj[r];", "Wi[r] += v[r] * phi[(long)i * npts + r];"),
    "M_sign": ("M_raw[(long)k * n + l] = -dV * s;", "M_raw[(long)k * n + l] = dV * s;"),
    "M_missing_dV": ("M_raw[(long)k * n + l] = -dV * s;", "M_raw[(long)k * n + l] = -s;"),
    "xi_transposed_L": (
        "s -= L[(long)k * n + l] * xi[(long)l * npts + r];",
        "s -= L[(long)l * n + k] * xi[(long)l * npts + r];",
    ),
    "apply_sign": ("out[(long)c * npts + r] = -s;", "out[(long)c * npts + r] = s;"),
    "apply_missing_dV": ("C[(long)k * m + c] = dV * s;", "C[(long)k * m + c] = s;"),
    "energy_factor": ("return 0.5 * spin_factor * t;", "return spin_factor * t;"),
    "screen_strict": ("(s >= rho_cut)", "(s > rho_cut)"),
    "screen_no_abs": ("s += fabs(a[r] * b[r]);", "s += a[r] * b[r];"),
    "screen_diag_not_kept": ("(i == j) || (rho_cut <= 0.0)", "(rho_cut <= 0.0)"),
    "scdm_argmin": ("if (d[r] > d[best]) best = r;", "if (d[r] < d[best]) best = r;"),
    "scdm_no_orthogonalisation": ("for (int pass = 0; pass < 2; ++pass)", "for (int pass = 0; pass < 0; ++pass)"),
    "scdm_no_downdate": ("d[r] -= p * p;", "d[r] -= 0.0 * p;"),
}


@pytest.fixture(scope="module")
def battery_inputs():
    rng = np.random.default_rng(7)
    grid = (12, 14, 15)
    phi, prims, D = gaussian_orbitals(grid, TRICLINIC, 3, 2, rng)
    coeffs = cf.prim_pair_coefficients(prims, TRICLINIC, grid, nalias=2, nimg=2)
    E = cf.pair_energies(D, coeffs, TRICLINIC, grid)
    rng2 = np.random.default_rng(1)
    z = rng2.standard_normal((6, 10, 15)) + 1j * rng2.standard_normal((6, 10, 15))
    n = 48
    x = np.arange(n) * 16.0 / n
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    iso_phi = (2 / np.pi) ** 0.75 * np.exp(-((X - 8.0) ** 2 + (Y - 8.0) ** 2 + (Z - 8.0) ** 2))
    import scipy.linalg

    A = np.random.default_rng(8).standard_normal((10, 200))
    P = list(scipy.linalg.qr(A, pivoting=True, mode="economic")[2][:10])
    return dict(grid=grid, phi=phi, E=E, z=z, iso_phi=iso_phi, iso_ref=2 * np.sqrt(1 / np.pi), scdm_A=A,
                scdm_P=P)


def _naive(z, sign):
    out = z
    for axis, n in enumerate(z.shape):
        k = np.arange(n)
        F = np.exp(sign * 2j * np.pi * np.outer(k, k) / n)
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, axis, 0), axes=(1, 0)), 0, axis)
    return out


def run_battery(orc, inp):
    """Returns the names of the failed checks."""
    failed = []
    z = inp["z"]
    for sign in (-1, 1):
        ref = _naive(z, sign)
        if not np.abs(orc.fft3d(z, sign) - ref).max() <= 1e-12 * np.abs(ref).max():
            failed.append(f"dft{sign}")
    phi, E = inp["phi"], inp["E"]
    dV = abs(np.linalg.det(TRICLINIC)) / np.prod(inp["grid"])
    r = orc.ace_build(phi, TRICLINIC, 0.0, 2.0)
    ref = -E.sum()
    if not abs(r["E_x"] - ref) <= 1e-12 * abs(ref):
        failed.append("closed_form_E_x")
    if r["status"] != 0:
        failed.append("cholesky")
    else:
        K = orc.ace_apply(r["xi"], phi, dV)
        if not np.abs(K + r["W"]).max() <= 1e-12 * np.abs(r["W"]).max():
            failed.append("K_phi_equals_minus_W")
        if not np.linalg.norm(r["M_raw"] - r["M_raw"].T) <= 1e-14 * np.linalg.norm(r["M_raw"]):
            failed.append("M_symmetric")
    flat = phi.reshape(3, -1)
    Oref = np.array([[dV * np.sum(np.abs(flat[i] * flat[j])) for j in range(3)] for i in range(3)])
    O, _ = orc.screen(phi, TRICLINIC, 0.0)
    if not np.abs(O - Oref).max() <= 1e-13 * Oref.max():
        failed.append("screen_values")
    cut = O[0, 1]
    _, mask = orc.screen(phi, TRICLINIC, cut)
    want = (O >= cut) | np.eye(3, dtype=bool)
    if not np.array_equal(mask, want):
        failed.append("screen_mask")
    big = 10 * O.max()
    _, mask = orc.screen(phi, TRICLINIC, big)
    if not np.array_equal(mask, np.eye(3, dtype=bool)):
        failed.append("screen_diagonal")
    # SCDM selection: the greedy column-pivoted QR of LAPACK on a random matrix
    if list(orc.scdm_select(inp["scdm_A"])) != inp["scdm_P"]:
        failed.append("scdm_pivots")
    # isolated-cell kernel: closed-form self-energy of a Gaussian density (default cut-off)
    g = inp["iso_phi"]
    e = orc.pair_energy(g, g, np.eye(3) * 16.0, orc.TRUNCATED, 0.0)
    if not abs(e - inp["iso_ref"]) <= 1e-9 * inp["iso_ref"]:
        failed.append("truncated_self_energy")
    return failed


def _compile(tmp_path, name, text):
    import oracle

    src = tmp_path / f"{name}.c"
    src.write_text(text)
    return oracle.bind(oracle.compile_source(str(src), str(tmp_path / f"lib{name}.so")))


def test_unmutated_passes_battery(tmp_path, battery_inputs):
    import oracle

    shutil.copy(SRC, tmp_path / "orig.c")
    lib = _compile(tmp_path, "orig", open(SRC).read())
    with oracle.using(lib):
        assert run_battery(oracle, battery_inputs) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, battery_inputs, name):
    import oracle

    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not unique"
    lib = _compile(tmp_path, name, text.replace(old, new))
    with oracle.using(lib):
        failed = run_battery(oracle, battery_inputs)
    assert failed, f"planted mistake '{name}' passed every pin"
