"""The oracle's pins must catch plausible mistakes.

Each mutant plants one mistake in a copy of the oracle's C source (a dropped
term, a wrong sign, a wrong index, a transposed operand, a wrong bound),
builds it on the CPU, routes the oracle module through it and re-runs the
pins: at least one pin has to fail for every mutant.
"""
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "bf_oracle.c")

MUTANTS = [
    ("transmit leg sign", "double tx = xp * st + zp * ct;", "double tx = -xp * st + zp * ct;"),
    ("transmit leg dropped", "double tx = xp * st + zp * ct;", "double tx = zp * ct;"),
    ("monostatic delay", "double n = (tx + rx) * kappa;", "double n = (rx + rx) * kappa;"),
    ("lateral offset transposed", "double dx = xp - xi;", "double dx = xp - zp;"),
    ("depth term dropped", "sqrt(dx * dx + zp * zp)", "sqrt(dx * dx + zp)"),
    ("interpolation reads one sample", "alpha * (double)u[kk + 1]", "alpha * (double)u[kk]"),
    ("interpolation weights swapped",
     "(1.0 - alpha) * (double)u[kk] + alpha * (double)u[kk + 1]",
     "alpha * (double)u[kk] + (1.0 - alpha) * (double)u[kk + 1]"),
    ("aperture uses F instead of 2F", "zp / (2.0 * fnum)", "zp / fnum"),
    ("aperture exclusive", "fabs(xp - xi) <= zp", "fabs(xp - xi) < zp"),
    ("record bound off by one", "k <= (double)(ns - 2)", "k <= (double)(ns - 3)"),
    ("DMAS diagonal sign", "0.5 * (t1 * t1 - t2)", "0.5 * (t1 * t1 + t2)"),
    ("DMAS without square root", "double s = signed_sqrt(v);", "double s = v;"),
    ("DMAS sign lost", "return -sqrt(-v);", "return sqrt(-v);"),
    ("CF without channel count", "(double)m * su2_tot", "su2_tot"),
    ("angle index frozen", "st[a], ct[a]", "st[0], ct[0]"),
    ("channel record index", "((size_t)a * ne + i) * (size_t)ns", "((size_t)a * ne) * (size_t)ns"),
    ("grid spacing", "(hi - lo) / (double)(n - 1)", "(hi - lo) / (double)n"),
    ("compounding keeps last angle", "s1_tot += s1;", "s1_tot = s1;"),
    ("pDAS power instead of root", "yt += signed_pow(v, 1.0 / p);", "yt += signed_pow(v, p);"),
    ("pDAS power dropped", "y += signed_pow(yt, p);", "y += yt;"),
    ("pDAS root loses the sign", "return -pow(-v, e);", "return pow(-v, e);"),
    ("pDAS keeps the last angle", "y += signed_pow(yt, p);", "y = signed_pow(yt, p);"),
    ("IQ carrier restored with the wrong sign", "double cr = cos(ph), ci = sin(ph);",
     "double cr = cos(ph), ci = -sin(ph);"),
    ("IQ interpolation weights swapped",
     "double br = (1.0 - alpha) * iq_re[o] + alpha * iq_re[o + 1];",
     "double br = alpha * iq_re[o] + (1.0 - alpha) * iq_re[o + 1];"),
    ("BB-DMAS without the square root", "double w = 1.0 / sqrt(mag);", "double w = 1.0;"),
    ("BB-DMAS without 1/M", "double ur = tr / (double)m, ui = ti / (double)m;",
     "double ur = tr, ui = ti;"),
    ("BB-DMAS squares the magnitude", "y2r += ur * ur - ui * ui;", "y2r += ur * ur + ui * ui;"),
]


def _pins_pass(golden_dir):
    checks = [
        lambda: pins.test_geometry_cases_match_hand_derivations(golden_dir),
        lambda: pins.test_aperture_counts_match_hand_derivations(golden_dir),
        lambda: pins.test_constant_record_closed_forms(golden_dir),
        pins.test_linear_interpolation_exact_on_a_ramp,
        lambda: pins.test_grid_coordinates_on_a_ramp(golden_dir),
        pins.test_dmas_identity_against_pairwise_brute_force,
        pins.test_das_is_linear_and_cf_bounded,
        lambda: pins.test_point_scatterer_images_within_quarter_wavelength(10.0, "das"),
        lambda: pins.test_pdas_constant_record_closed_form(golden_dir),
        pins.test_pdas_p1_is_das_and_single_channel_is_the_sample,
        pins.test_pdas_homogeneous_odd_and_brute_force,
        lambda: pins.test_iq_das_and_bb_dmas_hand_derived_case(golden_dir),
        pins.test_iq_combiners_against_a_numpy_evaluation,
        pins.test_iq_images_are_homogeneous_and_single_channel_bb_dmas_is_the_magnitude,
    ]
    for check in checks:
        try:
            check()
        except AssertionError:
            return False
    return True


def test_unmutated_oracle_passes_pins(golden_dir):
    assert _pins_pass(golden_dir)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, golden_dir, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    str(mutated), "-o", str(lib), "-lm"], check=True)
    with oracle.use_library(str(lib)):
        assert not _pins_pass(golden_dir), "mutant '%s' survived every pin" % name
