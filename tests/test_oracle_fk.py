"""Pins of the oracle's plane-wave f-k migrations (Sec. II-B-3, the two f-k
migrations the paper evaluates).

fk_migrate maps with the exact delay model of Eq. (1) with a plane-wave
transmit: point scatterers must image at their true position, within half an
element pitch laterally (the native grid has one column per element) and a
quarter wavelength axially, unsteered and steered.  fk_stolt is Stolt's
migration of the exploding-reflector model fitted to the plane-wave two-way
time (an approximation away from the scatterer's lateral position): within
one pitch laterally and a quarter wavelength axially.  Both are checked for
degree-1 homogeneity and for compounding (two angles' spectra add), and
planted mistakes in a copy of each function's source must each fail a pin.
"""
import inspect
import math
import textwrap

import numpy as np
import pytest

import oracle
import synth

ACQ = synth.Acquisition(n_elements=64, n_samples=1024, nx=64, nz=64)
POINTS = ((0.0, 15e-3), (3e-3, 22e-3), (-4.5e-3, 10e-3), (6.1e-3, 30e-3))


def _peak(img, acq):
    i, m = np.unravel_index(np.argmax(img), img.shape)
    return (i - 0.5 * (acq.n_elements - 1)) * acq.pitch_m, m * acq.c_mps / (2 * acq.fs_hz)


def _point_pins(fk, lateral=0.5):
    lam = ACQ.c_mps / ACQ.f0_hz
    for deg in (0.0, 10.0, -10.0):
        acq = ACQ.with_(angles_deg=(deg,))
        for xp, zp in POINTS:
            rf, _ = synth.point_frame(acq, xp, zp)
            img = fk(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
            assert img.shape == (acq.n_elements, acq.n_samples)
            xe, ze = _peak(img, acq)
            assert abs(xe - xp) <= lateral * acq.pitch_m + 1e-9, (deg, xp, zp, xe)
            assert abs(ze - zp) <= lam / 4, (deg, xp, zp, ze)


def _compounding_pin(fk, lateral=0.5):
    """Two angles: the image of both records is the magnitude of the sum of the
    complex images; at a point target seen at both angles the peak stays put
    and grows over either single-angle peak."""
    acq = ACQ.with_(angles_deg=(-8.0, 8.0))
    rf, _ = synth.point_frame(acq, 2e-3, 18e-3)
    both = fk(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    one = [fk(rf[a:a + 1], acq.pitch_m, acq.angles_rad[a:a + 1], acq.fs_hz, acq.c_mps)
           for a in range(2)]
    xe, ze = _peak(both, acq)
    assert abs(xe - 2e-3) <= lateral * acq.pitch_m + 1e-9
    assert abs(ze - 18e-3) <= acq.c_mps / acq.f0_hz / 4
    assert both.max() > 1.5 * max(o.max() for o in one)


def test_point_targets_image_in_place():
    _point_pins(oracle.fk_migrate)


def test_compounding_adds_the_angles_coherently():
    _compounding_pin(oracle.fk_migrate)


def test_stolt_point_targets_image_in_place():
    _point_pins(oracle.fk_stolt, lateral=1.0)


def test_stolt_compounding_adds_the_angles_coherently():
    _compounding_pin(oracle.fk_stolt, lateral=1.0)


@pytest.mark.parametrize("fk", [oracle.fk_migrate, oracle.fk_stolt], ids=["lu", "stolt"])
def test_homogeneous_and_zero(fk):
    acq = ACQ.with_(angles_deg=(5.0,))
    rf, _ = synth.speckle_points_frame(acq)
    rf = (rf // 4).astype(np.int16)
    a = fk(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    b = fk((3 * rf).astype(np.int16), acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    np.testing.assert_allclose(b, 3 * a, rtol=1e-9, atol=1e-9 * a.max())
    z = fk(np.zeros_like(rf), acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    assert np.all(z == 0)


def test_stolt_unsteered_reduces_to_the_exploding_reflector_at_half_speed():
    """At 0 deg the fit gives beta = sqrt(2): the exploding reflector of the
    plane wave's two-way time moves at c / sqrt(2), and Stolt's temporal bin of
    (X, Q) is sqrt(2 X^2 + Q^2), the exact mapping's (X^2 + Q^2) / Q to second
    order in X / Q; on the axis (X = 0) both are Q."""
    acq = ACQ.with_(angles_deg=(0.0,))
    rf, _ = synth.point_frame(acq, 0.0, 20e-3)
    a = oracle.fk_stolt(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    b = oracle.fk_migrate(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    # the same focus (column, and depth within one sample), and the centre
    # column's axial profiles agree closely
    (xa, za), (xb, zb) = (np.unravel_index(np.argmax(m), m.shape) for m in (a, b))
    assert xa == xb and abs(int(za) - int(zb)) <= 1, ((xa, za), (xb, zb))
    col = int(np.argmax(a.max(axis=1)))
    pa, pb = a[col] / a.max(), b[col] / b.max()
    assert np.max(np.abs(pa - pb)) < 0.2


MUTANTS = [
    ("lateral delay compensated with the wrong sign", "D = D * np.exp(1j * np.pi",
     "D = D * np.exp(-1j * np.pi"),
    ("mapping without the steering term", "den = XX * st + QQ * ct", "den = QQ * ct"),
    ("mapping off by a factor 2", "pos = num / den", "pos = 0.5 * num / den"),
    ("depth spacing of a one-way path", "dz = c / (2.0 * fs)", "dz = c / fs"),
    ("interpolation weights swapped", "val = (1 - al) * D[cols, i0] + al * D[cols, i1]",
     "val = al * D[cols, i0] + (1 - al) * D[cols, i1]"),
    ("lateral wavenumbers of a one-sample pitch", "X = ms * (nt * dz / (nk * pitch))",
     "X = ms * (nt * dz / nk)"),
]


STOLT_MUTANTS = [
    ("shear with the wrong sign", "Qp = (QQ - st * XX) / bet", "Qp = (QQ + st * XX) / bet"),
    ("no shear", "Qp = (QQ - st * XX) / bet", "Qp = QQ / bet"),
    ("depth scale of the unsteered fit", "bet = np.sqrt(1.0 + ct - 0.5 * st * st)",
     "bet = np.sqrt(2.0)"),
    ("velocity fit with the steering term's sign flipped", "bet = np.sqrt(1.0 + ct - 0.5 * st * st)",
     "bet = np.sqrt(1.0 + ct + st * st)"),
    ("temporal bin without the 2 / beta", "pos = (2.0 / bet) * rad", "pos = rad"),
    ("lateral delay compensated with the wrong sign", "D = D * np.exp(1j * np.pi",
     "D = D * np.exp(-1j * np.pi"),
    ("interpolation weights swapped", "val = (1 - al) * D[cols, i0] + al * D[cols, i1]",
     "val = al * D[cols, i0] + (1 - al) * D[cols, i1]"),
    ("depth spacing of a one-way path", "dz = c / (2.0 * fs)", "dz = c / fs"),
]


def _mutant_caught(fn, name, old, new, lateral):
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, name
    ns = {"np": np, "fk_sizes": oracle.fk_sizes}
    exec(src.replace(old, new), ns)
    mutated = ns[fn.__name__]
    for pin in (_point_pins, _compounding_pin):
        try:
            with np.errstate(all="ignore"):
                pin(mutated, lateral=lateral)
        except (AssertionError, IndexError, ValueError):
            return True
    return False


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    assert _mutant_caught(oracle.fk_migrate, name, old, new, 0.5), \
        "mutant '%s' survived every pin" % name


@pytest.mark.parametrize("name,old,new", STOLT_MUTANTS, ids=[m[0] for m in STOLT_MUTANTS])
def test_stolt_mutant_is_caught(name, old, new):
    assert _mutant_caught(oracle.fk_stolt, name, old, new, 1.0), \
        "mutant '%s' survived every pin" % name
