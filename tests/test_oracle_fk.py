"""Pins of the oracle's plane-wave f-k migration (Sec. II-B-3, the f-k
migrations the paper evaluates; the mapping is the exact one of the delay
model of Eq. (1) with a plane-wave transmit).

Point scatterers must image at their true position: within half an element
pitch laterally (the native grid has one column per element) and a quarter
wavelength axially, unsteered and steered.  The function is also checked for
degree-1 homogeneity and for compounding (two angles' spectra add), and six
planted mistakes in a copy of its source must each fail a pin.
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


def _point_pins(fk):
    lam = ACQ.c_mps / ACQ.f0_hz
    for deg in (0.0, 10.0, -10.0):
        acq = ACQ.with_(angles_deg=(deg,))
        for xp, zp in POINTS:
            rf, _ = synth.point_frame(acq, xp, zp)
            img = fk(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
            assert img.shape == (acq.n_elements, acq.n_samples)
            xe, ze = _peak(img, acq)
            assert abs(xe - xp) <= 0.5 * acq.pitch_m + 1e-9, (deg, xp, zp, xe)
            assert abs(ze - zp) <= lam / 4, (deg, xp, zp, ze)


def _compounding_pin(fk):
    """Two angles: the image of both records is the magnitude of the sum of the
    complex images; at a point target seen at both angles the peak stays put
    and grows over either single-angle peak."""
    acq = ACQ.with_(angles_deg=(-8.0, 8.0))
    rf, _ = synth.point_frame(acq, 2e-3, 18e-3)
    both = fk(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    one = [fk(rf[a:a + 1], acq.pitch_m, acq.angles_rad[a:a + 1], acq.fs_hz, acq.c_mps)
           for a in range(2)]
    xe, ze = _peak(both, acq)
    assert abs(xe - 2e-3) <= 0.5 * acq.pitch_m + 1e-9 and abs(ze - 18e-3) <= acq.c_mps / acq.f0_hz / 4
    assert both.max() > 1.5 * max(o.max() for o in one)


def test_point_targets_image_in_place():
    _point_pins(oracle.fk_migrate)


def test_compounding_adds_the_angles_coherently():
    _compounding_pin(oracle.fk_migrate)


def test_homogeneous_and_zero():
    acq = ACQ.with_(angles_deg=(5.0,))
    rf, _ = synth.speckle_points_frame(acq)
    rf = (rf // 4).astype(np.int16)
    a = oracle.fk_migrate(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    b = oracle.fk_migrate((3 * rf).astype(np.int16), acq.pitch_m, acq.angles_rad, acq.fs_hz,
                          acq.c_mps)
    np.testing.assert_allclose(b, 3 * a, rtol=1e-9, atol=1e-9 * a.max())
    z = oracle.fk_migrate(np.zeros_like(rf), acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    assert np.all(z == 0)


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


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new):
    src = textwrap.dedent(inspect.getsource(oracle.fk_migrate))
    assert src.count(old) == 1, name
    ns = {"np": np, "fk_sizes": oracle.fk_sizes}
    exec(src.replace(old, new), ns)
    mutated = ns["fk_migrate"]
    caught = False
    for pin in (_point_pins, _compounding_pin):
        try:
            with np.errstate(all="ignore"):
                pin(mutated)
        except (AssertionError, IndexError, ValueError):
            caught = True
            break
    assert caught, "mutant '%s' survived every pin" % name
