"""Pins of the FP64 oracle to values fixed by the paper's definitions and by mathematics.

Nothing here compares the oracle with itself: the expected values are hand
derivations (tests/golden), closed forms, library routines (scipy's Hilbert
transform), brute force on tiny apertures, invariants (linearity, scale,
Cauchy-Schwarz) and an end-to-end physical check (a point scatterer must image
within a quarter wavelength of where it was simulated).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth


def _load(golden_dir, name):
    with open(os.path.join(golden_dir, name)) as f:
        return json.load(f)


def _single_pixel_grid(x, z):
    return (1, 1, x, x, z, z)


# ---------------------------------------------------------------- geometry --

def test_geometry_cases_match_hand_derivations(golden_dir):
    spec = _load(golden_dir, "geometry_cases.json")
    rng = np.random.default_rng(1)
    for case in spec["cases"]:
        xe = np.array(case["x_elem_m"])
        th = np.array(case["angles_rad"])
        rf = rng.integers(-30000, 30000, (len(th), len(xe), 256)).astype(np.int16)
        x, z = case["pixel_m"]
        out = oracle.beamform(rf, xe, th, _single_pixel_grid(x, z), case["fs_hz"], case["c_mps"],
                              case["f_number"])
        want = sum(w * float(rf[a, i, k]) for a, i, k, w in case["expect"])
        got = float(out["das"][0, 0])
        assert got == pytest.approx(want, rel=1e-9, abs=1e-7), case["name"]


def test_grid_coordinates_on_a_ramp(golden_dir):
    """Inclusive linspace pixel grids: a ramp record returns each pixel's delay."""
    spec = _load(golden_dir, "geometry_cases.json")
    rf = np.arange(512, dtype=np.int16)[None, None, :]
    for case in spec["grid_cases"]:
        out = oracle.beamform(rf, case["x_elem_m"], [0.0], tuple(case["grid"]), case["fs_hz"],
                              case["c_mps"], case["f_number"])
        np.testing.assert_allclose(out["das"], case["ramp_das"], atol=1e-9, err_msg=case["name"])


def test_aperture_counts_match_hand_derivations(golden_dir):
    spec = _load(golden_dir, "aperture_counts.json")
    n = spec["n_elements"]
    xe = (np.arange(n) - 0.5 * (n - 1)) * spec["pitch_m"]
    rf = np.full((1, n, 4096), 1000, np.int16)
    for case in spec["cases"]:
        x, z = case["pixel_m"]
        v, act, rec = oracle.delayed_samples(rf, xe, [0.0], _single_pixel_grid(x, z), 0, 0, 20e6,
                                             1540.0, spec["f_number"])
        idx = np.nonzero(act[0])[0]
        assert len(idx) == case["count"]
        assert (idx.min(), idx.max()) == (case["first"], case["last"])
        assert np.all(idx == np.arange(case["first"], case["last"] + 1))
        # constant record -> every active in-record channel reads exactly 1000
        assert np.all(v[0][act[0]] == 1000.0)
    rb = spec["record_bound"]
    x, z = rb["pixel_m"]
    rf = np.full((1, n, rb["n_samples"]), 1000, np.int16)
    v, act, rec = oracle.delayed_samples(rf, xe, [0.0], _single_pixel_grid(x, z), 0, 0, rb["fs_hz"],
                                         rb["c_mps"], spec["f_number"])
    idx = np.nonzero(rec[0])[0]
    assert len(idx) == rb["count"] and (idx.min(), idx.max()) == (rb["first"], rb["last"])
    assert np.all(v[0][act[0] & ~rec[0]] == 0.0)
    tie = spec["edge_tie"]
    x, z = tie["pixel_m"]
    rf = np.full((1, 3, 256), 5, np.int16)
    v, act, rec = oracle.delayed_samples(rf, tie["x_elem_m"], [0.0], _single_pixel_grid(x, z), 0, 0,
                                         20e6, 1540.0, tie["f_number"])
    assert list(act[0]) == tie["active"]


def test_constant_record_closed_forms(golden_dir):
    """u = c everywhere: DAS = c*M_in, DMAS = |c|*M_in(M_in-1)/2, CF = c*M_in^2/M."""
    spec = _load(golden_dir, "aperture_counts.json")
    n = spec["n_elements"]
    xe = (np.arange(n) - 0.5 * (n - 1)) * spec["pitch_m"]
    rb = spec["record_bound"]
    x, z = rb["pixel_m"]
    rf = np.full((1, n, rb["n_samples"]), 1000, np.int16)
    out = oracle.beamform(rf, xe, [0.0], _single_pixel_grid(x, z), rb["fs_hz"], rb["c_mps"],
                          spec["f_number"])
    m_in, m_ap = rb["count"], spec["cases"][0]["count"]  # 14 in record of the 20 in the aperture
    assert out["das"][0, 0] == pytest.approx(1000.0 * m_in, rel=1e-12)
    assert out["dmas"][0, 0] == pytest.approx(1000.0 * m_in * (m_in - 1) / 2, rel=1e-12)
    assert out["cf"][0, 0] == pytest.approx(1000.0 * m_in ** 2 / m_ap, rel=1e-12)
    assert out["m"][0, 0] == m_ap
    # three compounded angles, long record: everything in range
    rf = np.full((3, n, 4096), -7, np.int16)
    th = np.deg2rad([-5.0, 0.0, 5.0])
    out = oracle.beamform(rf, xe, th, _single_pixel_grid(x, z), 20e6, 1540.0, 1.5)
    assert out["das"][0, 0] == pytest.approx(-7.0 * 3 * m_ap, rel=1e-12)
    # s_i s_j = (-sqrt 7)(-sqrt 7) = +7: DMAS keeps no sign of a uniform record
    assert out["dmas"][0, 0] == pytest.approx(7.0 * 3 * m_ap * (m_ap - 1) / 2, rel=1e-12)
    assert out["cf"][0, 0] == pytest.approx(-7.0 * 3 * m_ap, rel=1e-12)
    assert out["m"][0, 0] == 3 * m_ap


def test_linear_interpolation_exact_on_a_ramp():
    """u_i[n] = n: linear interpolation returns the fractional delay itself, so
    DAS of one element equals the delay n, which the 3-4-5 geometry fixes."""
    rf = np.arange(512, dtype=np.int16)[None, None, :]
    # 3-4-5 geometry with c = 1600, fs = 20 MHz: n = 112.5 (unsteered)
    out = oracle.beamform(rf, [0.0], [0.0], _single_pixel_grid(0.003, 0.004), 20e6, 1600.0, 0.5)
    assert out["das"][0, 0] == pytest.approx(112.5, abs=1e-9)
    # z shifted by 1 um: n = 12500 * (4.001e-3 + sqrt(9e-6 + 4.001e-3^2)), d n / d z = kappa (1 + z/r)
    out = oracle.beamform(rf, [0.0], [0.0], _single_pixel_grid(0.003, 0.004001), 20e6, 1600.0, 0.5)
    assert out["das"][0, 0] == pytest.approx(112.5 + 12500 * 1e-6 * (1 + 0.8), abs=2e-6)


# ------------------------------------------------------------- combiners --

def test_dmas_identity_against_pairwise_brute_force():
    """(sum s)^2 - sum s^2 = 2 sum_{i<j} s_i s_j, checked by a double loop."""
    rng = np.random.default_rng(7)
    n = 6
    xe = (np.arange(n) - 2.5) * 0.3e-3
    rf = rng.integers(-20000, 20000, (2, n, 512)).astype(np.int16)
    th = np.deg2rad([-4.0, 6.0])
    grid = (5, 7, -0.6e-3, 0.6e-3, 3e-3, 6e-3)
    out = oracle.beamform(rf, xe, th, grid, 20e6, 1540.0, 0.7)
    for ix in range(5):
        for iz in range(7):
            v, act, _ = oracle.delayed_samples(rf, xe, th, grid, ix, iz, 20e6, 1540.0, 0.7)
            s = np.sign(v) * np.sqrt(np.abs(v))
            brute, scale, das = 0.0, 0.0, 0.0
            for a in range(2):
                for i in range(n):
                    if not act[a, i]:
                        continue
                    das += v[a, i]
                    scale += s[a, i] ** 2
                    for j in range(i + 1, n):
                        if act[a, j]:
                            brute += s[a, i] * s[a, j]
            assert abs(out["dmas"][ix, iz] - brute) <= 1e-12 * max(scale, 1.0)
            assert out["das"][ix, iz] == pytest.approx(das, rel=1e-12, abs=1e-9)
    assert np.any(out["m"] > 1)


def test_das_is_linear_and_cf_bounded():
    rng = np.random.default_rng(11)
    acq = synth.SPECKLE_POINTS_128.with_(nx=9, nz=11, n_samples=1024)
    xe = acq.x_elements()
    r1 = rng.integers(-1000, 1000, (1, 64, 1024)).astype(np.int16)
    r2 = rng.integers(-1000, 1000, (1, 64, 1024)).astype(np.int16)
    r3 = (2 * r1.astype(np.int32) - 3 * r2.astype(np.int32)).astype(np.int16)
    grid = (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)
    o1, o2, o3 = (oracle.beamform(r, xe, [0.0], grid, acq.fs_hz, acq.c_mps, 1.5) for r in (r1, r2, r3))
    np.testing.assert_allclose(o3["das"], 2 * o1["das"] - 3 * o2["das"], rtol=1e-10, atol=1e-7)
    # CF-DAS = DAS * CF with CF = (sum v)^2 / (M sum v^2) in [0, 1] (Cauchy-Schwarz)
    ratio = o1["cf"] / np.where(o1["das"] == 0, 1, o1["das"])
    assert np.all(ratio >= -1e-15) and np.all(ratio <= 1 + 1e-12)
    # DMAS is homogeneous of degree 1 in the data; CF-DAS too
    o4 = oracle.beamform(4 * r1, xe, [0.0], grid, acq.fs_hz, acq.c_mps, 1.5)
    np.testing.assert_allclose(o4["dmas"], 4 * o1["dmas"], rtol=1e-10, atol=1e-6)
    np.testing.assert_allclose(o4["cf"], 4 * o1["cf"], rtol=1e-10, atol=1e-6)


def test_sign_of_zero_and_empty_aperture():
    # pixel at z = 0: aperture half width 0 -> only an element exactly below it is active
    rf = np.zeros((1, 3, 64), np.int16)
    out = oracle.beamform(rf, [-1e-3, 0.0, 1e-3], [0.0], _single_pixel_grid(0.0, 0.0), 20e6,
                          1540.0, 1.5)
    assert out["m"][0, 0] == 1 and out["das"][0, 0] == 0.0 and out["dmas"][0, 0] == 0.0
    assert out["cf"][0, 0] == 0.0  # 0/0 -> 0
    out = oracle.beamform(rf[:, :1], [5e-3], [0.0], _single_pixel_grid(0.0, 1e-3), 20e6, 1540.0,
                          1.5)
    assert out["m"][0, 0] == 0 and out["cf"][0, 0] == 0.0


# ------------------------------------------------------ envelope and log --

def test_envelope_matches_scipy_hilbert():
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(3)
    for L in (64, 77, 256, 1023):
        y = rng.normal(size=(3, L))
        np.testing.assert_allclose(oracle.envelope(y), np.abs(signal.hilbert(y, axis=-1)),
                                   rtol=1e-12, atol=1e-12)


def test_envelope_of_bin_centred_cosines():
    L, dz, c, f0 = 256, 20e-6, 1540.0, 5e6
    n = np.arange(L)
    # bin k is the RF frequency k c / (2 L dz) = k * 150390.6 Hz; pass band [f0, 3 f0] = bins 34..99
    inside = 3.0 * np.cos(2 * np.pi * 66 * n / L + 0.4)
    below = 2.0 * np.cos(2 * np.pi * 20 * n / L)
    above = 2.0 * np.cos(2 * np.pi * 110 * n / L)
    np.testing.assert_allclose(oracle.envelope(inside), 3.0, atol=1e-12)
    np.testing.assert_allclose(oracle.envelope(below), 2.0, atol=1e-12)
    env = oracle.envelope(inside + below + above + 5.0, bandpass=True, dz=dz, c=c, f0=f0)
    np.testing.assert_allclose(env, 3.0, atol=1e-12)
    assert np.max(oracle.envelope(below + 1.0, bandpass=True, dz=dz, c=c, f0=f0)) < 1e-12
    # band edges: bin 34 (5.11 MHz) passes, bin 33 (4.96 MHz) is stopped
    m = oracle.spectral_mask(L, bandpass=True, dz=dz, c=c, f0=f0)
    assert m[33] == 0 and m[34] == 2 and m[99] == 2 and m[100] == 0 and m[0] == 0


def test_log_compression_closed_form():
    env = np.array([2.0, 0.2, 0.02, 0.0, 2e-5, 2.0 * 10 ** (-3.5)])
    np.testing.assert_allclose(oracle.log_compress(env), [0, -20, -40, -70, -70, -70], atol=1e-12)
    np.testing.assert_allclose(oracle.log_compress(np.zeros(4)), -70.0)


# ------------------------------------------------------------------ metrics --

def test_fwhm_of_triangle_and_gaussian():
    r = 10 ** (-6 / 20)
    x = np.arange(-200, 201) * 0.01  # spacing 0.01
    tri = np.maximum(0.0, 1 - np.abs(x) / 1.0)
    assert oracle.fwhm(tri, 0.01) == pytest.approx(2 * (1 - r), abs=1e-12)
    s = 0.3
    g = np.exp(-x * x / (2 * s * s))
    assert oracle.fwhm(g, 0.01) == pytest.approx(2 * s * math.sqrt(-2 * math.log(r)), rel=2e-4)
    assert math.isnan(oracle.fwhm(np.ones(10)))


def test_contrast_metrics_closed_form():
    env = np.zeros(400)
    inside = np.zeros(400, bool)
    outside = np.zeros(400, bool)
    inside[:100] = True
    outside[200:400] = True
    env[:100] = 0.1 + 0.02 * np.where(np.arange(100) % 2 == 0, 1, -1)
    env[200:400] = 1.0 + 0.5 * np.where(np.arange(200) % 2 == 0, 1, -1)
    m = oracle.contrast(env, inside, outside)
    assert m["cr_db"] == pytest.approx(20 * math.log10(0.1), abs=1e-12)
    assert m["cnr"] == pytest.approx(0.9 / math.sqrt((0.02 ** 2 + 0.5 ** 2) / 2), rel=1e-12)
    assert m["cnr_printed"] == pytest.approx(-0.9 / math.sqrt(0.02 ** 2 + 0.5 ** 2 / 2), rel=1e-12)


def test_cyst_regions_geometry():
    grid = (201, 201, -5e-3, 5e-3, 15e-3, 25e-3)  # 50 um pixels
    ins, out = oracle.cyst_regions(grid, 0.0, 20e-3, 1e-3)
    xs, zs = oracle.grid_coords(grid)
    X, Z = np.meshgrid(xs, zs, indexing="ij")
    # inner disk of radius 0.8 mm centred on the cyst (boundary pixels may round either way)
    assert abs(X[ins].mean()) < 1e-5 and abs(Z[ins].mean() - 20e-3) < 1e-5
    assert abs(ins.sum() - math.pi * 0.8 ** 2 / 0.05 ** 2) < 0.05 * ins.sum()
    # two disks of the same size at the same depth, centred 2.5 mm either side
    right, left = out & (X > 0), out & (X < 0)
    assert abs(X[right].mean() - 2.5e-3) < 1e-5 and abs(X[left].mean() + 2.5e-3) < 1e-5
    assert abs(Z[right].mean() - 20e-3) < 1e-5 and abs(right.sum() - ins.sum()) <= 4
    assert not np.any(ins & out)


# ------------------------------------------------- end-to-end localisation --

@pytest.mark.parametrize("deg", [0.0, 10.0, -10.0])
@pytest.mark.parametrize("mode", ["das", "dmas"])
def test_point_scatterer_images_within_quarter_wavelength(deg, mode):
    acq = synth.Acquisition(angles_deg=(deg,), n_samples=1024)
    xs, zs = 1.3e-3, 20.0e-3
    rf, _ = synth.point_frame(acq, xs, zs)
    lam = acq.c_mps / acq.f0_hz
    nx, nz = 61, 201
    grid = (nx, nz, xs - 0.6e-3, xs + 0.6e-3, zs - 1.5e-3, zs + 1.5e-3)
    out = oracle.beamform(rf, acq.x_elements(), acq.angles_rad, grid, acq.fs_hz, acq.c_mps, 1.5)
    # The DMAS image is localised before its [f0, 3 f0] band-pass: with signed square roots the
    # second-harmonic content of s_i s_j grows with the phase spread between channels, so the
    # band-passed lateral profile of a point dips at the target itself (the band-pass mask is
    # pinned separately by the bin-centred cosine test).
    env = oracle.envelope(out[mode])
    ix, iz = np.unravel_index(np.argmax(env), env.shape)
    X, Z = oracle.grid_coords(grid)
    err = math.hypot(X[ix] - xs, Z[iz] - zs)
    assert err <= lam / 4, (mode, deg, err)


# ------------------------------------------------------------------ pDAS --

def test_pdas_constant_record_closed_form(golden_dir):
    """u = c everywhere, M channels in range: yt = M c^(1/p), pDAS = M^p c per
    angle (Eq. (2)-(3)); the sign of c is kept; angles add."""
    spec = _load(golden_dir, "aperture_counts.json")
    n = spec["n_elements"]
    xe = (np.arange(n) - 0.5 * (n - 1)) * spec["pitch_m"]
    rb = spec["record_bound"]
    x, z = rb["pixel_m"]
    m_in = rb["count"]
    rf = np.full((1, n, rb["n_samples"]), 1000, np.int16)
    grid = _single_pixel_grid(x, z)
    for p in (1.0, 2.0, 3.0, 1.7):
        y = oracle.beamform_pdas(rf, xe, [0.0], grid, rb["fs_hz"], rb["c_mps"], spec["f_number"], p)
        assert y[0, 0] == pytest.approx(m_in ** p * 1000.0, rel=1e-12), p
    m_ap = spec["cases"][0]["count"]
    rf = np.full((3, n, 4096), -7, np.int16)
    th = np.deg2rad([-5.0, 0.0, 5.0])
    y = oracle.beamform_pdas(rf, xe, th, grid, 20e6, 1540.0, 1.5, 2.0)
    assert y[0, 0] == pytest.approx(-7.0 * 3 * m_ap ** 2, rel=1e-12)


def _speckle_case():
    acq = synth.SPECKLE_POINTS_128.with_(nx=9, nz=7, n_elements=16, n_samples=1024,
                                         angles_deg=(-5.0, 3.0))
    rf, _ = synth.speckle_points_frame(acq)
    grid = (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)
    return acq, rf, grid


def test_pdas_p1_is_das_and_single_channel_is_the_sample():
    """p = 1: no compression, pDAS = DAS.  One receive element: the root and
    the power cancel for every p, pDAS = DAS = the delayed sample."""
    acq, rf, grid = _speckle_case()
    xe = acq.x_elements()
    ref = oracle.beamform(rf, xe, acq.angles_rad, grid, acq.fs_hz, acq.c_mps, acq.f_number)
    y1 = oracle.beamform_pdas(rf, xe, acq.angles_rad, grid, acq.fs_hz, acq.c_mps, acq.f_number, 1.0)
    np.testing.assert_allclose(y1, ref["das"], rtol=1e-12, atol=1e-9)
    one = rf[:, 5:6, :]
    ref1 = oracle.beamform(one, xe[5:6], acq.angles_rad, grid, acq.fs_hz, acq.c_mps, 0.1)
    for p in (2.0, 3.0, 4.5):
        y = oracle.beamform_pdas(one, xe[5:6], acq.angles_rad, grid, acq.fs_hz, acq.c_mps, 0.1, p)
        np.testing.assert_allclose(y, ref1["das"], rtol=1e-10, atol=1e-9)


def test_pdas_homogeneous_odd_and_brute_force():
    """pDAS(2 u) = 2 pDAS(u) (degree-1 homogeneous: (2^(1/p))^p = 2),
    pDAS(-u) = -pDAS(u), and a per-channel numpy evaluation of Eq. (2)-(3)
    from the delayed samples agrees."""
    acq, rf, grid = _speckle_case()
    rf = (rf // 4).astype(np.int16)
    xe = acq.x_elements()
    args = (xe, acq.angles_rad, grid, acq.fs_hz, acq.c_mps, acq.f_number)
    for p in (2.0, 3.0):
        y = oracle.beamform_pdas(rf, *args, p)
        y2 = oracle.beamform_pdas((2 * rf).astype(np.int16), *args, p)
        yn = oracle.beamform_pdas((-rf).astype(np.int16), *args, p)
        np.testing.assert_allclose(y2, 2 * y, rtol=1e-9, atol=1e-6 * np.max(np.abs(y)))
        np.testing.assert_allclose(yn, -y, rtol=1e-12, atol=0)
        for ix, iz in ((0, 0), (4, 3), (8, 6), (2, 5)):
            v, act, _ = oracle.delayed_samples(rf, xe, acq.angles_rad, grid, ix, iz, acq.fs_hz,
                                               acq.c_mps, acq.f_number)
            expect = 0.0
            for a in range(v.shape[0]):
                s = np.sum(np.sign(v[a][act[a]]) * np.abs(v[a][act[a]]) ** (1.0 / p))
                expect += np.sign(s) * abs(s) ** p
            assert y[ix, iz] == pytest.approx(expect, rel=1e-10, abs=1e-9)


# ---------------------------------------------------------- IQ / BB-DMAS --

def test_demodulation_of_a_bin_centred_tone_is_constant():
    """u[k] = A cos(2 pi k0 k / Ns + phi) on an exact bin, demodulated at
    f0 / fs = k0 / Ns: the analytic signal is A exp(j(2 pi k0 k / Ns + phi)),
    so the baseband record is the constant A exp(j phi)."""
    ns, k0, amp, phi = 512, 64, 3.0, 0.7
    k = np.arange(ns)
    u = amp * np.cos(2 * np.pi * k0 * k / ns + phi)
    iq = oracle.demodulate(u, fs=1.0, f0=k0 / ns)
    np.testing.assert_allclose(iq, amp * np.exp(1j * phi) * np.ones(ns), rtol=0, atol=1e-12)
    # a tone above the carrier keeps rotating at the difference frequency
    iq2 = oracle.demodulate(np.cos(2 * np.pi * 80 * k / ns), fs=1.0, f0=k0 / ns)
    np.testing.assert_allclose(iq2, np.exp(2j * np.pi * 16 * k / ns), rtol=0, atol=1e-12)


def test_iq_das_and_bb_dmas_hand_derived_case(golden_dir):
    spec = _load(golden_dir, "iq_cases.json")
    geo = _load(golden_dir, "geometry_cases.json")["cases"]
    steer = [c for c in geo if c["name"].startswith("3-4-5, wave steered")]
    assert len(steer) == 2
    ns, k0, amp = spec["n_samples"], spec["bin"], spec["amplitude"]
    k = np.arange(ns)
    u = np.rint(amp * np.cos(2 * np.pi * k0 * k / ns)).astype(np.int16)
    rf = np.stack([u[None, :], u[None, :]])  # [A=2][N=1][Ns]
    fs, c = steer[0]["fs_hz"], steer[0]["c_mps"]
    f0 = spec["f0_over_fs"] * fs
    angles = [steer[0]["angles_rad"][0], steer[1]["angles_rad"][0]]
    iq = oracle.demodulate(rf, fs, f0)
    out = oracle.beamform_iq(iq, [0.0], angles, _single_pixel_grid(0.003, 0.004), fs, c, 0.5, f0)
    r1 = k0 / ns
    expect_das = 2 * amp * abs(math.cos(math.pi * r1 * 45))
    expect_dmas = 2 * amp * abs(math.cos(2 * math.pi * r1 * 45))
    assert expect_das == pytest.approx(spec["expect_iq_das"], rel=1e-8)
    assert expect_dmas == pytest.approx(spec["expect_bb_dmas"], rel=1e-8)
    assert out["iqdas"][0, 0] == pytest.approx(expect_das, rel=1e-3)
    assert out["bbdmas"][0, 0] == pytest.approx(expect_dmas, rel=1e-3)


def _iq_case():
    acq = synth.SPECKLE_POINTS_128.with_(nx=9, nz=7, n_elements=16, n_samples=1024,
                                         angles_deg=(-5.0, 3.0))
    rf, _ = synth.speckle_points_frame(acq)
    grid = (acq.nx, acq.nz, acq.x0_m, acq.x1_m, acq.z0_m, acq.z1_m)
    return acq, rf, grid


def test_iq_combiners_against_a_numpy_evaluation():
    """Delays from a ramp record (linear interpolation returns n itself), then
    baseband interpolation, carrier restoration and both combiners in numpy."""
    acq, rf, grid = _iq_case()
    xe = acq.x_elements()
    iq = oracle.demodulate(rf, acq.fs_hz, acq.f0_hz)
    out = oracle.beamform_iq(iq, xe, acq.angles_rad, grid, acq.fs_hz, acq.c_mps, acq.f_number,
                             acq.f0_hz)
    ramp = np.broadcast_to(np.arange(acq.n_samples, dtype=np.int16), rf.shape).copy()
    for ix, iz in ((0, 0), (4, 3), (8, 6), (2, 5), (6, 1)):
        n, act, rec = oracle.delayed_samples(ramp, xe, acq.angles_rad, grid, ix, iz, acq.fs_hz,
                                             acq.c_mps, acq.f_number)
        y1 = 0j
        y2 = 0j
        for a in range(n.shape[0]):
            t = 0j
            for i in range(n.shape[1]):
                if not (act[a, i] and rec[a, i]):
                    continue
                k = int(math.floor(n[a, i]))
                al = n[a, i] - k
                b = (1 - al) * iq[a, i, k] + al * iq[a, i, k + 1]
                s = b * np.exp(2j * np.pi * acq.f0_hz * n[a, i] / acq.fs_hz)
                y1 += s
                if abs(s) > 0:
                    t += s / math.sqrt(abs(s))
            m = int(act[a].sum())
            if m:
                y2 += (t / m) ** 2
        assert out["iqdas"][ix, iz] == pytest.approx(abs(y1), rel=1e-9, abs=1e-9)
        assert out["bbdmas"][ix, iz] == pytest.approx(abs(y2), rel=1e-9, abs=1e-9)


def test_iq_images_are_homogeneous_and_single_channel_bb_dmas_is_the_magnitude():
    """|IQ-DAS| and |BB-DMAS| are degree-1 homogeneous in the record; with one
    receive element and one angle, |BB-DMAS| = |s| = |IQ-DAS|."""
    acq, rf, grid = _iq_case()
    xe = acq.x_elements()
    args = (xe, acq.angles_rad, grid, acq.fs_hz, acq.c_mps, acq.f_number, acq.f0_hz)
    iq = oracle.demodulate(rf, acq.fs_hz, acq.f0_hz)
    o1 = oracle.beamform_iq(iq, *args)
    o3 = oracle.beamform_iq(3.0 * iq, *args)
    np.testing.assert_allclose(o3["iqdas"], 3 * o1["iqdas"], rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(o3["bbdmas"], 3 * o1["bbdmas"], rtol=1e-12, atol=1e-9)
    one = oracle.beamform_iq(iq[:1, 5:6], xe[5:6], acq.angles_rad[:1], grid, acq.fs_hz, acq.c_mps,
                             0.1, acq.f0_hz)
    np.testing.assert_allclose(one["bbdmas"], one["iqdas"], rtol=1e-12, atol=1e-9)
