"""Plane-wave f-k migration (bf_fkmig) on the GPU against the FP64 oracle:
the exact plane-wave mapping (oracle.fk_migrate) and Stolt's (BF_FK_STOLT,
oracle.fk_stolt).

The GPU transforms are FP32 (time length nt up to 8192, lateral nk); the
mapping's bin position and decisions are double precision on both sides (the
library tabulates them on the host: no double-precision arithmetic runs on
the GPU).
Bound (derived from the arithmetic): four FP32 transform stages of relative
error ~log2(n) * 6e-8 each give a few 1e-6 of the image's RMS, so rel-L2
<= 2e-5 over the image and per pixel <= 1e-4 of its peak.
"""
import numpy as np
import pytest

import oracle
import paper_2311_00482_gb300 as bf
import synth
from test_gpu_parity import make_handle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch

    from paper_2311_00482_gb300 import build as bfbuild

    bfbuild.build()
    bf.load()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    return torch


def run_fk(torch, acq, rf, flags=bf.BF_OUT_RF):
    h = make_handle(acq)
    try:
        rf_d = torch.from_numpy(np.ascontiguousarray(rf)).cuda()
        out = torch.full((acq.n_elements, rf.shape[2]), float("nan"), device="cuda")
        bf.bf_fkmig(h, rf_d, rf.shape[2], acq.angles_rad, flags, out)
        bf.bf_sync(h)
        return out.cpu().numpy().astype(np.float64)
    finally:
        bf.bf_destroy(h)


def check(got, ref, what):
    assert np.all(np.isfinite(got)), what
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 2e-5, "%s: rel-L2 %.3e" % (what, err)
    assert np.max(np.abs(got - ref)) <= 1e-4 * np.max(ref), what


@pytest.mark.parametrize("angles", [(0.0,), (10.0,), (-7.0, 0.0, 7.0)])
def test_fk_matches_oracle(torch, angles):
    acq = synth.CYST_WIRES_512.with_(n_samples=2048, angles_deg=angles)
    rf, _ = synth.cyst_wires_frame(acq)
    ref = oracle.fk_migrate(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    got = run_fk(torch, acq, rf)
    assert got.shape == ref.shape == (64, 2048)
    check(got, ref, "fk %s" % (angles,))


@pytest.mark.parametrize("angles", [(0.0,), (10.0,), (-7.0, 0.0, 7.0)])
def test_stolt_matches_oracle(torch, angles):
    acq = synth.CYST_WIRES_512.with_(n_samples=2048, angles_deg=angles)
    rf, _ = synth.cyst_wires_frame(acq)
    ref = oracle.fk_stolt(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    got = run_fk(torch, acq, rf, bf.BF_OUT_RF | bf.BF_FK_STOLT)
    assert got.shape == ref.shape == (64, 2048)
    check(got, ref, "stolt %s" % (angles,))


def test_mappings_alternate_on_one_handle(torch):
    """The mapping tables follow the flags, the angles and the sample count from
    call to call on one handle."""
    acq = synth.SPECKLE_POINTS_128.with_(n_elements=64, n_samples=1024, angles_deg=(6.0,))
    rf, _ = synth.speckle_points_frame(acq)
    h = make_handle(acq)
    try:
        rf_d = torch.from_numpy(rf).cuda()
        out = torch.zeros((64, 1024), device="cuda")
        cases = [(bf.BF_FK_STOLT, oracle.fk_stolt), (0, oracle.fk_migrate),
                 (bf.BF_FK_STOLT, oracle.fk_stolt)]
        for flags, fn in cases:
            bf.bf_fkmig(h, rf_d, 1024, acq.angles_rad, flags, out)
            bf.bf_sync(h)
            check(out.cpu().numpy().astype(np.float64),
                  fn(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps), "alternating")
        rf2 = rf[:, :, :800].copy()
        bf.bf_fkmig(h, torch.from_numpy(rf2).cuda(), 800, [-6.0 * np.pi / 180], bf.BF_FK_STOLT,
                    out)
        bf.bf_sync(h)
        got = out.view(-1)[:64 * 800].view(64, 800).cpu().numpy().astype(np.float64)
        check(got, oracle.fk_stolt(rf2, acq.pitch_m, np.array([-6.0 * np.pi / 180]), acq.fs_hz,
                                   acq.c_mps), "800 samples")
    finally:
        bf.bf_destroy(h)


def test_fk_odd_sizes_and_log(torch):
    """47 elements (nk = 128), 1000 samples (nt = 2048, not a multiple of anything)."""
    acq = synth.SPECKLE_POINTS_128.with_(n_elements=47, n_samples=1000, angles_deg=(4.0,))
    rf, _ = synth.speckle_points_frame(acq)
    ref = oracle.fk_migrate(rf, acq.pitch_m, acq.angles_rad, acq.fs_hz, acq.c_mps)
    got = run_fk(torch, acq, rf)
    check(got, ref, "fk odd")
    db = run_fk(torch, acq, rf, bf.BF_OUT_LOGDB)
    assert np.max(np.abs(db - oracle.log_compress(ref))) <= 0.05


def test_fk_point_targets_in_place(torch):
    acq = synth.Acquisition(n_elements=64, n_samples=1024, angles_deg=(10.0,))
    lam = acq.c_mps / acq.f0_hz
    for xp, zp in ((0.0, 15e-3), (3e-3, 22e-3)):
        rf, _ = synth.point_frame(acq, xp, zp)
        img = run_fk(torch, acq, rf)
        i, m = np.unravel_index(np.argmax(img), img.shape)
        assert abs((i - 31.5) * acq.pitch_m - xp) <= 0.5 * acq.pitch_m + 1e-9
        assert abs(m * acq.c_mps / (2 * acq.fs_hz) - zp) <= lam / 4


def test_fk_argument_checks(torch):
    acq = synth.SPECKLE_POINTS_128
    h = make_handle(acq)
    try:
        rf = torch.zeros((1, 64, 1024), dtype=torch.int16, device="cuda")
        out = torch.zeros((64, 1024), device="cuda")
        for flags in (bf.BF_DAS, bf.BF_PREC_FP16, bf.BF_IQDAS, bf.BF_FK_STOLT | bf.BF_DMAS):
            with pytest.raises(bf.BFError):
                bf.bf_fkmig(h, rf, 1024, [0.0], flags, out)
        big = torch.zeros((1, 64, 5000), dtype=torch.int16, device="cuda")
        with pytest.raises(bf.BFError):
            bf.bf_fkmig(h, big, 5000, [0.0], 0, torch.zeros((64, 5000), device="cuda"))
    finally:
        bf.bf_destroy(h)
